"""Pointwise physics for the oracle; every function accepts complex arrays so that
the residual can be differentiated by complex step.

State layout: last axis is the component (m = d + 2): (rho, rho V_1..d, rho E) for
u and (v_1, v_2..v_{d+1}, v_m) for the entropy variables.

Nondimensionalisation (freestream density, speed and length 1): p_inf = 1/(gamma M^2),
c_v = 1/(gamma (gamma-1) M^2), c_p = gamma c_v, mu = 1/Re, kappa = c_p mu / Pr, beta = 0
(Sec. 2.2, Eq. closuresNS; Sec. 5 for Pr, gamma, beta).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Physics:
    gamma: float = 1.4
    mach: float = 0.5
    reynolds: float = 0.0            # 0 = inviscid (Euler)
    prandtl: float = 0.71
    mu_exponent: float = 0.0         # power law mu = (1/Re) (T / T_inf)^omega (Sec. 5.6 uses 3/4); 0: constant
    stabilization: str = "slf"       # "slf": sigma_SLF of Eq. sLxF (Sec. 5); "s": sigma_S of Eq. symStab

    @property
    def viscous(self) -> bool:
        return self.reynolds > 0

    @property
    def cv(self) -> float:
        return 1.0 / (self.gamma * (self.gamma - 1.0) * self.mach ** 2)

    @property
    def mu(self) -> float:
        return 1.0 / self.reynolds if self.reynolds > 0 else 0.0

    @property
    def kappa(self) -> float:
        return self.gamma * self.cv * self.mu / self.prandtl

    def viscosity_factor(self, vm):
        """(T / T_inf)^omega at entropy variable v_m, T = 1 / (c_v (-v_m)); the freestream
        temperature of this nondimensionalisation is T_inf = p_inf / ((gamma - 1) c_v) = 1."""
        if self.mu_exponent == 0.0:
            return 1.0
        return (1.0 / (self.cv * (-vm))) ** self.mu_exponent


def cabs(x):
    """|x| continued for complex step with d|x|/dx = sign(x), sign(0) = 0."""
    re = np.real(x)
    return x * np.sign(re)


# -- conservation <-> entropy variables (Sec. 2.3) --------------------------------------
def primitives_of_u(u, gamma):
    rho = u[..., 0]
    vel = u[..., 1:-1] / rho[..., None]
    p = (gamma - 1.0) * (u[..., -1] - 0.5 * rho * np.sum(vel * vel, axis=-1))
    return rho, vel, p


def u_of_primitives(rho, vel, p, gamma):
    rhoE = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=-1)
    return np.concatenate([rho[..., None], rho[..., None] * vel, rhoE[..., None]], axis=-1)


def thermo_entropy(rho, p, gamma):
    """s = log(p / rho^gamma) with baseline s_0 = 0 (Sec. 2.3)."""
    return np.log(p) - gamma * np.log(rho)


def v_of_u(u, gamma):
    """Entropy variables v = dH/du for H = -rho s, as printed in Sec. 2.3."""
    rho, vel, p = primitives_of_u(u, gamma)
    s = thermo_entropy(rho, p, gamma)
    g1 = gamma - 1.0
    v1 = -s + (gamma + 1.0) - g1 * u[..., -1] / p
    vmid = g1 * u[..., 1:-1] / p[..., None]
    vm = -g1 * rho / p
    return np.concatenate([v1[..., None], vmid, vm[..., None]], axis=-1)


def primitives_of_v(v, gamma):
    """Inverse map (not printed in the paper): from the printed v(u),
    s = gamma - v_1 + |w|^2/(2 v_m), log rho = (log(gamma-1) - log(-v_m) - s)/(gamma-1),
    p = rho (gamma-1)/(-v_m), V = -w / v_m, with w = (v_2..v_{d+1})."""
    g1 = gamma - 1.0
    v1, w, vm = v[..., 0], v[..., 1:-1], v[..., -1]
    s = gamma - v1 + np.sum(w * w, axis=-1) / (2.0 * vm)
    lnrho = (np.log(g1) - np.log(-vm) - s) / g1
    rho = np.exp(lnrho)
    p = rho * g1 / (-vm)
    vel = -w / vm[..., None]
    return rho, vel, p


def u_of_v(v, gamma):
    rho, vel, p = primitives_of_v(v, gamma)
    return u_of_primitives(rho, vel, p, gamma)


def du_of_v(v, dv, gamma):
    """Directional derivative A0(v) dv of u(v) along dv, written out by the chain rule
    on the inverse map (A0 = du/dv is the metric tensor of Sec. 4.1)."""
    g1 = gamma - 1.0
    rho, vel, p = primitives_of_v(v, gamma)
    w, vm = v[..., 1:-1], v[..., -1]
    dv1, dw, dvm = dv[..., 0], dv[..., 1:-1], dv[..., -1]
    ww = np.sum(w * w, axis=-1)
    ds = -dv1 + np.sum(w * dw, axis=-1) / vm - ww * dvm / (2.0 * vm * vm)
    dlnrho = (-dvm / vm - ds) / g1
    drho = rho * dlnrho
    dvel = -dw / vm[..., None] + w * (dvm / (vm * vm))[..., None]
    dp = p * (dlnrho - dvm / vm)
    dmom = drho[..., None] * vel + rho[..., None] * dvel
    dE = dp / g1 + 0.5 * drho * np.sum(vel * vel, axis=-1) + rho * np.sum(vel * dvel, axis=-1)
    return np.concatenate([drho[..., None], dmom, dE[..., None]], axis=-1)


def A0_of_v(v, gamma):
    """A0 = du/dv as a matrix [..., m, m] (row = u component)."""
    m = v.shape[-1]
    cols = [du_of_v(v, np.broadcast_to(np.eye(m)[l], v.shape), gamma) for l in range(m)]
    return np.stack(cols, axis=-1)


# -- fluxes (Eqs. flux, viscFlux, closuresNS) ------------------------------------------
def inviscid_flux_prim(rho, vel, p, gamma):
    """F(u) [..., m, d]: rows (rho V_j, rho V_i V_j + delta_ij p, V_j (rho E + p))."""
    d = vel.shape[-1]
    rhoE = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=-1)
    rows = [rho[..., None] * vel]
    for i in range(d):
        r = rho[..., None] * vel[..., i:i + 1] * vel
        r = r + p[..., None] * np.eye(d)[i]
        rows.append(r)
    rows.append(vel * (rhoE + p)[..., None])
    return np.stack(rows, axis=-2)


def inviscid_flux_v(v, gamma):
    rho, vel, p = primitives_of_v(v, gamma)
    return inviscid_flux_prim(rho, vel, p, gamma)


def inviscid_flux_u(u, gamma):
    rho, vel, p = primitives_of_u(u, gamma)
    return inviscid_flux_prim(rho, vel, p, gamma)


def viscous_flux(v, q, phys: Physics):
    """G(v, q) [..., m, d] of Eq. viscFlux with q ~ grad v (Sec. 3.3).

    The matrices K_jk are not printed; G is evaluated through the primitive gradients
    grad V_i = -grad w_i / v_m + w_i grad v_m / v_m^2 and T = 1/(c_v (-v_m)),
    grad T = grad v_m / (c_v v_m^2), which equals -K_jk (du/dv) q. With a power law
    (Physics.mu_exponent, Sec. 5.6) mu and kappa are scaled by (T / T_inf)^omega."""
    gamma = phys.gamma
    d = v.shape[-1] - 2
    w, vm = v[..., 1:-1], v[..., -1]
    vel = -w / vm[..., None]
    qw, qm = q[..., 1:-1, :], q[..., -1, :]                       # [..., d, d], [..., d]
    gradV = -qw / vm[..., None, None] + w[..., :, None] * (qm / (vm * vm)[..., None])[..., None, :]
    gradT = qm / (phys.cv * (vm * vm)[..., None])
    div = np.trace(gradV, axis1=-2, axis2=-1)
    mu_fac = phys.viscosity_factor(vm)               # mu(T) / mu_ref = kappa(T) / kappa_ref (Pr fixed)
    mu = phys.mu * mu_fac
    kappa = phys.kappa * mu_fac
    if np.ndim(mu_fac):
        mu, kappa = mu[..., None, None], kappa[..., None]
    tau = mu * (gradV + np.swapaxes(gradV, -1, -2)
                - (2.0 / 3.0) * div[..., None, None] * np.eye(d))
    f = -kappa * gradT
    zero = np.zeros(v.shape[:-1] + (1, d), dtype=tau.dtype)
    energy = np.einsum("...i,...ij->...j", vel, tau) - f
    return -np.concatenate([zero, tau, energy[..., None, :]], axis=-2)


# -- entropy pair and stabilization -------------------------------------------------------
def entropy_H(u, gamma):
    rho, _vel, p = primitives_of_u(u, gamma)
    return -rho * thermo_entropy(rho, p, gamma)


def entropy_flux(u, gamma):
    rho, vel, p = primitives_of_u(u, gamma)
    return (-rho * thermo_entropy(rho, p, gamma))[..., None] * vel


def lambda_max(v, n, gamma):
    """Largest-magnitude eigenvalue of A_n = (dF/du) n: |V.n| + c (Eq. sLxF)."""
    rho, vel, p = primitives_of_v(v, gamma)
    c = np.sqrt(gamma * p / rho)
    return cabs(np.sum(vel * n, axis=-1)) + c


def flux_jacobian_u(v, n, gamma):
    """A_n = (dF/du) . n at the state v [..., m, m] (row = flux component, column = u
    component), the textbook Jacobian of the Euler flux in conservation variables written in
    primitives: with V_n = V . n, k = |V|^2 / 2 and total enthalpy H = (rho E + p) / rho,
      mass row      (0, n, 0)
      momentum i    ((gamma-1) k n_i - V_i V_n,  V_i n_j - (gamma-1) n_i V_j + V_n delta_ij,  (gamma-1) n_i)
      energy row    (V_n ((gamma-1) k - H),  H n_j - (gamma-1) V_n V_j,  gamma V_n)."""
    g1 = gamma - 1.0
    rho, vel, p = primitives_of_v(v, gamma)
    d = vel.shape[-1]
    m = d + 2
    n = np.asarray(n, dtype=float)
    vn = np.sum(vel * n, axis=-1)
    k = 0.5 * np.sum(vel * vel, axis=-1)
    H = gamma * p / (g1 * rho) + k
    A = np.zeros(v.shape[:-1] + (m, m), dtype=np.result_type(v, float))
    A[..., 0, 1:1 + d] = n
    for i in range(d):
        A[..., 1 + i, 0] = g1 * k * n[i] - vel[..., i] * vn
        for j in range(d):
            A[..., 1 + i, 1 + j] = vel[..., i] * n[j] - g1 * n[i] * vel[..., j] + (vn if i == j else 0.0)
        A[..., 1 + i, m - 1] = g1 * n[i]
    A[..., m - 1, 0] = vn * (g1 * k - H)
    A[..., m - 1, 1:1 + d] = H[..., None] * n - g1 * vn[..., None] * vel
    A[..., m - 1, m - 1] = gamma * vn
    return A


def abs_flux_jacobian(v, n, gamma):
    """|A_n| at the state v: A_n is diagonalisable with the three distinct eigenvalues
    l_1 = V_n - c, l_2 = V_n (multiplicity d), l_3 = V_n + c (c > 0), so the matrix function
    is the Lagrange-Sylvester sum  |A_n| = sum_k |l_k| prod_{j != k} (A_n - l_j I) / (l_k - l_j)."""
    rho, vel, p = primitives_of_v(v, gamma)
    c = np.sqrt(gamma * p / rho)
    vn = np.sum(vel * np.asarray(n, dtype=float), axis=-1)
    A = flux_jacobian_u(v, n, gamma)
    eye = np.eye(A.shape[-1])
    lam = [vn - c, vn, vn + c]
    out = np.zeros_like(A)
    for kk in range(3):
        P = np.broadcast_to(eye, A.shape).astype(A.dtype)
        for j in range(3):
            if j != kk:
                P = np.einsum("...ij,...jk->...ik", P, A - lam[j][..., None, None] * eye)
                P = P / (lam[kk] - lam[j])[..., None, None]
        out = out + cabs(lam[kk])[..., None, None] * P
    return out


def numerical_flux_inviscid(vhat, v, n, gamma, stabilization="slf"):
    """Eq. numericalFlux at v* = vhat (Sec. 5) with
      "slf": sigma_SLF(v*) = lambda_max(v*) A0(v*)            (Eq. sLxF, the choice of Sec. 5)
      "s":   sigma_S(v*)   = |A_n(v*)|_{A0} = |A_n(v*)| A0(v*)  (Eq. symStab, Sec. 4.1)."""
    Fn = 0.5 * np.einsum("...ij,...j->...i", inviscid_flux_v(vhat, gamma) + inviscid_flux_v(v, gamma), n)
    du = du_of_v(vhat, v - vhat, gamma)
    if stabilization == "slf":
        lam = lambda_max(vhat, n, gamma)
        return Fn + 0.5 * lam[..., None] * du
    if stabilization == "s":
        return Fn + 0.5 * np.einsum("...ij,...j->...i", abs_flux_jacobian(vhat, n, gamma), du)
    raise ValueError(stabilization)
