"""Seeded synthetic flow fields shaped like the paper's workloads.

This module is shared by the CPU oracle and the GPU path as the single source of
inputs. It holds no arithmetic of the discretisation: it only evaluates the
closed-form fields in primitive variables (density, velocity, pressure) at points
the caller supplies (initial states, and the exact steady solutions of Secs.
5.1-5.2 with the Couette flow's source term), and draws the seeded random numbers
(vortex positions and strengths, trace perturbations, per-element degrees).

Nondimensionalisation: freestream (or reference) density 1, speed 1, length 1,
so p_inf = 1 / (gamma M^2).

Sources in the paper:
  * isentropic (Shu) vortex, Sec. 5.4 "Case description". The printed density
    factor psi^2 M_inf is read as psi^2 M_inf^2: only the squared Mach number
    gives radial equilibrium dp/dr = rho u_theta^2 / r together with the printed
    isentropic pressure law (checked in tests/test_oracle_convergence.py).
  * Taylor-Green vortex, Sec. 5.5, Eq. (initialCondTGV), with rho0 = V0 = L = 1
    and P0 = 1 / (gamma M0^2) (M0 = V0 / c0).
  * Couette flow with its source term, Sec. 5.2, with V0 = L = 1 and P0 = 1 / (gamma M0^2).
  * Ringleb flow, Sec. 5.1 (the standard hodograph form; the printed one is garbled).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = 1.4


def _min_image(d: np.ndarray, period: float) -> np.ndarray:
    """Signed offset reduced to the nearest periodic image."""
    return d - period * np.round(d / period)


@dataclass(frozen=True)
class Vortex:
    x0: float
    y0: float
    psi: float


def vortex_field(x: np.ndarray, vortices: list[Vortex], mach: float,
                 vinf=(1.0, 0.0), period: float | None = None, t: float = 0.0,
                 gamma: float = GAMMA):
    """Superposed isentropic vortices advected by the free stream.

    x: [..., 2] points. Returns (rho [...], vel [..., 2], p [...]).
    Each vortex adds the velocity perturbation psi/(2 pi) e^{1-r^2} (-y', x')
    and an enthalpy deficit (gamma-1) M^2 psi^2 e^{2(1-r^2)} / (16 pi^2); the
    density follows from the isentropic law and p = rho^gamma / (gamma M^2).
    With one vortex this is the Shu vortex of Sec. 5.4 (with M^2, see above).
    """
    x = np.asarray(x, dtype=np.float64)
    vinf = np.asarray(vinf, dtype=np.float64)
    h = np.ones(x.shape[:-1])
    vel = np.broadcast_to(vinf, x.shape).copy()
    for vt in vortices:
        dx = x[..., 0] - vt.x0 - vinf[0] * t
        dy = x[..., 1] - vt.y0 - vinf[1] * t
        if period is not None:
            dx = _min_image(dx, period)
            dy = _min_image(dy, period)
        r2 = dx * dx + dy * dy
        e1 = np.exp(1.0 - r2)
        amp = vt.psi / (2.0 * math.pi) * e1
        vel[..., 0] -= amp * dy
        vel[..., 1] += amp * dx
        h -= (gamma - 1.0) * mach ** 2 * vt.psi ** 2 * e1 * e1 / (16.0 * math.pi ** 2)
    rho = h ** (1.0 / (gamma - 1.0))
    p = rho ** gamma / (gamma * mach ** 2)
    return rho, vel, p


def draw_vortices(n: int, period: float, seed: int, psi_lo=1.0, psi_hi=5.0) -> list[Vortex]:
    """n vortices with centres uniform in [0, period)^2 and strengths U[psi_lo, psi_hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xy = rng.uniform(0.0, period, size=(n, 2))
    psi = rng.uniform(psi_lo, psi_hi, size=n)
    return [Vortex(float(a), float(b), float(s)) for (a, b), s in zip(xy, psi)]


def tgv_field(x: np.ndarray, mach: float, gamma: float = GAMMA):
    """Taylor-Green vortex initial state (Sec. 5.5) with rho0 = V0 = L = 1."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    rho = np.ones(X.shape)
    vel = np.stack([np.sin(X) * np.cos(Y) * np.cos(Z),
                    -np.cos(X) * np.sin(Y) * np.cos(Z),
                    np.zeros(X.shape)], axis=-1)
    p0 = 1.0 / (gamma * mach ** 2)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    return rho, vel, p


def couette_field(x: np.ndarray, mach: float, prandtl: float = 0.71, alpha: float = 0.8,
                  beta: float = 0.85, L: float = 1.0, gamma: float = GAMMA):
    """Steady compressible Couette flow of Sec. 5.2 on (0, L)^2 with V0 = 1, P0 = 1/(gamma M^2)
    (so T0 = 1 and rho0 = 1 in this nondimensionalisation): V_x = ybar log(1 + ybar), V_y = 0,
    p = P0, T = alpha + ybar (beta - alpha) + Pr (gamma - 1) M^2 ybar (1 - ybar) / 2 (the paper's
    V0^2 Pr / (2 c_v gamma) with c_v = 1/(gamma (gamma - 1) M^2)), rho = 1 / T (ideal gas).
    Accepts complex points (complex-step derivatives of the exact state)."""
    x = np.asarray(x)
    yb = x[..., 1] / L
    T = alpha + yb * (beta - alpha) + 0.5 * prandtl * (gamma - 1.0) * mach ** 2 * yb * (1.0 - yb)
    vel = np.stack([yb * np.log1p(yb), np.zeros_like(yb)], axis=-1)
    p = np.full(yb.shape, 1.0 / (gamma * mach ** 2)) + 0.0 * yb
    return 1.0 / T, vel, p


def couette_source(x: np.ndarray, mu: float, L: float = 1.0):
    """The source s [..., 4] (conservative components) that makes couette_field a steady solution
    of d u/dt + div(F + G) = s with constant mu, kappa = c_p mu / Pr and Stokes' hypothesis. Only
    y-derivatives survive: s_momx = -d/dy(mu V_x'), s_energy = -d/dy(mu V_x V_x' + kappa T'), where
    kappa T'' = -mu / L^2 by the choice of T's quadratic term; this is the source the paper prints
    for the problem (V0 = 1)."""
    yb = np.asarray(x)[..., 1] / L
    lg = np.log1p(yb)
    d1 = lg + yb / (1.0 + yb)                      # L V_x'
    d2 = (2.0 + yb) / (1.0 + yb) ** 2              # L^2 V_x''
    s = np.zeros(yb.shape + (4,), dtype=np.result_type(yb, np.float64))
    s[..., 1] = -mu / L ** 2 * d2
    s[..., 3] = -mu / L ** 2 * (d1 * d1 + yb * lg * d2 - 1.0)
    return s


def _ringleb_J(c):
    return 1.0 / c + 1.0 / (3.0 * c ** 3) + 1.0 / (5.0 * c ** 5) - 0.5 * np.log((1.0 + c) / (1.0 - c))


def ringleb_field(x: np.ndarray, gamma: float = GAMMA):
    """Ringleb flow (Sec. 5.1), the hodograph solution of the steady Euler equations for
    gamma = 1.4 (Chiocchia 1985), with rho0 V0^2 = rho E0: at speed q the sound speed is
    c = sqrt(1 - q^2/5), rho = c^5 and p = rho^gamma / gamma; q solves
    (x - J/2)^2 + y^2 = 1 / (4 rho^2 q^4),  J = 1/c + 1/(3c^3) + 1/(5c^5) - ln((1+c)/(1-c))/2
    on the subsonic branch (found by bisection between 0 and the sonic speed sqrt(5/6)), and the
    flow angle is theta = arcsin(psi q), psi = sqrt(1/(2 q^2) - rho (x - J/2)).
    The printed forms of the first equation and of J are garbled (a squared A inside the bracket,
    the bracket not squared, c^2 in J's second term); this is the standard form, which balances
    the Euler fluxes exactly (tests/test_oracle_ringleb.py)."""
    x = np.asarray(x, dtype=np.float64)
    X, Y = x[..., 0], x[..., 1]

    def f(q):
        c = np.sqrt(1.0 - q * q / 5.0)
        return (X - 0.5 * _ringleb_J(c)) ** 2 + Y * Y - 1.0 / (4.0 * c ** 10 * q ** 4)
    lo = np.full(X.shape, 1e-3)
    hi = np.full(X.shape, math.sqrt(5.0 / 6.0))
    if np.any(f(lo) >= 0.0) or np.any(f(hi) <= 0.0):
        raise ValueError("ringleb_field: point outside the subsonic region of the flow")
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        neg = f(mid) < 0.0
        lo, hi = np.where(neg, mid, lo), np.where(neg, hi, mid)
    q = 0.5 * (lo + hi)
    c = np.sqrt(1.0 - q * q / 5.0)
    rho = c ** 5
    psi = np.sqrt(1.0 / (2.0 * q * q) - rho * (X - 0.5 * _ringleb_J(c)))
    th = np.arcsin(psi * q)
    vel = np.stack([q * np.cos(th), q * np.sin(th)], axis=-1)
    return rho, vel, rho ** gamma / gamma


def uniform_noise(shape, seed: int) -> np.ndarray:
    """Seeded U(-1, 1) numbers (PCG64), e.g. for relative trace perturbations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=shape)


def perturb(arr: np.ndarray, eps: float, seed: int) -> np.ndarray:
    """arr + eps * scale_c * U(-1, 1), additive, with one scale per state component c:
    max |arr[..., c]| for the first and last component and the max over all middle
    (momentum-like) components for the others. Additive noise moves exactly vanishing
    components (e.g. V_z = 0 of the Taylor-Green state) away from zero, so no face point
    sits on the kink of |V.n|."""
    arr = np.asarray(arr, dtype=np.float64)
    axes = tuple(range(arr.ndim - 1))
    s = np.abs(arr).max(axis=axes)
    if s.size > 2:
        s[1:-1] = s[1:-1].max()
    return arr + eps * s * uniform_noise(arr.shape, seed)


def draw_degrees(n_elem: int, seed: int, degrees=(1, 2, 3, 4),
                 weights=(0.1, 0.3, 0.4, 0.2)) -> np.ndarray:
    """Per-element polynomial degree for the mixed-degree batch (int8)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.choice(np.asarray(degrees, dtype=np.int8), size=n_elem,
                      p=np.asarray(weights, dtype=np.float64))


# ---------------------------------------------------------------------------
# Named workloads (mesh sizes, physics, seeds).
# ---------------------------------------------------------------------------
WORKLOADS = {
    # 2D Euler p=2, 8x8 periodic [0,10]^2, one Shu vortex (psi=5, M=0.5) at (5,5).
    "euler2d_p2_vortex": dict(dim=2, n=8, lo=0.0, hi=10.0, p=2, viscous=False,
                              mach=0.5, reynolds=0.0, prandtl=0.71, dt=0.05, bdf=1,
                              seed=1),
    # 2D NS p=4, 64x64 periodic, 16 vortices, M=0.3, Re=1000, Pr=0.72, BDF2 dt=0.01.
    "ns2d_p4_vortices": dict(dim=2, n=64, lo=0.0, hi=80.0, p=4, viscous=True,
                             mach=0.3, reynolds=1000.0, prandtl=0.72, dt=0.01, bdf=2,
                             seed=2, n_vortices=16),
    # 3D NS p=3 tets, 24^3 periodic cube [0,2pi]^3, TGV M0=0.1 Re=1600.
    "ns3d_p3_tgv": dict(dim=3, n=24, lo=0.0, hi=2.0 * math.pi, p=3, viscous=True,
                        mach=0.1, reynolds=1600.0, prandtl=0.71, dt=0.01, bdf=2,
                        seed=3, trace_noise=1e-3),
    # 3D NS tets of mixed degree, 32^3 periodic cube [0,2pi]^3 (196,608 tets), degree per element
    # drawn from {1,2,3,4} with weights 0.1/0.3/0.4/0.2 (seed 4), TGV M0=0.1 Re=1600.
    "ns3d_mixed_tgv": dict(dim=3, n=32, lo=0.0, hi=2.0 * math.pi, p=4, viscous=True,
                           mach=0.1, reynolds=1600.0, prandtl=0.71, dt=0.01, bdf=2,
                           seed=3, trace_noise=1e-3, p_draw=((1, 2, 3, 4), (0.1, 0.3, 0.4, 0.2), 4)),
    # 2D NS p=3, 128x128 periodic, 32 vortices, M=0.5, Re=5000 (learned warm start).
    "ns2d_p3_vortices": dict(dim=2, n=128, lo=0.0, hi=160.0, p=3, viscous=True,
                             mach=0.5, reynolds=5000.0, prandtl=0.71, dt=0.01, bdf=2,
                             seed=5, n_vortices=32),
    # the same flow on a 16x16 patch (same h, 4 vortices): the learned-warm-start test case
    "ns2d_p3_vortices_small": dict(dim=2, n=16, lo=0.0, hi=20.0, p=3, viscous=True,
                                   mach=0.5, reynolds=5000.0, prandtl=0.71, dt=0.01, bdf=2,
                                   seed=5, n_vortices=4),
}


def primitive_state(name: str, x: np.ndarray, **over):
    """Evaluate the named workload's initial primitive state at points x."""
    w = dict(WORKLOADS[name]); w.update(over)
    if w["dim"] == 3:
        return tgv_field(x, w["mach"])
    period = w["hi"] - w["lo"]
    if "n_vortices" in w:
        vs = draw_vortices(w["n_vortices"], period, w["seed"])
    else:
        c = 0.5 * (w["lo"] + w["hi"])
        vs = [Vortex(c, c, 5.0)]
    return vortex_field(x, vs, w["mach"], period=period)


def draw_degrees(name: str, n_elem: int):
    """Per-element degrees of a mixed-degree workload (seeded draw), or None."""
    w = WORKLOADS[name]
    if "p_draw" not in w:
        return None
    degs, weights, seed = w["p_draw"]
    return np.random.default_rng(seed).choice(degs, size=n_elem, p=weights).astype(np.int8)
