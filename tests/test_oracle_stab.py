"""Pins of the oracle's symmetric variable stabilization matrix sigma_S = |A_n(v*)|_{A0} =
|A_n| A0 (Eq. symStab with the generalised absolute value of Sec. 4.1, v* = vhat):
* A_n = (dF/du) . n written out equals the complex-step derivative of the flux in
  conservation variables;
* |A_n| by the Lagrange-Sylvester sum equals R |Lambda| R^-1 from a library eigendecomposition;
* sigma_S is symmetric positive semidefinite, its eigenvalues relative to A0 are |V_n - c|,
  |V_n| (d times), |V_n + c|, and sigma_SLF - sigma_S is positive semidefinite;
* for supersonic normal flow the whole numerical flux reduces to the upwind form
  1/2 (F(vhat) + F(v)) . n + 1/2 sign(V_n) (d(F . n)/dv)(vhat) (v - vhat), the last
  Jacobian by complex step of the flux in entropy variables;
* the scheme with sigma_S is entropy stable on periodic Euler (Sec. 4, corollary (ii)):
  int H does not increase over BDF1 steps and int u is conserved."""
import numpy as np
import pytest

from oracle import physics as ph
from oracle.hdg import time_step
from test_oracle_hdg import vortex_problem

GAMMA = 1.4


def _random_states(d, count, seed, mach_range=(0.1, 0.9)):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, count)
    p = rng.uniform(0.5, 2.0, count)
    c = np.sqrt(GAMMA * p / rho)
    dirs = rng.normal(size=(count, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    vel = dirs * (c * rng.uniform(*mach_range, count))[:, None]
    n = rng.normal(size=(count, d))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    u = ph.u_of_primitives(rho, vel, p, GAMMA)
    return ph.v_of_u(u, GAMMA), u, n, c, vel


@pytest.mark.parametrize("d", [2, 3])
def test_flux_jacobian_against_complex_step(d):
    v, u, n, _, _ = _random_states(d, 8, 1 + d)
    m = d + 2
    h = 1e-30
    for s in range(len(u)):
        A = ph.flux_jacobian_u(v[s], n[s], GAMMA)
        for l in range(m):
            up = u[s].astype(complex)
            up[l] += 1j * h
            col = np.imag(ph.inviscid_flux_u(up, GAMMA) @ n[s]) / h
            assert np.abs(A[:, l] - col).max() <= 1e-12 * max(1.0, np.abs(col).max())


@pytest.mark.parametrize("d", [2, 3])
def test_abs_flux_jacobian_is_the_eigendecomposition(d):
    v, _, n, _, _ = _random_states(d, 10, 11 + d, mach_range=(0.05, 1.6))
    for s in range(len(v)):
        A = ph.flux_jacobian_u(v[s], n[s], GAMMA)
        lam, R = np.linalg.eig(A)
        assert np.abs(lam.imag).max() < 1e-12
        ref = (R * np.abs(lam.real)) @ np.linalg.inv(R)
        got = ph.abs_flux_jacobian(v[s], n[s], GAMMA)
        assert np.abs(got - ref.real).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("d", [2, 3])
def test_sigma_s_symmetric_semidefinite_with_the_absolute_spectrum(d):
    v, _, n, c, vel = _random_states(d, 10, 21 + d, mach_range=(0.05, 1.6))
    for s in range(len(v)):
        A0 = ph.A0_of_v(v[s], GAMMA)
        sig = ph.abs_flux_jacobian(v[s], n[s], GAMMA) @ A0
        scale = np.abs(sig).max()
        assert np.abs(sig - sig.T).max() <= 1e-12 * scale
        assert np.linalg.eigvalsh(0.5 * (sig + sig.T)).min() >= -1e-12 * scale
        vn = vel[s] @ n[s]
        expect = np.sort([abs(vn - c[s])] + [abs(vn)] * d + [abs(vn + c[s])])
        got = np.sort(np.linalg.eigvals(np.linalg.solve(A0, sig)).real)
        assert np.abs(got - expect).max() <= 1e-10 * expect.max()
        # sigma_SLF = lambda_max A0 dominates sigma_S
        slf = ph.lambda_max(v[s], n[s], GAMMA) * A0
        diff = slf - sig
        assert np.linalg.eigvalsh(0.5 * (diff + diff.T)).min() >= -1e-11 * scale


@pytest.mark.parametrize("d", [2, 3])
def test_sigma_s_flux_is_upwind_for_supersonic_normal_flow(d):
    rng = np.random.default_rng(31 + d)
    m = d + 2
    for s in range(6):
        n = rng.normal(size=d)
        n /= np.linalg.norm(n)
        sign = 1.0 if s % 2 == 0 else -1.0
        rho, p = rng.uniform(0.7, 1.5), rng.uniform(0.7, 1.5)
        c = np.sqrt(GAMMA * p / rho)
        vel = sign * rng.uniform(1.3, 2.0) * c * n + 0.2 * c * rng.normal(size=d)
        vh = ph.v_of_u(ph.u_of_primitives(np.array(rho), vel, np.array(p), GAMMA), GAMMA)
        v = vh * (1.0 + 1e-2 * rng.uniform(-1, 1, m))
        vn = vel @ n
        assert abs(vn) > c
        An = np.zeros((m, m))
        for l in range(m):
            z = vh.astype(complex)
            z[l] += 1e-30j
            An[:, l] = np.imag(ph.inviscid_flux_v(z, GAMMA) @ n) / 1e-30
        ref = 0.5 * (ph.inviscid_flux_v(vh, GAMMA) + ph.inviscid_flux_v(v, GAMMA)) @ n \
            + 0.5 * np.sign(vn) * An @ (v - vh)
        got = ph.numerical_flux_inviscid(vh, v, n, GAMMA, "s")
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        # the Lax-Friedrichs flux differs: it adds lambda_max A0 instead
        slf = ph.numerical_flux_inviscid(vh, v, n, GAMMA, "slf")
        assert np.abs(slf - ref).max() > 1e-6 * np.abs(ref).max()


def test_sigma_s_scheme_is_entropy_stable():
    """Periodic Euler with sigma_S, BDF1, under-resolved: int H does not increase over the
    steps and int u is conserved (corollary (ii) of Sec. 4 with the time step's convexity)."""
    phys = ph.Physics(mach=0.5, stabilization="s")
    prob, Q, V, Vh = vortex_problem(2, 3, 1, phys, L=6.0, deg=5, noise=0.0)
    u0, H0 = prob.integrals(V)
    Hs = [H0]
    Vc = V
    for step in range(3):
        res = time_step(prob, None, Vc, Vh, [Vc], 1, 0.2, tol=1e-12, max_it=10)
        Vc, Vh = res.V, res.Vhat
        u, Hc = prob.integrals(Vc)
        assert np.allclose(u, u0, rtol=0, atol=1e-10 * np.abs(u0).max())
        Hs.append(Hc)
    for a, b in zip(Hs, Hs[1:]):
        assert b <= a + 1e-12 * abs(a)
    assert Hs[-1] < Hs[0]
    # the Lax-Friedrichs stabilization gives a different first step from the same start
    prob_slf, _, V0, Vh0 = vortex_problem(2, 3, 1, ph.Physics(mach=0.5), L=6.0, deg=5, noise=0.0)
    first_s = time_step(prob, None, V0, Vh0, [V0], 1, 0.2, tol=1e-12, max_it=10).V
    first_slf = time_step(prob_slf, None, V0, Vh0, [V0], 1, 0.2, tol=1e-12, max_it=10).V
    assert np.abs(first_s - first_slf).max() > 1e-8
