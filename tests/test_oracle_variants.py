"""Pins of the oracle's variants of the scheme (the NEXT row of variants):
* viscous numerical flux option 1, ghat = G(v_h, q_h) . n (Eq. numericalFluxNS_1): the viscous
  part of the trace residual does not depend on vhat at fixed (v, q), and the scheme decays the
  shear wave at the closed-form rate like option 2;
* power-law viscosity mu = mu_ref (T / T_inf)^omega with omega = 3/4 (Sec. 5.6): at T0 = 2 the
  shear wave decays at mu_ref 2^(3/4) k^2 and not at the constant-viscosity rate;
* the entropy-production diagnostic Pi_S of Eq. PiS (Sec. 5.6): its physical term equals the
  closed-form -d/dt int H = int Phi / (c_v T0) of the shear wave at t = 0, and the scheme's own
  part Pi_S is small against it for the resolved wave (BDF1 step)."""
import math

import numpy as np

from oracle import physics as ph
from oracle.hdg import consistent_Q
from test_oracle_viscous import _shear_problem, _shear_state, shear_wave, viscous_face_part


def test_option_1_viscous_flux_ignores_the_trace():
    prob = _shear_problem(2, 2, 50.0, 0.3, flux_option=1)
    rng = np.random.default_rng(23)
    m, Np, d = prob.m, prob.Np, prob.d
    v0 = ph.v_of_u(ph.u_of_primitives(np.array(1.1), np.array([0.3, -0.2]), np.array(8.0), 1.4), 1.4)
    for e in (0, 5):
        V = v0 + 1e-2 * np.abs(v0) * rng.uniform(-1, 1, (Np, m))
        Vh = v0 + 1e-2 * np.abs(v0) * rng.uniform(-1, 1, (prob.nF, prob.Nf, m))
        Q = 0.1 * np.abs(v0)[None, :, None] * rng.uniform(-1, 1, (Np, m, d))
        ref = viscous_face_part(prob, e, Q, V, Vh)
        Vh2 = Vh + 1e-2 * np.abs(v0) * rng.uniform(-1, 1, Vh.shape)
        assert np.abs(viscous_face_part(prob, e, Q, V, Vh2) - ref).max() <= 1e-10 * np.abs(ref).max()
        V2 = V + 1e-2 * np.abs(v0) * rng.uniform(-1, 1, V.shape)   # ... but does depend on v
        assert np.abs(viscous_face_part(prob, e, Q, V2, Vh) - ref).max() > 1e-4 * np.abs(ref).max()


def test_option_1_shear_wave_decay():
    ratio, exact, _, _ = shear_wave(4, 2, 3, 2, 0.01, 1e-2, flux_option=1)
    assert abs(ratio[-1] - exact[-1]) / exact[-1] < 1e-3


def test_power_law_viscosity_shear_wave_decay():
    """omega = 3/4 at T0 = 2: the decay follows mu_ref 2^(3/4) (measured error ~2e-4 at p = 2),
    far from the constant-viscosity rate (the two decays differ by ~6 % after three steps)."""
    ratio, exact, _, _ = shear_wave(4, 2, 3, 2, 0.01, 1e-2, T0=2.0, mu_exponent=0.75)
    assert abs(ratio[-1] - exact[-1]) / exact[-1] < 1e-3
    lam_const = (1.0 / 20.0) * (2 * math.pi) ** 2
    const = math.exp(-lam_const * 0.03)
    assert abs(ratio[-1] - const) / const > 0.03


def test_entropy_production_diagnostic_on_the_shear_wave():
    n, p, eps, mach, T0, omega = 4, 2, 2e-2, 0.3, 2.0, 0.75
    probs = []
    dt = 0.002
    _, _, dH, dH_exact = shear_wave(n, p, 1, 1, dt, eps, mach=mach, T0=T0, mu_exponent=omega, prob_out=probs)
    prob = probs[0]
    mesh = prob.mesh
    k = 2.0 * math.pi
    mu0 = prob.phys.mu * T0 ** omega
    lam = mu0 * k * k
    p0 = T0 / (1.4 * mach ** 2)
    owner = np.array([s[0] for s in mesh.face_elems])
    fn = np.array(mesh.ref.face_nodes)
    V = _shear_state(prob, mesh.xnode, 0.0, eps, k, lam, p0)
    Vh = V[owner[:, 0][:, None], fn[owner[:, 1]]]
    Q = consistent_Q(prob, V, Vh)
    _, phys_term = prob.entropy_production_terms(Q, V)
    rate = mu0 * (1.4 - 1.0) / p0 * eps ** 2 * k ** 2 / 2.0      # int Phi / (c_v T0) at t = 0
    assert abs(phys_term - rate) <= 0.02 * rate, (phys_term, rate)
    # Pi_S over one BDF1 step: d/dt int rho s = -d/dt int H (H = -rho s), minus the physical term
    pi_s = -dH[0] / dt - phys_term
    assert abs(pi_s) <= 0.1 * rate, (pi_s, rate)
