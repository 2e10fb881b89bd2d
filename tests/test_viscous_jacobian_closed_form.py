"""The contraction sum_j c_j dG_ij/dq_lk of the viscous flux (Eq. viscFlux) written out by
hand, as the pointwise kernels evaluate it, against the oracle's viscous flux at unit
gradients (G is linear in q, so G(v, E_lk) is the column dG/dq_lk exactly). Runs on the CPU;
the GPU parity tests check the kernels' output against the oracle end to end."""
import numpy as np
import pytest

from oracle import physics as ph


def closed_form(v, c, phys):
    """out[i, l, k] = sum_j c_j dG_ij/dq_lk with V_a = -w_a/v_m, A_a = w_a/v_m^2."""
    d = v.shape[-1] - 2
    m = d + 2
    w, vm = v[1:-1], v[-1]
    ivm, ivm2 = 1.0 / vm, 1.0 / (vm * vm)
    vel, A = -w * ivm, w * ivm2
    cA, cV, VA = c @ A, c @ vel, vel @ A
    mu, kc = phys.mu, phys.kappa / phys.cv
    out = np.zeros((m, m, d))
    for k in range(d):
        for a in range(d):
            for b in range(d):
                out[1 + a, 1 + b, k] = mu * ivm * ((c[k] if a == b else 0.0) + (c[b] if a == k else 0.0)
                                                   - (2.0 / 3.0) * (c[a] if b == k else 0.0))
            out[1 + a, m - 1, k] = -mu * (A[a] * c[k] + (cA if a == k else 0.0) - (2.0 / 3.0) * A[k] * c[a])
        for b in range(d):
            out[m - 1, 1 + b, k] = mu * ivm * (vel[b] * c[k] + vel[k] * c[b] - (2.0 / 3.0) * (cV if b == k else 0.0))
        out[m - 1, m - 1, k] = -mu * (VA * c[k] + vel[k] * cA - (2.0 / 3.0) * A[k] * cV) - kc * ivm2 * c[k]
    return out


@pytest.mark.parametrize("d", [2, 3])
def test_closed_form_matches_unit_gradient_columns(d):
    rng = np.random.default_rng(11 + d)
    phys = ph.Physics(gamma=1.4, mach=0.3, reynolds=400.0, prandtl=0.71)
    m = d + 2
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        vel = rng.normal(0.0, 1.0, d)
        p = rng.uniform(0.5, 3.0) / (phys.gamma * phys.mach ** 2)
        v = ph.v_of_u(ph.u_of_primitives(np.array(rho), vel, np.array(p), phys.gamma), phys.gamma)
        c = rng.normal(0.0, 1.0, d)
        ref = np.zeros((m, m, d))
        for l in range(m):
            for k in range(d):
                E = np.zeros((m, d))
                E[l, k] = 1.0
                ref[:, l, k] = ph.viscous_flux(v, E, phys) @ c
        got = closed_form(v, c, phys)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        # the rows and columns the kernels skip are zero
        assert not ref[0].any() and not ref[:, 0].any()
