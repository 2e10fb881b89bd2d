"""Pins of the oracle's DIRK(3,3) time step, the integrator of the paper's unsteady examples
(Sec. 5; Alexander's three-stage, third-order, L-stable method):
* the tableau satisfies the four order conditions of order three, is stiffly accurate and
  L-stable (stability function -> 0 at infinity, |R| <= 1 on the imaginary axis);
* on the viscous shear wave the step converges in time at order ~3 (self-convergence of the
  state as dt halves), against ~2 for BDF2."""
import math

import numpy as np

from oracle.hdg import consistent_Q, dirk3_step, dirk3_tableau
from test_oracle_viscous import _shear_problem, _shear_state


def test_tableau_order_conditions_and_stability():
    A, b, c = dirk3_tableau()
    g = A[0, 0]
    assert abs(g ** 3 - 3 * g ** 2 + 1.5 * g - 1.0 / 6.0) < 1e-15 and 1 / 6 < g < 0.5
    assert np.allclose(np.triu(A, 1), 0.0) and np.allclose(np.diag(A), g)     # diagonally implicit
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    assert np.allclose(A[2], b)                                              # stiffly accurate
    assert abs(b.sum() - 1.0) < 1e-15
    assert abs(b @ c - 0.5) < 1e-15
    assert abs(b @ c ** 2 - 1.0 / 3.0) < 1e-15
    assert abs(b @ A @ c - 1.0 / 6.0) < 1e-15
    R = lambda z: 1.0 + z * b @ np.linalg.solve(np.eye(3) - z * A, np.ones(3))
    assert abs(R(-1e8)) < 1e-7                                               # L-stable
    assert all(abs(R(1j * y)) <= 1.0 + 1e-12 for y in np.linspace(-50, 50, 101))
    z = -0.05                                                                # third order: R - e^z = O(z^4)
    assert abs(R(z) - math.exp(z)) < 0.05 * abs(z) ** 4


def _march(dt, nsteps, n=4, p=1, eps=1e-2):
    prob = _shear_problem(n, p, 20.0, 0.3)
    mesh = prob.mesh
    k = 2 * math.pi
    lam = prob.phys.mu * k * k
    p0 = 1.0 / (1.4 * 0.09)
    owner = np.array([s[0] for s in mesh.face_elems])
    fn = np.array(mesh.ref.face_nodes)
    V = _shear_state(prob, mesh.xnode, 0.0, eps, k, lam, p0)
    Vh = V[owner[:, 0][:, None], fn[owner[:, 1]]]
    Q = consistent_Q(prob, V, Vh)
    for _ in range(nsteps):
        res, iters = dirk3_step(prob, Q, V, Vh, dt, tol=1e-12)
        assert len(iters) == 3
        V, Vh, Q = res.V, res.Vhat, res.Q
    return V


def test_dirk3_temporal_order_on_the_shear_wave():
    T = 0.2
    Vs = [_march(T / m, m) for m in (2, 4, 8)]
    d1 = np.linalg.norm(Vs[0] - Vs[1])
    d2 = np.linalg.norm(Vs[1] - Vs[2])
    assert math.log2(d1 / d2) > 2.7, (d1, d2)          # measured 3.4 (BDF2 would give 2)
