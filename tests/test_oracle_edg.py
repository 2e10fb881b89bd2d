"""Pins of the oracle's EDG scheme (Sec. 3.4: E^E_h = all faces, a continuous trace with one
unknown per skeleton node; IEDG coincides with it on periodic meshes):
* the number of global trace unknowns is alpha_DOF N_v m of Table t:dofs (EDG rows);
* uniform flow with the trace equal to it has zero residual (free stream);
* static condensation + the assembled EDG trace solve + recovery equal one Newton step of the
  monolithic global system (all q, v and the continuous vhat; complex-step Jacobian);
* the total generalised entropy does not increase on periodic Euler BDF1 steps (Theorem 1);
and on bounded meshes: IEDG (E^E_h = the interior faces: each boundary face keeps its own
trace nodes) with the count of unknowns in closed form, and both IEDG and EDG (whose boundary
nodes are shared with interior faces, so the given state is imposed strongly there: the node's
equation is vhat = v_b) with free stream and with condensation + trace solve + recovery equal to
the monolithic Newton step. EDG with a slip wall is refused."""
import numpy as np
import pytest

import workloads as wl
from oracle import physics as ph
from oracle.hdg import (Problem, bdf_coefficients, consistent_Q, face_states, interpolate_state, newton_iteration,
                        residual_norm, time_step)
from oracle.mesh import Mesh
from test_oracle_hdg import EULER, NS, _global_newton_update
from test_oracle_refel_mesh import _golden


def edg_problem(dim, n, p, phys, L=4.0, noise=1e-2, deg=None, seed=0):
    prob = Problem(Mesh(dim, n, 0.0, L, p, deg), phys, scheme="edg")
    if dim == 2:
        field = lambda x: wl.vortex_field(x, [wl.Vortex(L / 2, L / 2, 3.0)], phys.mach, period=L)
    else:
        field = lambda x: wl.tgv_field(x * (2 * np.pi / L) + 0.3, phys.mach)
    V, Vh = interpolate_state(prob, field)
    if noise:
        Vh = wl.perturb(Vh, noise, seed)
        V = wl.perturb(V, noise, seed + 1)
    Q = consistent_Q(prob, V, Vh)
    return prob, Q, V, Vh


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 2), (3, 3)])
def test_edg_unknowns_match_table(dim, k):
    g = _golden()
    n = 4 if dim == 2 else 3
    mesh = Mesh(dim, n, 0.0, 1.0, k)
    prob = Problem(mesh, NS, scheme="edg")
    assert prob.n_trace == g[("dof", "EDG", dim)][k - 1] * mesh.n_vertices * (dim + 2)
    # every local face node of an element maps to a node, copies of a node are its copies
    assert prob.edg_index.min() == 0 and prob.edg_index.max() == prob.n_edg - 1


@pytest.mark.parametrize("dim,p,phys", [(2, 2, EULER), (2, 3, NS), (3, 2, NS)])
def test_edg_free_stream(dim, p, phys):
    mesh = Mesh(dim, 2, 0.0, 1.0, p)
    prob = Problem(mesh, phys, scheme="edg")
    u0 = ph.u_of_primitives(np.array(1.1), np.array([0.9, -0.4, 0.3][:dim]),
                            np.array(1 / (1.4 * phys.mach ** 2)), 1.4)
    v0 = ph.v_of_u(u0, 1.4)
    V = np.broadcast_to(v0, (mesh.E, prob.Np, prob.m)).copy()
    Vh = np.broadcast_to(v0, prob.trace_shape).copy()
    Q = consistent_Q(prob, V, Vh)
    scale = np.abs(v0).max() * np.abs(u0).max()
    rt = np.zeros(prob.n_trace)
    for e in range(mesh.E):
        Rl, Rt = prob.local_residual(e, None if Q is None else Q[e], V[e], prob.gather_trace(Vh, e))
        assert np.abs(Rl).max() < 1e-13 * scale
        np.add.at(rt, prob.trace_index(e), Rt)
    assert np.abs(rt).max() < 1e-13 * scale


@pytest.mark.parametrize("dim,n,p,phys", [(2, 2, 2, EULER), (2, 2, 2, NS), (3, 1, 2, NS)])
def test_edg_condensed_equals_monolithic(dim, n, p, phys):
    prob, Q, V, Vh = edg_problem(dim, n, p, phys)
    mass, coefs = bdf_coefficients(1, 0.2)
    hist = np.stack([prob.history_weak(e, [V[e]], coefs) for e in range(prob.mesh.E)])
    Qc, Vc, Vhc, _rn, _dvh, _ = newton_iteration(prob, Q, V, Vh, mass, hist)
    Qm, Vm, Vhm = _global_newton_update(prob, Q, V, Vh, mass, hist)
    assert np.allclose(Vc, Vm, rtol=0, atol=1e-11 * np.abs(V).max())
    assert np.allclose(Vhc, Vhm, rtol=0, atol=1e-11 * np.abs(Vh).max())
    if Q is not None:
        assert np.allclose(Qc, Qm, rtol=0, atol=1e-10 * max(1.0, np.abs(Q).max()))


def test_edg_entropy_non_increasing():
    L = 6.0
    prob, Q, V, Vh = edg_problem(2, 3, 1, ph.Physics(mach=0.5), L=L, deg=5, noise=0.0)
    u0, H0 = prob.integrals(V)
    Hs = [H0]
    for _ in range(3):
        res = time_step(prob, None, V, Vh, [V], 1, 0.2, tol=1e-12, max_it=10)
        V, Vh = res.V, res.Vhat
        u, Hc = prob.integrals(V)
        assert np.allclose(u, u0, rtol=0, atol=1e-10 * np.abs(u0).max())
        Hs.append(Hc)
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(Hs, Hs[1:])) and Hs[-1] < Hs[0]


BOX2 = [("state", "state"), ("state", "state")]


@pytest.mark.parametrize("n,p", [(2, 1), (3, 2), (4, 3)])
def test_iedg_unknowns_on_a_box(n, p):
    """2D, all four sides bounded: the interior skeleton keeps every EDG node except those that
    lie on boundary faces only (the p - 1 inner nodes of each of the 4n boundary faces and the
    two corners that no diagonal reaches), and each boundary face adds its own p + 1 nodes:
    n_IEDG = n_EDG - 4n(p - 1) - 2 + 4n(p + 1) = n_EDG + 8n - 2."""
    mesh = Mesh(2, n, 0.0, 1.0, p, bc=BOX2)
    n_edg, _ = mesh.edg_numbering()
    prob = Problem(mesh, EULER, scheme="iedg")
    assert prob.n_edg == n_edg + 8 * n - 2
    assert n_edg == (n * p + 1) ** 2 - 2 * n * n * (p - 1) * (p - 2) // 2    # lattice minus element interiors
    idx = prob.edg_index
    for F, sides in enumerate(mesh.face_elems):
        if mesh.face_bc[F]:                          # its nodes belong to this face alone
            e, f = sides[0]
            mine = set(idx[e, f].tolist())
            others = set(np.delete(idx.reshape(-1, idx.shape[-1]), e * mesh.ref.nF + f, axis=0).ravel().tolist())
            assert len(mine) == mesh.ref.Nf and not mine & others
    with pytest.raises(ValueError):             # EDG with boundaries: the given state only
        Problem(Mesh(2, n, 0.0, 1.0, p, bc=[("state", "state"), ("slip", "slip")]), EULER, scheme="edg")


def _iedg_box(dim, n, p, phys, bc, noise=1e-2, scheme="iedg"):
    prob = Problem(Mesh(dim, n, 0.0, 4.0, p, bc=bc), phys, scheme=scheme)
    if dim == 2:
        field = lambda x: wl.vortex_field(x, [wl.Vortex(2.0, 2.0, 3.0)], phys.mach, vinf=(0.5, 0.2))
    else:
        field = lambda x: wl.tgv_field(x * (2 * np.pi / 4.0) + 0.3, phys.mach)
    V, Vh = interpolate_state(prob, field)
    prob.boundary_state = face_states(prob, V)
    if noise:
        Vh = wl.perturb(Vh, noise, 0)
        V = wl.perturb(V, noise, 1)
    return prob, consistent_Q(prob, V, Vh), V, Vh


@pytest.mark.parametrize("scheme", ["iedg", "edg"])
@pytest.mark.parametrize("dim,p,phys,bc", [(2, 2, EULER, BOX2), (2, 2, NS, BOX2),
                                           (3, 1, NS, [("periodic", "periodic"), ("state", "state"),
                                                       ("periodic", "periodic")])])
def test_iedg_free_stream_with_boundaries(dim, p, phys, bc, scheme):
    mesh = Mesh(dim, 2, 0.0, 1.0, p, bc=bc)
    prob = Problem(mesh, phys, scheme=scheme)
    u0 = ph.u_of_primitives(np.array(1.1), np.array([0.9, -0.4, 0.3][:dim]),
                            np.array(1 / (1.4 * phys.mach ** 2)), 1.4)
    v0 = ph.v_of_u(u0, 1.4)
    V = np.broadcast_to(v0, (mesh.E, prob.Np, prob.m)).copy()
    Vh = np.broadcast_to(v0, prob.trace_shape).copy()
    prob.boundary_state = face_states(prob, V)
    Q = consistent_Q(prob, V, Vh)
    scale = np.abs(v0).max() * np.abs(u0).max()
    locs = [prob.condense(e, None if Q is None else Q[e], V[e], prob.gather_trace(Vh, e)) for e in range(mesh.E)]
    assert residual_norm(prob, locs, Vh) < 1e-13 * scale


@pytest.mark.parametrize("scheme", ["iedg", "edg"])
@pytest.mark.parametrize("phys", [EULER, NS])
def test_iedg_condensed_equals_monolithic_with_boundaries(phys, scheme):
    prob, Q, V, Vh = _iedg_box(2, 2, 2, phys, BOX2, scheme=scheme)
    mass, coefs = bdf_coefficients(1, 0.2)
    hist = np.stack([prob.history_weak(e, [V[e]], coefs) for e in range(prob.mesh.E)])
    Qc, Vc, Vhc, _rn, _dvh, _ = newton_iteration(prob, Q, V, Vh, mass, hist)
    Qm, Vm, Vhm = _global_newton_update(prob, Q, V, Vh, mass, hist)
    assert np.allclose(Vc, Vm, rtol=0, atol=1e-11 * np.abs(V).max())
    assert np.allclose(Vhc, Vhm, rtol=0, atol=1e-11 * np.abs(Vh).max())
    if Q is not None:
        assert np.allclose(Qc, Qm, rtol=0, atol=1e-10 * max(1.0, np.abs(Q).max()))
