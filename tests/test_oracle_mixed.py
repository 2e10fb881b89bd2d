"""Pins of the oracle's mixed-degree discretisation (element degree p_e per element, face
degree max(p_L, p_R); an extension the paper does not have, which uses one degree k).

* With every element at the same degree the mixed code is the uniform discretisation.
* Free stream is preserved on mixed meshes (2D Euler, 2D and 3D Navier-Stokes).
* Face matching: the face nodes both sides of a face address coincide in space.
* Static condensation + trace solve + recovery equals the Newton step of the monolithic
  global system (complex-step global Jacobian) on small mixed meshes.
* On a checkerboard of degrees 1 and 2 the steady vortex converges at order >= 1.6 (the
  lower degree plus the margin the uniform test allows) in u and in the trace.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import physics as ph
from oracle.hdg import (Problem, bdf_coefficients, consistent_Q, interpolate_state, newton_iteration,
                        time_step)
from oracle.mesh import Mesh
from oracle.refel import refel

EULER = ph.Physics(mach=0.5)
NS = ph.Physics(mach=0.3, reynolds=200.0, prandtl=0.72)


def _field(dim, phys, L):
    if dim == 2:
        return lambda x: wl.vortex_field(x, [wl.Vortex(L / 2, L / 2, 3.0)], phys.mach, period=L)
    return lambda x: wl.tgv_field(x * (2 * np.pi / L) + 0.3, phys.mach)


def _elements(dim, n):
    return 2 * n * n if dim == 2 else 6 * n ** 3


@pytest.mark.parametrize("dim,n,p,phys", [(2, 2, 2, EULER), (2, 2, 3, NS), (3, 1, 2, NS)])
def test_uniform_degrees_reduce_to_the_uniform_discretisation(dim, n, p, phys):
    L = 4.0
    m0 = Mesh(dim, n, 0.0, L, p)
    mm = Mesh(dim, n, 0.0, L, 0, p_elem=np.full(m0.E, p))
    P0, Pm = Problem(m0, phys), Problem(mm, phys)
    V0, Vh0 = interpolate_state(P0, _field(dim, phys, L))
    Vm, Vhm = interpolate_state(Pm, _field(dim, phys, L))
    assert np.array_equal(np.stack(Vm), V0)
    assert np.array_equal(Vhm.reshape(Vh0.shape), Vh0)
    Vh0 = wl.perturb(Vh0, 1e-3, 3)
    Vhm = Vh0.reshape(Vhm.shape)
    Q0, Qm = consistent_Q(P0, V0, Vh0), consistent_Q(Pm, Vm, Vhm)
    for e in (0, m0.E - 1):
        a = P0.condense(e, None if Q0 is None else Q0[e], V0[e], P0.gather_trace(Vh0, e), 1.0)
        b = Pm.condense(e, None if Qm is None else Qm[e], Vm[e], Pm.gather_trace(Vhm, e), 1.0)
        assert np.array_equal(P0.trace_index(e), Pm.trace_index(e))
        for k in ("S", "g", "X", "y"):
            assert np.abs(a[k] - b[k]).max() <= 1e-13 * np.abs(a[k]).max(), k


@pytest.mark.parametrize("dim,n,degs,phys", [(2, 2, (1, 2, 3), EULER), (2, 2, (1, 3), NS), (3, 1, (1, 2, 3), NS)])
def test_mixed_free_stream(dim, n, degs, phys):
    rng = np.random.default_rng(11)
    mesh = Mesh(dim, n, 0.0, 1.0, 0, p_elem=rng.choice(degs, size=_elements(dim, n)))
    prob = Problem(mesh, phys)
    u0 = ph.u_of_primitives(np.array(1.1), np.array([0.9, -0.4, 0.3][:dim]),
                            np.array(1 / (1.4 * phys.mach ** 2)), 1.4)
    v0 = ph.v_of_u(u0, 1.4)
    V = [np.broadcast_to(v0, (prob.np_e(e), prob.m)).copy() for e in range(mesh.E)]
    Vh = np.broadcast_to(v0, prob.trace_shape).copy()
    Q = consistent_Q(prob, V, Vh)
    scale = np.abs(v0).max() * np.abs(u0).max()
    rt = np.zeros(prob.n_trace)
    for e in range(mesh.E):
        if Q is not None:
            assert np.abs(Q[e]).max() < 1e-12
        Rl, Rt = prob.local_residual(e, None if Q is None else Q[e], V[e], prob.gather_trace(Vh, e))
        assert np.abs(Rl).max() < 1e-13 * scale
        np.add.at(rt, prob.trace_index(e), Rt)
    assert np.abs(rt).max() < 1e-13 * scale


@pytest.mark.parametrize("dim,n", [(2, 3), (3, 2)])
def test_face_degrees_and_node_matching(dim, n):
    rng = np.random.default_rng(5)
    pe = rng.choice([1, 2, 3, 4] if dim == 2 else [1, 2, 3], size=_elements(dim, n))
    mesh = Mesh(dim, n, 0.0, 1.0, 0, p_elem=pe)
    period = mesh.hi - mesh.lo
    for F, sides in enumerate(mesh.face_elems):
        assert mesh.face_deg[F] == max(pe[e] for e, _ in sides)
        q = int(mesh.face_deg[F])
        r = refel(dim, q)
        assert mesh.face_nnodes[F] == r.Nf
        xs = []
        for (e, f) in sides:
            assert mesh.elem_face_deg[e, f] == q
            x = mesh.X[e, 0] + r.nodes[r.face_nodes[f]] @ mesh.J[e].T        # local face-node order
            canon = np.empty_like(x)
            canon[mesh.fnode_map_mixed[e, f, :r.Nf]] = x
            assert np.all(mesh.fnode_map_mixed[e, f, r.Nf:] == -1)
            xs.append(canon)
        if len(xs) == 2:
            d = (xs[1] - xs[0]) / period
            assert np.allclose(d, np.round(d), atol=1e-12)                    # equal up to a period
            assert np.allclose(d - np.round(d)[0], 0.0, atol=1e-12)           # one translation per face
    assert np.array_equal(mesh.elem_trace_deg, mesh.elem_face_deg.max(axis=1))
    assert np.all(mesh.elem_trace_deg >= pe)


def _global_newton_update(prob, Q, V, Vh, mass, hist):
    """Newton update of the monolithic global system (every element's q, v and the trace) by a
    dense complex-step Jacobian of the global residual; no condensation involved."""
    E = prob.mesh.E
    sizes = [(0 if Q is None else Q[e].size, V[e].size) for e in range(E)]
    off = np.concatenate([[0], np.cumsum([a + b for a, b in sizes])])
    nt = prob.n_trace
    N = int(off[-1]) + nt

    def unpack(z):
        Qz, Vz = [], []
        for e in range(E):
            x = z[off[e]:off[e + 1]]
            nq = sizes[e][0]
            Qz.append(None if Q is None else x[:nq].reshape(Q[e].shape))
            Vz.append(x[nq:].reshape(V[e].shape))
        return Qz, Vz, z[off[-1]:].reshape(Vh.shape)

    def global_res(z):
        Qz, Vz, Vhz = unpack(z)
        out = np.zeros(N, dtype=z.dtype)
        for e in range(E):
            Rq, Rv, Rt = prob.element_residual(e, None if Q is None else Qz[e][None], Vz[e][None],
                                               prob.gather_trace(Vhz, e)[None], mass, hist[e])
            Rl = Rv.reshape(-1) if Rq is None else np.concatenate([Rq.reshape(-1), Rv.reshape(-1)])
            out[off[e]:off[e + 1]] = Rl
            np.add.at(out, off[-1] + prob.trace_index(e), Rt.reshape(-1)[prob.trace_mask(e)])
        return out

    z0 = np.concatenate([np.concatenate(([] if Q is None else [Q[e].ravel()]) + [V[e].ravel()])
                         for e in range(E)] + [Vh.ravel()])
    J = np.zeros((N, N))
    for j in range(N):
        zc = z0.astype(np.complex128)
        zc[j] += 1j * 1e-30
        J[:, j] = np.imag(global_res(zc)) / 1e-30
    dz = np.linalg.solve(J, -global_res(z0))
    return unpack(z0 + dz)


@pytest.mark.parametrize("dim,n,degs,phys", [(2, 2, (1, 2), EULER), (2, 2, (1, 2), NS), (3, 1, (1, 2), NS)])
def test_mixed_condensed_equals_monolithic(dim, n, degs, phys):
    L = 4.0
    rng = np.random.default_rng(3)
    mesh = Mesh(dim, n, 0.0, L, 0, p_elem=rng.choice(degs, size=_elements(dim, n)))
    prob = Problem(mesh, phys)
    V, Vh = interpolate_state(prob, _field(dim, phys, L))
    Vh = wl.perturb(Vh, 1e-2, 7)
    V = [wl.perturb(v, 1e-2, 8 + e) for e, v in enumerate(V)]
    Q = consistent_Q(prob, V, Vh)
    mass, coefs = bdf_coefficients(1, 0.2)
    hist = [prob.history_weak(e, [V[e]], coefs) for e in range(mesh.E)]
    Qc, Vc, Vhc, _rn, _dvh, _ = newton_iteration(prob, Q, V, Vh, mass, hist)
    Qm, Vm, Vhm = _global_newton_update(prob, Q, V, Vh, mass, hist)
    vs = max(np.abs(v).max() for v in V)
    for e in range(mesh.E):
        assert np.allclose(Vc[e], Vm[e], rtol=0, atol=1e-11 * vs)
        if Q is not None:
            assert np.allclose(Qc[e], Qm[e], rtol=0, atol=1e-10 * max(1.0, np.abs(Q[e]).max()))
    assert np.allclose(Vhc, Vhm, rtol=0, atol=1e-11 * np.abs(Vh).max())


def _checkerboard(n, lo, hi):
    c = np.arange(2 * n * n) // 2                  # element e = 2 c + t, cell c = j n + i
    return np.where((c % n + c // n) % 2 == 0, lo, hi)


def _steady_vortex_errors(n, degs, L=8.0):
    phys = EULER
    field = lambda x: wl.vortex_field(x, [wl.Vortex(L / 2, L / 2, 3.0)], 0.5, vinf=(0.0, 0.0), period=L)
    mesh = Mesh(2, n, 0.0, L, 0, p_elem=_checkerboard(n, *degs))
    prob = Problem(mesh, phys)
    V, Vh = interpolate_state(prob, field)
    res = time_step(prob, None, V, Vh, [V], 1, 0.5, tol=1e-11, max_it=8)
    assert res.res_norms[-1] <= 1e-11 * max(1.0, res.res_norms[0])
    err = 0.0
    for e in range(mesh.E):
        T = prob.tables(e)
        xq = mesh.X[e, 0] + refel(2, int(mesh.p_elem[e])).qp @ mesh.J[e].T
        rho, vel, pr = field(xq)
        uh = ph.u_of_v(T.phi @ res.V[e], 1.4)
        err += T.W @ np.sum((uh - ph.u_of_primitives(rho, vel, pr, 1.4)) ** 2, axis=1)
    _, Vh_exact = interpolate_state(prob, field)
    return math.sqrt(err), np.abs(res.Vhat - Vh_exact).max()


def test_mixed_convergence_order():
    """Degrees 1 and 2 on alternate cells, meshes 8x8 -> 16x16: the error in u and the error of
    the trace at its nodes fall at order >= 1.6 (measured 2.18 and 1.73). A face-node map that
    ignores the node coordinates (identity on the second side) gives 1.03 and 0.22."""
    e8, t8 = _steady_vortex_errors(8, (1, 2))
    e16, t16 = _steady_vortex_errors(16, (1, 2))
    assert math.log2(e8 / e16) >= 1.6, (e8, e16)
    assert math.log2(t8 / t16) >= 1.6, (t8, t16)
