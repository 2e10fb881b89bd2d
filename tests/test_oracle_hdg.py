"""Pins of the oracle's discretisation: free-stream preservation, u-conservation
(Sec. 3.2 remark), Jacobians against central differences, static condensation +
trace solve + recovery equal to a Newton step on the monolithic global system
(Sec. 3.2/3.3 local elimination), Newton convergence and the entropy bound
(Theorem 1) on a periodic Euler run."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import physics as ph
from oracle.hdg import (Problem, bdf_coefficients, consistent_Q, interpolate_state,
                        newton_iteration, newton_solve, time_step)
from oracle.mesh import Mesh

EULER = ph.Physics(mach=0.5)
NS = ph.Physics(mach=0.3, reynolds=200.0, prandtl=0.72)


def vortex_problem(dim, n, p, phys, L=10.0, deg=None, seed=0, noise=1e-3):
    mesh = Mesh(dim, n, 0.0, L, p, deg)
    prob = Problem(mesh, phys)
    if dim == 2:
        V, Vh = interpolate_state(prob, lambda x: wl.vortex_field(
            x, [wl.Vortex(L / 2, L / 2, 3.0)], phys.mach, period=L))
    else:
        V, Vh = interpolate_state(prob, lambda x: wl.tgv_field(x * (2 * np.pi / L) + 0.3, phys.mach))
    if noise:
        Vh = wl.perturb(Vh, noise, seed)
        V = wl.perturb(V, noise, seed + 1)
    Q = consistent_Q(prob, V, Vh)
    if Q is not None and noise:
        Q = Q + noise * wl.uniform_noise(Q.shape, seed + 2)
    return prob, Q, V, Vh


@pytest.mark.parametrize("dim,p,phys", [(2, 2, EULER), (2, 3, NS), (3, 2, NS)])
def test_free_stream(dim, p, phys):
    mesh = Mesh(dim, 2, 0.0, 1.0, p)
    prob = Problem(mesh, phys)
    u0 = ph.u_of_primitives(np.array(1.1), np.array([0.9, -0.4, 0.3][:dim]),
                            np.array(1 / (1.4 * phys.mach ** 2)), 1.4)
    v0 = ph.v_of_u(u0, 1.4)
    V = np.broadcast_to(v0, (mesh.E, prob.Np, prob.m)).copy()
    Vh = np.broadcast_to(v0, (mesh.nFaces, prob.Nf, prob.m)).copy()
    Q = consistent_Q(prob, V, Vh)
    if Q is not None:
        assert np.abs(Q).max() < 1e-12
    scale = np.abs(v0).max() * np.abs(u0).max()
    for e in range(mesh.E):
        Rl, Rt = prob.local_residual(e, None if Q is None else Q[e], V[e], prob.gather_trace(Vh, e))
        assert np.abs(Rl).max() < 1e-13 * scale
    # the assembled trace residual vanishes too (fluxes cancel across faces)
    rt = np.zeros(prob.n_trace)
    for e in range(mesh.E):
        _, Rt = prob.local_residual(e, None if Q is None else Q[e], V[e], prob.gather_trace(Vh, e))
        np.add.at(rt, prob.trace_index(e), Rt)
    assert np.abs(rt).max() < 1e-13 * scale


@pytest.mark.parametrize("dim,p,phys", [(2, 2, EULER), (2, 2, NS), (3, 1, NS)])
def test_u_conservation_per_element(dim, p, phys):
    """Testing with w = e_i and mu = e_i: sum_a R_v - sum_c R_t = mass (u, 1) - sum hist."""
    prob, Q, V, Vh = vortex_problem(dim, 2, p, phys, L=4.0)
    mass, coefs = bdf_coefficients(1, 0.1)
    for e in range(prob.mesh.E):
        hist = prob.history_weak(e, [V[e] * 1.01], coefs)
        Rl, Rt = prob.local_residual(e, None if Q is None else Q[e], V[e],
                                     prob.gather_trace(Vh, e), mass, hist)
        Rv = Rl[-prob.Np * prob.m:].reshape(prob.Np, prob.m)
        T = prob.tables(e)
        tot_u = T.W @ ph.u_of_v(T.phi @ V[e], 1.4)
        lhs = Rv.sum(0) - Rt.reshape(-1, prob.m).sum(0)
        rhs = mass * tot_u - hist.sum(0)
        assert np.allclose(lhs, rhs, atol=1e-11 * np.abs(Rv).max())


@pytest.mark.parametrize("dim,p,phys", [(2, 2, EULER), (2, 2, NS), (3, 1, NS)])
def test_jacobian_against_central_differences(dim, p, phys):
    prob, Q, V, Vh = vortex_problem(dim, 2, p, phys, L=4.0)
    e = 1
    Qe = None if Q is None else Q[e]
    Vhe = prob.gather_trace(Vh, e)
    mass = 10.0
    A, B, C, D = prob.local_jacobian(e, Qe, V[e], Vhe, mass)
    x0 = V[e].ravel() if Qe is None else np.concatenate([Qe.ravel(), V[e].ravel()])
    y0 = Vhe.ravel()

    def res(x, y):
        if Qe is None:
            Rl, Rt = prob.local_residual(e, None, x.reshape(V[e].shape), y.reshape(Vhe.shape), mass)
        else:
            nq = Qe.size
            Rl, Rt = prob.local_residual(e, x[:nq].reshape(Qe.shape), x[nq:].reshape(V[e].shape),
                                         y.reshape(Vhe.shape), mass)
        return np.concatenate([Rl, Rt])

    full = np.block([[A, B], [C, D]])
    rng = np.random.default_rng(7)
    for j in rng.choice(x0.size + y0.size, size=12, replace=False):
        h = 1e-6 * max(1.0, abs(np.concatenate([x0, y0])[j]))
        dxp = np.concatenate([x0, y0]); dxp[j] += h
        dxm = np.concatenate([x0, y0]); dxm[j] -= h
        fd = (res(dxp[:x0.size], dxp[x0.size:]) - res(dxm[:x0.size], dxm[x0.size:])) / (2 * h)
        assert np.allclose(full[:, j], fd, atol=1e-6 * max(1.0, np.abs(full[:, j]).max()))


def _global_newton_update(prob, Q, V, Vh, mass, hist):
    """Newton update of the monolithic global system (all q, v, vhat) by a dense
    complex-step Jacobian of the global residual; no condensation involved."""
    E, m = prob.mesh.E, prob.m
    nq = 0 if Q is None else Q[0].size
    nv = V[0].size
    ni = nq + nv
    nt = prob.n_trace
    N = E * ni + nt

    def unpack(z):
        Qz = None if Q is None else z[:E * ni].reshape(E, ni)[:, :nq].reshape(Q.shape)
        Vz = z[:E * ni].reshape(E, ni)[:, nq:].reshape(V.shape)
        return Qz, Vz, z[E * ni:].reshape(Vh.shape)

    def global_res(z):
        Qz, Vz, Vhz = unpack(z)
        out = np.zeros(N, dtype=z.dtype)
        for e in range(E):
            Rq, Rv, Rt = prob.element_residual(e, None if Qz is None else Qz[e][None], Vz[e][None],
                                               prob.gather_trace(Vhz, e)[None], mass,
                                               None if hist is None else hist[e])
            Rl = Rv.reshape(-1) if Rq is None else np.concatenate([Rq.reshape(-1), Rv.reshape(-1)])
            out[e * ni:(e + 1) * ni] = Rl
            np.add.at(out, E * ni + prob.trace_index(e), Rt.reshape(-1))
        if getattr(prob, "edg_dirichlet", False):        # EDG with boundaries: vhat = v_b there
            nodes, vb = prob.dirichlet_nodes()
            out[E * ni + (nodes[:, None] * m + np.arange(m)).ravel()] = (Vhz[nodes] - vb).ravel()
        return out

    z0 = np.concatenate([np.concatenate([Q[e].ravel(), V[e].ravel()]) if Q is not None else V[e].ravel()
                         for e in range(E)] + [Vh.ravel()])
    J = np.zeros((N, N))
    for j in range(N):
        zc = z0.astype(np.complex128)
        zc[j] += 1j * 1e-30
        J[:, j] = np.imag(global_res(zc)) / 1e-30
    F = global_res(z0)
    dz = np.linalg.solve(J, -F)
    return unpack(z0 + dz)


@pytest.mark.parametrize("dim,n,p,phys", [(2, 2, 1, EULER), (2, 2, 2, NS), (3, 1, 1, NS)])
def test_condensed_equals_monolithic(dim, n, p, phys):
    prob, Q, V, Vh = vortex_problem(dim, n, p, phys, L=4.0, noise=1e-2)
    mass, coefs = bdf_coefficients(1, 0.2)
    hist = np.stack([prob.history_weak(e, [V[e]], coefs) for e in range(prob.mesh.E)])
    Qc, Vc, Vhc, _rn, _dvh, _ = newton_iteration(prob, Q, V, Vh, mass, hist)
    Qm, Vm, Vhm = _global_newton_update(prob, Q, V, Vh, mass, hist)
    assert np.allclose(Vc, Vm, rtol=0, atol=1e-11 * np.abs(V).max())
    assert np.allclose(Vhc, Vhm, rtol=0, atol=1e-11 * np.abs(Vh).max())
    if Q is not None:
        assert np.allclose(Qc, Qm, rtol=0, atol=1e-10 * max(1.0, np.abs(Q).max()))


def test_newton_converges_quadratically():
    prob, Q, V, Vh = vortex_problem(2, 3, 2, EULER, L=6.0, noise=1e-3)
    mass, coefs = bdf_coefficients(1, 0.1)
    hist = np.stack([prob.history_weak(e, [V[e]], coefs) for e in range(prob.mesh.E)])
    res = newton_solve(prob, Q, V, Vh, mass, hist, tol=1e-13, max_it=8)
    r = res.res_norms
    assert r[-1] <= 1e-13 * r[0]
    assert len(r) <= 6
    # quadratic: once in the asymptotic range the exponent of the ratio doubles
    assert r[2] / r[1] < 10 * (r[1] / r[0]) ** 1.5 + 1e-12


def test_entropy_non_increasing_and_bounded():
    """Periodic Euler, BDF1 (entropy stable by convexity of H), under-resolved so that
    the face-jump production dominates; int H must not increase and must stay above
    int H(u*) (Theorem 1, Eq. entropyBound), and int u is conserved."""
    L = 6.0
    prob, Q, V, Vh = vortex_problem(2, 3, 1, ph.Physics(mach=0.5), L=L, deg=5, noise=0.0)
    u0, H0 = prob.integrals(V)
    ustar = u0 / L ** 2
    Hstar = ph.entropy_H(ustar, 1.4) * L ** 2
    Hs = [H0]
    Vs = [V]
    for step in range(3):
        res = time_step(prob, None, Vs[-1], Vh, [Vs[-1]], 1, 0.2, tol=1e-12, max_it=10)
        Vs.append(res.V); Vh = res.Vhat
        u, Hc = prob.integrals(res.V)
        assert np.allclose(u, u0, rtol=0, atol=1e-10 * np.abs(u0).max())
        Hs.append(Hc)
    for a, b in zip(Hs, Hs[1:]):
        assert b <= a + 1e-12 * abs(a)
    assert Hs[-1] < Hs[0]
    assert min(Hs) >= Hstar - 1e-12 * abs(Hstar)


@pytest.mark.parametrize("dim", [2, 3])
def test_history_weak_closed_form(dim):
    """For p = 1 and a uniform state, (u, phi_a)_K = u |K| / (d + 1) for every vertex
    basis function (the integral of a barycentric coordinate)."""
    mesh = Mesh(dim, 2, 0.0, 3.0, 1)
    prob = Problem(mesh, NS)
    u0 = ph.u_of_primitives(np.array(1.2), np.array([0.3, -0.2, 0.1][:dim]), np.array(9.0), 1.4)
    v0 = ph.v_of_u(u0, 1.4)
    Vc = np.broadcast_to(v0, (prob.Np, prob.m))
    for e in (0, mesh.E - 1):
        h = prob.history_weak(e, [Vc], [2.5])
        vol = abs(mesh.detJ[e]) / math.factorial(dim)
        assert np.allclose(h, 2.5 * u0[None, :] * vol / (dim + 1), rtol=1e-13)


@pytest.mark.parametrize("dim,p", [(2, 2), (3, 2)])
def test_consistent_q_is_exact_gradient(dim, p):
    """With v linear in x and vhat its exact trace, Eq. hDG_NS0 gives q = grad v."""
    mesh = Mesh(dim, 2, 0.0, 3.0, p)
    prob = Problem(mesh, NS)
    rng = np.random.default_rng(9)
    m = dim + 2
    a0 = np.array([-5.0] + [0.1] * dim + [-0.2])
    Gr = 0.01 * rng.normal(size=(m, dim))
    for e in (0, 5, mesh.E - 1):
        x = mesh.xnode[e]                                   # element nodes (unreduced)
        V = a0 + x @ Gr.T
        Vh = V[np.array(mesh.ref.face_nodes)]               # exact trace in local order
        Q = prob.consistent_q(e, V, Vh)
        assert np.allclose(Q, np.broadcast_to(Gr, Q.shape), atol=1e-12)


def test_equilibrated_solve_recovers_exact_solution():
    """The oracle's local solve (power-of-two row and column equilibration, then LU): on a
    well-conditioned integer matrix with rows and columns scaled by 2^-30..2^30 and an integer
    solution (so that B = A X is exact), X comes back to rounding."""
    from oracle.hdg import solve_equilibrated
    rng = np.random.default_rng(17)
    n = 60
    A0 = rng.integers(-9, 10, size=(n, n)).astype(float) + 40.0 * np.eye(n)
    X = rng.integers(-50, 51, size=(n, 7)).astype(float)
    r = np.exp2(rng.integers(-30, 31, size=n).astype(float))
    c = np.exp2(rng.integers(-30, 31, size=n).astype(float))
    A = r[:, None] * A0 * c[None, :]
    Xs = X / c[:, None]                       # the solution of the scaled system
    B = A @ Xs                                # = r (A0 X): exact, the entries are small integers x 2^k
    assert np.array_equal(B, r[:, None] * (A0 @ X))
    err = lambda Y, Xt=X: np.abs(Y * c[:, None] - Xt).max() / np.abs(Xt).max()
    assert err(solve_equilibrated(A, B)) < 1e-13
    assert err(solve_equilibrated(A, B[:, 0])[:, None], X[:, :1]) < 1e-13
