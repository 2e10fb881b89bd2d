"""Pins of the oracle's boundary terms b_h (Eqs. hDG2 / hDG_NS2; the paper leaves b_h open):
* bounded meshes: the one-sided faces lie on the walls of the bounded axes, with the outward
  normal of the box, and every other face keeps two sides;
* free stream: a uniform state is an exact discrete solution with the boundary state equal to
  it (Euler and Navier-Stokes) and with slip walls parallel to the flow;
* BC_STATE: the stationary isentropic vortex is an exact steady solution of the Euler
  equations; with it prescribed on all four sides of a box, pseudo-time marching from it
  stays within O(h^(p+1)) of it and the trace equals the boundary state on the boundary faces;
* BC_SLIP: the closed slip box is the mirror-symmetric doubled periodic problem restricted to
  one quadrant (the state after a BDF1 step equals the doubled problem's on the original
  elements); mass and energy are conserved, the trace's normal velocity vanishes on the walls,
  and int H does not increase."""
import numpy as np
import pytest

import workloads as wl
from oracle import physics as ph
from oracle.hdg import Problem, interpolate_state, residual_norm, time_step
from oracle.mesh import BC_SLIP, BC_STATE, Mesh

EULER = ph.Physics(mach=0.5)
NS = ph.Physics(mach=0.3, reynolds=200.0, prandtl=0.72)


def _wall_check(mesh):
    n, dim = mesh.n, mesh.dim
    for F, sides in enumerate(mesh.face_elems):
        if len(sides) == 2:
            assert mesh.face_bc[F] == 0
            continue
        r, s = mesh.face_wall[F]
        e, f = sides[0]
        fv = mesh.L[e, mesh.ref.face_verts[f]]
        assert np.all(fv[:, r] == (0 if s == 0 else n))
        expect = np.zeros(dim)
        expect[r] = -1.0 if s == 0 else 1.0
        assert np.allclose(mesh.normal[e, f], expect, atol=1e-14)


@pytest.mark.parametrize("dim,n", [(2, 3), (3, 2)])
def test_bounded_mesh_topology(dim, n):
    bc = [("periodic", "periodic")] * dim
    bc[1] = ("state", "slip")
    mesh = Mesh(dim, n, 0.0, 1.0, 1, bc=bc)
    per_side = n ** (dim - 1) * (1 if dim == 2 else 2)
    assert np.sum(mesh.face_bc == BC_STATE) == per_side
    assert np.sum(mesh.face_bc == BC_SLIP) == per_side
    periodic_faces = (3 if dim == 2 else 12) * n ** dim
    assert mesh.nFaces == periodic_faces + per_side        # the identified wall faces split in two
    _wall_check(mesh)


def _uniform(prob, prim):
    rho, vel, p = prim
    v0 = ph.v_of_u(ph.u_of_primitives(np.array(rho), np.array(vel), np.array(p), prob.phys.gamma), prob.phys.gamma)
    V = np.broadcast_to(v0, (prob.mesh.E, prob.Np, prob.m)).copy()
    Vh = np.broadcast_to(v0, prob.trace_shape).copy()
    return v0, V, Vh


@pytest.mark.parametrize("dim,p,phys,bc,vel", [
    (2, 2, EULER, [("state", "state"), ("slip", "slip")], (0.9, 0.0)),
    (2, 3, NS, [("state", "state"), ("periodic", "periodic")], (0.7, -0.3)),
    (3, 1, NS, [("periodic", "periodic"), ("state", "state"), ("state", "state")], (0.4, 0.2, -0.3)),
    (3, 2, EULER, [("slip", "slip"), ("periodic", "periodic"), ("state", "state")], (0.0, 0.5, 0.3)),
])
def test_free_stream_with_boundaries(dim, p, phys, bc, vel):
    mesh = Mesh(dim, 2, 0.0, 1.0, p, bc=bc)
    prob = Problem(mesh, phys)
    v0, V, Vh = _uniform(prob, (1.2, vel, 0.9 / (1.4 * phys.mach ** 2)))
    prob.boundary_state = Vh.copy()
    Q = None if not phys.viscous else np.zeros((mesh.E, prob.Np, prob.m, dim))
    locs = [prob.condense(e, None if Q is None else Q[e], V[e], prob.gather_trace(Vh, e)) for e in range(mesh.E)]
    assert residual_norm(prob, locs) <= 1e-12        # local residuals and the assembled trace residual


def _vortex_box(n, p, L=8.0, psi=3.0):
    mesh = Mesh(2, n, 0.0, L, p, deg=2 * p + 2, bc=[("state", "state"), ("state", "state")])
    prob = Problem(mesh, EULER)
    prim = lambda x: wl.vortex_field(x, [wl.Vortex(L / 2, L / 2, psi)], EULER.mach, vinf=(0.0, 0.0))
    V, Vh = interpolate_state(prob, prim)
    prob.boundary_state = Vh.copy()
    return prob, prim, V, Vh


def _l2_error(prob, V, prim):
    err = 0.0
    for e in range(prob.mesh.E):
        T = prob.tables(e)
        xq = prob.mesh.X[e, 0] + prob.mesh.ref.qp @ prob.mesh.J[e].T
        rho, vel, p = prim(xq)
        ue = ph.u_of_primitives(rho, vel, p, prob.phys.gamma)
        uh = ph.u_of_v(T.phi @ V[e], prob.phys.gamma)
        err += T.W @ np.sum((uh - ue) ** 2, axis=-1)
    return np.sqrt(err)


def test_state_bc_steady_vortex_converges_and_takes_the_boundary_state():
    """Pseudo-time marching (one backward Euler step of 0.5, as for the periodic convergence
    test) from the exact stationary vortex, prescribed on all four sides of the box [0, 8]^2
    (without periodic images): the error against the exact state falls at order ~p+1."""
    p = 2
    errs = []
    for n in (6, 12):
        prob, prim, V, Vh = _vortex_box(n, p)
        res = time_step(prob, None, V, Vh, [V], 1, 0.5, tol=1e-12, max_it=10)
        assert res.res_norms[-1] <= 1e-12 * max(1.0, res.res_norms[0])
        errs.append(_l2_error(prob, res.V, prim))
        wall = prob.mesh.face_bc == BC_STATE
        assert np.abs(res.Vhat[wall] - prob.boundary_state[wall]).max() <= 1e-12 * np.abs(res.Vhat).max()
    order = np.log2(errs[0] / errs[1])
    assert order >= p + 0.6, (errs, order)


# -- the slip wall as a mirror ------------------------------------------------------------
def _mirrored(n, L, p):
    """The doubled periodic mesh of [-L, L]^2: the Kuhn mesh of [0, L]^2 and its mirror images
    in x, in y and in both, each image keeping the vertex order of its original, so that its
    reference map and quadrature points are the mirror images too (a single mirror leaves it
    negatively oriented; the residual uses |det J| and outward normals). Returns the mesh and,
    per element of the doubled mesh, (original element, mirror flags)."""
    base = Mesh(2, n, 0.0, L, p)
    blocks, origin = [], []
    for sx in (0, 1):
        for sy in (0, 1):
            v = base.L.copy()
            v[..., 0] = n - v[..., 0] if sx else v[..., 0] + n
            v[..., 1] = n - v[..., 1] if sy else v[..., 1] + n
            blocks.append(v)
            origin += [(e, sx, sy) for e in range(base.E)]
    return Mesh(2, 2 * n, -L, L, p, verts=np.concatenate(blocks)), origin


def _mirror_state(mesh_d, origin, mesh_h, Vh_elem):
    """Element states of the doubled mesh: the mirror image of the original element's."""
    Vd = np.zeros((mesh_d.E,) + Vh_elem.shape[1:])
    for ed, (e, sx, sy) in enumerate(origin):
        sgn = np.array([-1.0 if sx else 1.0, -1.0 if sy else 1.0])
        for a in range(mesh_d.ref.Np):
            x = mesh_d.xnode[ed, a] * sgn
            b = int(np.argmin(np.linalg.norm(mesh_h.xnode[e] - x, axis=-1)))
            assert np.linalg.norm(mesh_h.xnode[e, b] - x) < 1e-12
            v = Vh_elem[e, b].copy()
            v[1:3] *= sgn
            Vd[ed, a] = v
    return Vd


def _owner_trace(prob, V):
    fn = np.array(prob.mesh.ref.face_nodes)
    owner = np.array([s[0] for s in prob.mesh.face_elems])
    return V[owner[:, 0][:, None], fn[owner[:, 1]]]


def _slip_start(n, L, p):
    mesh = Mesh(2, n, 0.0, L, p, bc=[("slip", "slip"), ("slip", "slip")])
    prob = Problem(mesh, EULER)
    prim = lambda x: wl.vortex_field(x, [wl.Vortex(0.4 * L, 0.6 * L, 3.0)], EULER.mach, vinf=(0.3, -0.2))
    V, Vh = interpolate_state(prob, prim)
    return prob, V, Vh


def test_slip_box_is_the_mirror_symmetric_doubled_problem():
    n, L, p, dt = 2, 6.0, 2, 0.2
    prob, V, Vh = _slip_start(n, L, p)
    half = time_step(prob, None, V, Vh, [V], 1, dt, tol=1e-12, max_it=12)
    mesh_d, origin = _mirrored(n, L, p)
    prob_d = Problem(mesh_d, EULER)
    Vd = _mirror_state(mesh_d, origin, prob.mesh, V)
    full = time_step(prob_d, None, Vd, _owner_trace(prob_d, Vd), [Vd], 1, dt, tol=1e-12, max_it=12)
    assert full.res_norms[-1] <= 1e-12 * full.res_norms[0]
    scale = np.abs(half.V).max()
    for ed, (e, sx, sy) in enumerate(origin):
        if sx == 0 and sy == 0:
            assert np.abs(full.V[ed] - half.V[e]).max() <= 1e-10 * scale, ed
    # the mirror images carry the reflected state
    Vd_half = _mirror_state(mesh_d, origin, prob.mesh, half.V)
    assert np.abs(full.V - Vd_half).max() <= 1e-10 * scale


def test_slip_box_conserves_mass_and_energy_and_entropy():
    n, L, p, dt = 3, 6.0, 1, 0.2
    prob, V, Vh = _slip_start(n, L, p)
    u0, H0 = prob.integrals(V)
    Hs = [H0]
    wall = prob.mesh.face_bc == BC_SLIP
    for step in range(3):
        res = time_step(prob, None, V, Vh, [V], 1, dt, tol=1e-12, max_it=12)
        V, Vh = res.V, res.Vhat
        u, H = prob.integrals(V)
        assert abs(u[0] - u0[0]) <= 1e-11 * abs(u0[0]) and abs(u[-1] - u0[-1]) <= 1e-11 * abs(u0[-1])
        Hs.append(H)
        for F in np.nonzero(wall)[0]:
            r, _ = prob.mesh.face_wall[F]
            assert np.abs(Vh[F, :, 1 + r]).max() <= 1e-10 * np.abs(Vh[F, :, 1:3]).max()   # w . n = 0
    assert abs(u[1] - u0[1]) > 1e-6 * abs(u0[0])            # the walls' pressure does change momentum
    for a, b in zip(Hs, Hs[1:]):
        assert b <= a + 1e-12 * abs(a)
