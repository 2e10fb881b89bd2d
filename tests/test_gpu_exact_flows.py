"""GPU parity of steady solves of the paper's exact flows with the oracle, in both precisions:
* the Couette flow of Sec. 5.2 (Navier-Stokes with a source term; periodic in x, the exact
  state on the walls y = 0, 1; Re0 = 0.1, M0 = 0.15): hdg_add_source gives the oracle's
  (s_h, phi_a)_K element by element, and a steady Newton solve (no time term, the source as the
  history) from the interpolated exact state takes the oracle's number of updates to its state;
* the Ringleb flow of Sec. 5.1 (Euler, the exact state on the whole boundary): the same, with
  the HDG, IEDG and EDG trace spaces (EDG: the state imposed strongly at the boundary nodes)."""
import numpy as np
import pytest

import workloads as wl
from hdg_cases import rel_fro

pytestmark = pytest.mark.gpu

MACH, RE, PR = 0.15, 0.1, 0.71
BC = (("periodic", "periodic"), ("state", "state"))


def _prim(x):
    rho, vel, p = wl.couette_field(x, MACH, PR)
    return np.concatenate([rho[..., None], vel, p[..., None]], axis=-1)


def _gpu(n, p):
    import torch
    from paper_1808_05066_gb300 import hdg
    mesh = hdg.Mesh(2, n, 0.0, 1.0, p, bc=BC)
    ctx = hdg.Context(mesh, 1.4, MACH, RE, PR, 0)
    xnode, xfnode, _ = mesh.coords()
    dev = torch.device("cuda", 0)

    def entropy(prim):
        t = torch.from_numpy(np.ascontiguousarray(prim)).to(dev)
        out = torch.empty_like(t)
        hdg.hdg_prim_to_entropy(ctx.handle, t, t.numel() // t.shape[-1], out)
        return out
    V, Vh = entropy(_prim(xnode)), entropy(_prim(xfnode))
    hdg.hdg_ctx_set_boundary_state(ctx.handle, Vh.clone())
    src = torch.from_numpy(np.ascontiguousarray(wl.couette_source(xnode, 1.0 / RE))).to(dev)
    hist = torch.zeros_like(V)
    hdg.hdg_add_source(ctx.handle, src, 1.0, hist)
    torch.cuda.synchronize()
    return hdg, mesh, ctx, V, Vh, hist, src


def _oracle(n, p):
    from oracle import physics as ph
    from oracle.hdg import Problem, consistent_Q, interpolate_state
    from oracle.mesh import Mesh
    prob = Problem(Mesh(2, n, 0.0, 1.0, p, bc=[list(b) for b in BC]), ph.Physics(mach=MACH, reynolds=RE, prandtl=PR))
    V, Vh = interpolate_state(prob, lambda x: wl.couette_field(x, MACH, PR))
    prob.boundary_state = Vh.copy()
    src = np.stack([prob.source_weak(e, wl.couette_source(prob.mesh.xnode[e], 1.0 / RE))
                    for e in range(prob.mesh.E)])
    return prob, consistent_Q(prob, V, Vh), V, Vh, src


def test_add_source_matches_oracle():
    n, p = 3, 3
    hdg, mesh, ctx, V, Vh, hist, src = _gpu(n, p)
    prob, _, _, _, src_o = _oracle(n, p)
    h = hist.cpu().numpy()
    assert np.abs(h - src_o).max() <= 1e-13 * np.abs(src_o).max()
    hdg.hdg_add_source(ctx.handle, src, -0.5, hist)          # accumulates with its scale
    assert np.abs(hist.cpu().numpy() - 0.5 * src_o).max() <= 1e-13 * np.abs(src_o).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_steady_couette_newton_matches_oracle(precision):
    from oracle.hdg import newton_solve
    n, p = 4, 3
    hdg, mesh, ctx, V, Vh, hist, _ = _gpu(n, p)
    prob, Q, Vo, Vho, src_o = _oracle(n, p)
    assert rel_fro(V.cpu().numpy(), Vo) < 1e-14 and rel_fro(Vh.cpu().numpy(), Vho) < 1e-14
    res = newton_solve(prob, Q, Vo, Vho, 0.0, src_o, tol=1e-10, max_it=8)
    it, rn = hdg.hdg_newton_solve(ctx.handle, V, Vh, hist, 0.0, precision, 1e-10, 8)
    assert it == res.iters >= 1, (it, res.iters)
    assert rel_fro(V.cpu().numpy(), res.V) < 1e-10
    assert rel_fro(Vh.cpu().numpy(), res.Vhat) < 1e-10
    wall = prob.mesh.face_bc != 0                # the trace takes the wall state
    assert np.abs(Vh.cpu().numpy()[wall] - prob.boundary_state[wall]).max() <= 1e-12 * np.abs(Vho).max()


def test_add_source_on_mixed_degrees_is_unsupported():
    import torch
    from paper_1808_05066_gb300 import hdg
    pe = np.array([1, 2] * 12, dtype=np.int8)                 # 2 x 2 x 2 cube: 48 tets
    pe = np.resize(pe, 48)
    mesh = hdg.Mesh(3, 2, 0.0, 1.0, 2, p_per_elem=pe)
    ctx = hdg.Context(mesh, 1.4, 0.3, 100.0, 0.71, 0)
    buf = torch.zeros(mesh.info["len_V"], dtype=torch.float64, device="cuda")
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_add_source(ctx.handle, buf, 1.0, buf.clone())
    assert ei.value.code == hdg.HDG_ERR_UNSUPPORTED


@pytest.mark.parametrize("scheme", ["hdg", "iedg", "edg"])
def test_steady_ringleb_newton_matches_oracle(scheme):
    import torch
    from paper_1808_05066_gb300 import hdg
    from oracle import physics as ph
    from oracle.hdg import Problem, face_states, interpolate_state, newton_solve
    from oracle.mesh import Mesh
    n, p, shift = 4, 2, np.array([-5.0, 1.0])          # the box [0, 4]^2 moved onto (-5, -1) x (1, 5)
    bc = (("state", "state"), ("state", "state"))

    def prim(x):
        rho, vel, pr = wl.ringleb_field(np.asarray(x) + shift)
        return np.concatenate([rho[..., None], vel, pr[..., None]], axis=-1)
    prob = Problem(Mesh(2, n, 0.0, 4.0, p, bc=[list(b) for b in bc]), ph.Physics(mach=0.5), scheme=scheme)
    Vo, Vho = interpolate_state(prob, lambda x: wl.ringleb_field(np.asarray(x) + shift))
    prob.boundary_state = face_states(prob, Vo)
    res = newton_solve(prob, None, Vo, Vho, 0.0, None, tol=1e-9, max_it=8)   # |R|: 7e-3, 8e-6, 8e-11
    for precision in (0, 1):
        mesh = hdg.Mesh(2, n, 0.0, 4.0, p, bc=bc, scheme={"hdg": hdg.HDG_SCHEME_HDG, "iedg": hdg.HDG_SCHEME_IEDG,
                                                          "edg": hdg.HDG_SCHEME_EDG}[scheme])
        ctx = hdg.Context(mesh, 1.4, 0.5, 0.0, 0.71, 0)
        xnode, xfnode, _ = mesh.coords()
        dev = torch.device("cuda", 0)
        V = torch.from_numpy(np.ascontiguousarray(prim(xnode))).to(dev)
        Vh = torch.from_numpy(np.ascontiguousarray(prim(xfnode))).to(dev)
        hdg.hdg_prim_to_entropy(ctx.handle, V.clone(), V.numel() // 4, V)
        hdg.hdg_prim_to_entropy(ctx.handle, Vh.clone(), Vh.numel() // 4, Vh)
        hdg.hdg_ctx_set_boundary_state(ctx.handle, Vh.clone())
        assert rel_fro(V.cpu().numpy(), Vo) < 1e-14 and rel_fro(Vh.cpu().numpy(), Vho) < 1e-14
        it, rn = hdg.hdg_newton_solve(ctx.handle, V, Vh, None, 0.0, precision, 1e-9, 8)
        assert it == res.iters >= 1, (precision, it, res.iters)
        assert rel_fro(V.cpu().numpy(), res.V) < 1e-10
        assert rel_fro(Vh.cpu().numpy(), res.Vhat) < 1e-10
