"""GPU parity of the mixed-degree assemble + condense (one persistent launch over the element
classes (p_e, largest face degree)) against the FP64 oracle, element by element, on 3D
Navier-Stokes tetrahedra with seeded random degrees 1..4 (face degree max(p_L, p_R)); every class
present is compared on every element, or on a seeded sample for the larger mesh."""
import functools
import math

import numpy as np
import pytest

import workloads as wl
from hdg_cases import rel_fro

pytestmark = pytest.mark.gpu

MACH, RE, PR = 0.1, 1600.0, 0.71
L = 2 * math.pi
MASS = 20.0


def _prim(x):
    rho, vel, p = wl.tgv_field(x * (2 * math.pi / L) + 0.3, MACH)
    return np.concatenate([rho[..., None], vel, p[..., None]], axis=-1)


def _setup(n, degs, seed, stabilization="slf"):
    import torch
    from oracle import physics as ph
    from oracle.hdg import Problem, consistent_Q, interpolate_state
    from oracle.mesh import Mesh as OMesh
    from paper_1808_05066_gb300 import hdg
    E = 6 * n ** 3
    pe = np.random.default_rng(seed).choice(degs, size=E).astype(np.int8)
    # oracle
    om = OMesh(3, n, 0.0, L, 0, p_elem=pe)
    prob = Problem(om, ph.Physics(mach=MACH, reynolds=RE, prandtl=PR, stabilization=stabilization))
    prim_fn = lambda x: wl.tgv_field(x * (2 * math.pi / L) + 0.3, MACH)
    V, Vh = interpolate_state(prob, prim_fn)
    Vh = wl.perturb(Vh, 1e-3, seed + 1)
    hist = [prob.history_weak(e, [V[e] * (1 + 1e-3)], [MASS]) for e in range(om.E)]
    # GPU: its own mesh, coordinates and state conversion
    mesh = hdg.Mesh(3, n, 0.0, L, 0, p_per_elem=pe)
    ctx = hdg.Context(mesh, 1.4, MACH, RE, PR, stabilization=1 if stabilization == "s" else 0)
    info, lay = mesh.info, mesh.layout()
    xnode, xfnode, _ = mesh.coords()
    dev = torch.device("cuda", 0)

    def to_v(prim):
        t = torch.from_numpy(np.ascontiguousarray(prim)).to(dev)
        out = torch.empty_like(t)
        hdg.hdg_prim_to_entropy(ctx.handle, t, t.numel() // 5, out)
        return out

    Vg = to_v(_prim(xnode)).reshape(-1)
    Vhg = to_v(_prim(xfnode))
    Vhg = torch.from_numpy(wl.perturb(Vhg.cpu().numpy(), 1e-3, seed + 1)).to(dev).contiguous()
    histg = torch.from_numpy(np.concatenate([h.ravel() for h in hist])).to(dev)
    return prob, V, Vh, hist, (hdg, mesh, ctx, info, lay, Vg, Vhg, histg, pe)


def _run_gpu(g):
    import torch
    hdg, mesh, ctx, info, lay, Vg, Vhg, histg, pe = g
    dev = Vg.device
    out = dict(S=torch.empty(info["len_S"], dtype=torch.float64, device=dev),
               g=torch.empty(info["len_g"], dtype=torch.float64, device=dev),
               recov=torch.empty(info["len_recov"], dtype=torch.float64, device=dev),
               R=torch.empty(info["len_R"], dtype=torch.float64, device=dev))
    st = torch.zeros(info["n_elem"], dtype=torch.int32, device=dev)
    hdg.hdg_assemble_condense(ctx.handle, Vg, Vhg, histg, MASS, hdg.HDG_PREC_FP64, out["S"], out["g"],
                              out["recov"], out["R"], st)
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare(prob, V, Vh, hist, g, res, elems):
    lay = g[4]
    worst = {}
    for e in elems:
        Q = prob.consistent_q(e, V[e], prob.gather_trace(Vh, e))
        ref = prob.condense(e, Q, V[e], prob.gather_trace(Vh, e), MASS, hist[e])
        nt = int(lay["toff"][e + 1] - lay["toff"][e])
        nv = V[e].size
        S = res["S"][lay["soff"][e]:lay["soff"][e + 1]].reshape(nt, nt)
        ge = res["g"][lay["toff"][e]:lay["toff"][e + 1]]
        rec = res["recov"][lay["roff"][e]:lay["roff"][e + 1]]
        X, y = rec[:nv * nt].reshape(nv, nt), rec[nv * nt:]
        R = res["R"][lay["Roff"][e]:lay["Roff"][e + 1]]
        nq = Q.size                               # the oracle keeps q; compare the v rows
        errs = dict(S=rel_fro(S, ref["S"]), g=rel_fro(ge, ref["g"]), X=rel_fro(X, ref["X"][nq:]),
                    y=rel_fro(y, ref["y"][nq:]))
        # residuals against the oracle's v rows (its q rows vanish at the consistent q), relative to
        # the largest of the terms they sum
        Rv = ref["Rl"][nq:]
        scale = max(np.abs(Rv).max(), np.abs(ref["Rt"]).max(), np.abs(hist[e]).max(), 1.0)
        errs["Rv"] = float(np.abs(R[:nv] - Rv).max() / scale)
        errs["Rt"] = float(np.abs(R[nv:] - ref["Rt"]).max() / scale)
        key = (int(prob.mesh.p_elem[e]), int(prob.mesh.elem_trace_deg[e]))
        for k, v in errs.items():
            worst[(key, k)] = max(worst.get((key, k), 0.0), v)
    return worst


# classes covered: (1,4), (4,4) (every element); (1,2) (1,3) (2,2) (2,3) (3,3) ... (three of each);
# (1,4) (2,4) (3,3) (3,4) (4,4) (one of each: a p = 4 element costs the oracle about 4 s)
@pytest.mark.parametrize("n,degs,seed,sample", [(1, (1, 2, 3, 4), 3, None), (2, (1, 2, 3), 5, 3),
                                                (2, (1, 2, 3, 4), 7, 1)])
def test_mixed_degree_condensation_matches_oracle(n, degs, seed, sample):
    prob, V, Vh, hist, g = _setup(n, degs, seed)
    res = _run_gpu(g)
    E = prob.mesh.E
    if sample is None:
        elems = range(E)
    else:   # up to `sample` elements of every class present
        rng = np.random.default_rng(seed)
        cls = [(int(prob.mesh.p_elem[e]), int(prob.mesh.elem_trace_deg[e])) for e in range(E)]
        elems = []
        for c in sorted(set(cls)):
            ids = [e for e in range(E) if cls[e] == c]
            elems += list(rng.choice(ids, size=min(sample, len(ids)), replace=False))
    worst = _compare(prob, V, Vh, hist, g, res, elems)
    classes = sorted({k[0] for k in worst})
    assert len(classes) >= 2, classes
    for (cls, k), v in worst.items():
        tol = 1e-12 if k in ("Rv", "Rt") else 1e-10
        assert v <= tol, (cls, k, v)


@functools.lru_cache(maxsize=None)
def _oracle_bdf2_step(dt):
    from oracle.hdg import time_step
    prob, V, Vh, _hist, _g = _setup(2, (1, 2), 9)
    Q = [prob.consistent_q(e, V[e], prob.gather_trace(Vh, e)) for e in range(prob.mesh.E)]
    return time_step(prob, Q, V, Vh, [V, [v * (1.0 + 1e-3) for v in V]], 2, dt, tol=1e-12, max_it=12)


@pytest.mark.parametrize("solver", ["dense", "gmres"])
def test_mixed_degree_bdf_newton_step_matches_oracle(solver):
    """One BDF2 time step on a mixed-degree mesh (3D Navier-Stokes, degrees 1 and 2, 48 tets):
    hdg_newton_step (condensation in one persistent launch, trace solve with the dense LU or
    GMRES with face blocks of each face's own size, recovery) against the oracle's time step: the
    same Newton updates, the same first residual and the same state."""
    import torch
    prob, V, Vh, _hist, g = _setup(2, (1, 2), 9)
    hdg, mesh, ctx, info, lay, Vg, Vhg, _histg, pe = g
    dt = 0.05
    res = _oracle_bdf2_step(dt)
    hdg.hdg_ctx_set_trace_solver(ctx.handle, hdg.HDG_SOLVER_DENSE if solver == "dense" else hdg.HDG_SOLVER_GMRES,
                                 1e-13, 3000)
    V_gpu, Vh_gpu = Vg.clone(), Vhg.clone()
    V_nm1 = (Vg * (1.0 + 1e-3)).contiguous()
    it, rn, rh, _tr = hdg.hdg_newton_step(ctx.handle, V_gpu, Vh_gpu, Vg, V_nm1, dt, 2, hdg.HDG_PREC_FP64, 1e-12, 12,
                                          history=True)
    torch.cuda.synchronize()
    assert it == res.iters, (it, res.iters)
    assert abs(rh[0] - res.res_norms[0]) <= 1e-12 * res.res_norms[0]
    assert rn <= 1e-12 * max(1.0, rh[0])
    Vo = np.concatenate([v.ravel() for v in res.V])
    assert rel_fro(V_gpu.cpu().numpy(), Vo) < 1e-10
    assert rel_fro(Vh_gpu.cpu().numpy().reshape(-1), res.Vhat.reshape(-1)) < 1e-10


def test_uniform_3d_p4_runs_on_the_class_kernels():
    """3D Navier-Stokes at one degree p = 4 (no uniform kernels): the mesh keeps the uniform
    layout and the element-class launch condenses it; two elements against the oracle."""
    prob, V, Vh, hist, g = _setup(1, (4,), 13)
    assert g[3]["mixed"] == 0 and g[3]["p"] == 4 and g[3]["nt"] == 300 and g[3]["nv"] == 175
    lay = g[4]
    assert list(lay["soff"][:3]) == [0, 300 * 300, 2 * 300 * 300]
    res = _run_gpu(g)
    worst = _compare(prob, V, Vh, hist, g, res, [0, 5])
    for (cls, k), v in worst.items():
        assert cls == (4, 4)
        assert v <= (1e-12 if k in ("Rv", "Rt") else 1e-10), (k, v)


def test_mixed_degree_with_symmetric_stabilization():
    """The fused launch with sigma_S = |A_n| A0 (Eq. symStab) in place of sigma_SLF, every element
    of a six-tet mesh of degrees 1..3 against the oracle."""
    prob, V, Vh, hist, g = _setup(1, (1, 2, 3), 17, stabilization="s")
    res = _run_gpu(g)
    worst = _compare(prob, V, Vh, hist, g, res, range(prob.mesh.E))
    for (cls, k), v in worst.items():
        assert v <= (1e-12 if k in ("Rv", "Rt") else 1e-10), (cls, k, v)


def test_mixed_degree_dirk3_step_matches_oracle():
    """One DIRK(3,3) step (Sec. 5's integrator) on a mesh of degrees 1 and 2: the same Newton
    updates per stage and the same state as the oracle's DIRK step."""
    import torch
    from oracle.hdg import dirk3_step
    prob, V, Vh, _hist, g = _setup(1, (1, 2), 21)
    hdg, mesh, ctx, info, lay, Vg, Vhg, _histg, pe = g
    Q = [prob.consistent_q(e, V[e], prob.gather_trace(Vh, e)) for e in range(prob.mesh.E)]
    dt = 0.05
    res, iters = dirk3_step(prob, Q, V, Vh, dt, tol=1e-10, max_it=10)
    V_gpu, Vh_gpu = Vg.clone(), Vhg.clone()
    its, rn, tr = hdg.hdg_dirk3_step(ctx.handle, V_gpu, Vh_gpu, Vg, dt, hdg.HDG_PREC_FP64, 1e-10, 10)
    torch.cuda.synchronize()
    assert list(its) == list(iters), (its, iters)
    assert rel_fro(V_gpu.cpu().numpy(), np.concatenate([v.ravel() for v in res.V])) < 1e-10
    assert rel_fro(Vh_gpu.cpu().numpy().reshape(-1), res.Vhat.reshape(-1)) < 1e-10
