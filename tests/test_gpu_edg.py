"""GPU parity of the EDG scheme (Sec. 3.4: a continuous trace, one unknown per skeleton node) with
the oracle's EDG problem on the same seeded inputs: the element-local condensation (unchanged from
HDG, fed through the continuous numbering), the assembled trace solve (dense LU and GMRES with the
node-block Jacobi preconditioner), the recovery, and whole Newton steps."""
import dataclasses

import numpy as np
import pytest

from hdg_cases import CASES, GpuCase, oracle_hist, oracle_setup, rel_fro

pytestmark = pytest.mark.gpu

EDG = {name: dataclasses.replace(CASES[name], scheme="edg") for name in ("euler2d_p2", "ns2d_p3", "ns3d_p2")}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(EDG))
def test_edg_assemble_condense_matches_oracle(name, precision):
    case = EDG[name]
    gc = GpuCase(case)
    prob, Q, V, Vh = oracle_setup(case)
    assert gc.Vhat.shape == Vh.shape == (prob.n_edg, prob.m)
    assert rel_fro(gc.Vhat.cpu().numpy(), Vh) < 1e-14
    hist_o = oracle_hist(prob, V, case)
    gc.assemble(gc.history(), precision=precision)
    assert int(gc.status.abs().sum()) == 0
    S, g, rec, R = gc.S.cpu().numpy(), gc.g.cpu().numpy(), gc.recov.cpu().numpy(), gc.R.cpu().numpy()
    nv, nt = gc.info["nv"], gc.info["nt"]
    for e in sorted({0, 5, prob.mesh.E - 1}):
        L = prob.condense(e, None if Q is None else Q[e], V[e], prob.gather_trace(Vh, e), case.mass_coef, hist_o[e])
        nq = L["Rl"].size - nv
        scale = max(np.abs(L["Rl"]).max(), np.abs(L["Rt"]).max(), np.abs(hist_o[e]).max(), 1.0)
        assert np.abs(L["Rl"][nq:] - R[e, :nv]).max() <= 1e-12 * scale
        assert np.abs(L["Rt"] - R[e, nv:]).max() <= 1e-12 * scale
        assert rel_fro(S[e], L["S"]) < 1e-10 and rel_fro(g[e], L["g"]) < 1e-10
        assert rel_fro(rec[e, :nv * nt].reshape(nv, nt), L["X"][nq:]) < 1e-10


@pytest.mark.parametrize("method", [2, 1])
@pytest.mark.parametrize("name", ["euler2d_p2", "ns2d_p3"])
def test_edg_trace_solve_and_recovery_match_oracle(name, method):
    from oracle.hdg import newton_iteration
    case = EDG[name]
    gc = GpuCase(case)
    prob, Q, V, Vh = oracle_setup(case)
    hist_o = oracle_hist(prob, V, case)
    Qn, Vn, Vhn, rn, dvh, _ = newton_iteration(prob, Q, V, Vh, case.mass_coef, hist_o)
    gc.assemble(gc.history())
    torch = gc.torch
    dVh = torch.empty_like(gc.Vhat)
    it, res = gc.hdg.hdg_trace_solve(gc.ctx.handle, gc.S, gc.g, dVh, method, 1e-13, 2000)
    assert res < 1e-11
    assert rel_fro(dVh.cpu().numpy().ravel(), dvh) < 1e-9
    dV = torch.empty_like(gc.V)
    gc.hdg.hdg_recover_interior(gc.ctx.handle, gc.recov, dVh, dV)
    assert rel_fro(dV.cpu().numpy(), Vn - V) < 1e-9
    assert abs(gc.hdg.hdg_residual_norm(gc.ctx.handle, gc.R) - rn) <= 1e-12 * rn


@pytest.mark.parametrize("name,precision,order", [("euler2d_p2", 0, 1), ("ns2d_p3", 0, 2), ("ns2d_p3", 1, 2)])
def test_edg_newton_step_matches_oracle(name, precision, order):
    """A BDF step of the EDG scheme to |R| <= 1e-10 max(1, |R0|), GMRES trace solves with the
    node-block preconditioner, against the oracle's (dense trace solves): the same Newton updates
    and the same state."""
    from oracle.hdg import time_step
    case = EDG[name]
    gc = GpuCase(case)
    prob, Q, V, Vh = oracle_setup(case)
    dt = 0.05
    hist = [V] if order == 1 else [V, V * (1.0 + 1e-3)]
    res = time_step(prob, Q, V, Vh, hist, order, dt, tol=1e-10, max_it=10)
    gc.hdg.hdg_ctx_set_trace_solver(gc.ctx.handle, gc.hdg.HDG_SOLVER_GMRES, 1e-13, 3000)
    V_gpu, Vh_gpu = gc.V.clone(), gc.Vhat.clone()
    V_nm1 = None if order == 1 else (gc.V * (1.0 + 1e-3)).contiguous()
    it, rn = gc.hdg.hdg_newton_step(gc.ctx.handle, V_gpu, Vh_gpu, gc.V, V_nm1, dt, order, precision, 1e-10, 10)
    assert it == res.iters, (it, res.iters)
    assert rel_fro(V_gpu.cpu().numpy(), res.V) < 1e-10
    assert rel_fro(Vh_gpu.cpu().numpy(), res.Vhat) < 1e-10
