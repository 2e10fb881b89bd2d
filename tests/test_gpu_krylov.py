"""GMRES with device-resident restart cycles: each cycle's Arnoldi steps run on the GPU without
a host round trip and are replayed as a CUDA graph. The solution matches the oracle's dense
trace solve, the iteration count equals that of the same solve with the tolerance reached, and the
cycles were graph replays; a second solve on the same buffers replays the same graph."""
import pytest

from hdg_cases import CASES, GpuCase, oracle_hist, oracle_setup, rel_fro

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["euler2d_p2", "ns2d_p3"])
def test_gmres_cycles_replay_as_graphs_and_match_oracle(name):
    from oracle.hdg import newton_iteration
    case = CASES[name]
    gc = GpuCase(case)
    prob, Q, V, Vh = oracle_setup(case)
    hist_o = oracle_hist(prob, V, case)
    _Qn, _Vn, _Vhn, _rn, dvh, _ = newton_iteration(prob, Q, V, Vh, case.mass_coef, hist_o)
    gc.assemble(gc.history())
    hdg, torch = gc.hdg, gc.torch
    c0, r0 = hdg.hdg_ctx_trace_cycles(gc.ctx.handle)
    dVh = torch.empty_like(gc.Vhat)
    it1, res1 = hdg.hdg_trace_solve(gc.ctx.handle, gc.S, gc.g, dVh, hdg.HDG_SOLVER_GMRES, 1e-13, 2000)
    c1, r1 = hdg.hdg_ctx_trace_cycles(gc.ctx.handle)
    assert res1 <= 1e-12
    assert rel_fro(dVh.cpu().numpy().ravel(), dvh) < 1e-9
    assert c1 - c0 >= max(1, (it1 + 29) // 30)       # at least one cycle per 30 iterations
    assert r1 - r0 == c1 - c0                         # every cycle was a graph replay
    # the same solve again: the captured graph is replayed, with the same iterations and result
    dVh2 = torch.empty_like(gc.Vhat)
    it2, res2 = hdg.hdg_trace_solve(gc.ctx.handle, gc.S, gc.g, dVh2, hdg.HDG_SOLVER_GMRES, 1e-13, 2000)
    c2, r2 = hdg.hdg_ctx_trace_cycles(gc.ctx.handle)
    assert it2 == it1 and r2 - r1 == c2 - c1 > 0
    assert rel_fro(dVh2.cpu().numpy().ravel(), dvh) < 1e-9
    # the iteration limit still stops a solve mid-cycle with HDG_ERR_NOT_CONVERGED
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_trace_solve(gc.ctx.handle, gc.S, gc.g, dVh2, hdg.HDG_SOLVER_GMRES, 1e-13, 7)
    assert ei.value.code == hdg.HDG_ERR_NOT_CONVERGED


@pytest.mark.parametrize("precision", [0, 1])
def test_newton_iterations_replay_graphs(precision):
    """A BDF1 Newton step with GMRES trace solves: every update after the first replays the
    captured assemble + condense sequence, every GMRES cycle is a graph replay, and the step
    reaches the same state as the oracle's time step."""
    from oracle.hdg import time_step
    case = CASES["euler2d_p2"]
    gc = GpuCase(case)
    prob, Q, V, Vh = oracle_setup(case)
    dt = 0.05
    res = time_step(prob, Q, V, Vh, [V], 1, dt, tol=1e-12, max_it=10)
    hdg = gc.hdg
    hdg.hdg_ctx_set_trace_solver(gc.ctx.handle, hdg.HDG_SOLVER_GMRES, 1e-13, 2000)
    g0 = hdg.hdg_ctx_graph_replays(gc.ctx.handle)
    c0, r0 = hdg.hdg_ctx_trace_cycles(gc.ctx.handle)
    V_gpu, Vh_gpu = gc.V.clone(), gc.Vhat.clone()
    it, rn = hdg.hdg_newton_step(gc.ctx.handle, V_gpu, Vh_gpu, gc.V, None, dt, 1, precision, 1e-12, 10)
    g1 = hdg.hdg_ctx_graph_replays(gc.ctx.handle)
    c1, r1 = hdg.hdg_ctx_trace_cycles(gc.ctx.handle)
    assert it == res.iters >= 2
    assert g1 - g0 == it                    # it + 1 assemblies: the first captures, the rest replay
    assert c1 - c0 >= it and r1 - r0 == c1 - c0
    assert rel_fro(V_gpu.cpu().numpy(), res.V) < 1e-10
    assert rel_fro(Vh_gpu.cpu().numpy(), res.Vhat) < 1e-10
