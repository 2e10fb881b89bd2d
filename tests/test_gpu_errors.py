"""The error contract of the C-ABI on the GPU: every HDG_ERR_* code the header declares for a
compute call is produced by input data or by a call's own limits, and the per-element status
bits say which elements caused it. Nothing here faults or hangs a GPU: the failures are a
non-physical state, a time coefficient that is not a number, iteration limits, a refinement
tolerance no block can meet, and a bounded wait that runs out because the host asked the
kernel not to issue the copy it waits for."""
import math

import numpy as np
import pytest

from hdg_cases import CASES, GpuCase, rel_fro

pytestmark = pytest.mark.gpu


def _code(fn):
    from paper_1808_05066_gb300 import hdg
    with pytest.raises(hdg.HdgError) as ei:
        fn()
    return ei.value.code


def test_gmres_iteration_limit_is_not_converged():
    gc = GpuCase(CASES["ns2d_p3"])
    hdg = gc.hdg
    gc.assemble(gc.history())
    dVh = gc.torch.empty_like(gc.Vhat)
    code = _code(lambda: hdg.hdg_trace_solve(gc.ctx.handle, gc.S, gc.g, dVh, hdg.HDG_SOLVER_GMRES, 1e-13, 1))
    assert code == hdg.HDG_ERR_NOT_CONVERGED
    # the same system solves with enough iterations
    it, res = hdg.hdg_trace_solve(gc.ctx.handle, gc.S, gc.g, dVh, hdg.HDG_SOLVER_GMRES, 1e-13, 2000)
    assert res <= 1e-13 and it > 1


def test_newton_update_limit_is_not_converged():
    gc = GpuCase(CASES["euler2d_p2"])
    hdg = gc.hdg
    V, Vh = gc.V.clone(), gc.Vhat.clone()
    code = _code(lambda: hdg.hdg_newton_step(gc.ctx.handle, V, Vh, gc.V, None, 0.05, 1, 0, 1e-10, 0))
    assert code == hdg.HDG_ERR_NOT_CONVERGED
    assert gc.torch.equal(V, gc.V) and gc.torch.equal(Vh, gc.Vhat)   # no update was made


def test_nonphysical_state_in_newton():
    gc = GpuCase(CASES["euler2d_p2"])
    hdg = gc.hdg
    V = gc.V.clone()
    V[7, 2, -1] = 0.25                      # v_m > 0 at one node
    Vh = gc.Vhat.clone()
    code = _code(lambda: hdg.hdg_newton_step(gc.ctx.handle, V, Vh, gc.V, None, 0.05, 1, 0, 1e-10, 5))
    assert code == hdg.HDG_ERR_NONPHYSICAL


@pytest.mark.parametrize("precision", [0, 1])
def test_non_finite_time_coefficient_is_singular(precision):
    """A time coefficient that is not a number leaves no usable pivot in any element block:
    every element reports SINGULAR (the state itself is physical) and the Newton solve
    returns HDG_ERR_SINGULAR."""
    gc = GpuCase(CASES["ns2d_p3"])
    hdg = gc.hdg
    hist = gc.history()
    gc.status.zero_()
    hdg.hdg_assemble_condense(gc.ctx.handle, gc.V, gc.Vhat, hist, math.nan, precision, gc.S, gc.g, gc.recov,
                              gc.R, gc.status)
    st = gc.status.cpu().numpy()
    assert (st & hdg.HDG_ELEM_SINGULAR).all()
    assert not (st & hdg.HDG_ELEM_NONPHYSICAL).any()
    V, Vh = gc.V.clone(), gc.Vhat.clone()
    code = _code(lambda: hdg.hdg_newton_solve(gc.ctx.handle, V, Vh, hist, math.nan, precision, 1e-10, 3))
    assert code == hdg.HDG_ERR_SINGULAR


def test_refinement_failure_fallback_and_error():
    """Mixed form with a refinement tolerance no block meets (0): with the FP64 recomputation
    on (the default behaviour) every element carries HDG_ELEM_FP64 and its outputs are the FP64
    form's bit for bit; with it off the REFINE bit stays and the Newton solve returns
    HDG_ERR_REFINE."""
    gc = GpuCase(CASES["ns3d_p2"])
    hdg, torch = gc.hdg, gc.torch
    hist = gc.history()
    gc.assemble(hist, precision=0)
    ref = [t.clone() for t in (gc.S, gc.g, gc.recov, gc.R)]
    hdg.hdg_ctx_set_refinement(gc.ctx.handle, 0.0, True)
    gc.assemble(hist, precision=1)
    st = gc.status.cpu().numpy()
    assert (st == hdg.HDG_ELEM_FP64).all()
    for a, b in zip((gc.S, gc.g, gc.recov, gc.R), ref):
        assert torch.equal(a, b)
    hdg.hdg_ctx_set_refinement(gc.ctx.handle, 0.0, False)
    gc.assemble(hist, precision=1)
    st = gc.status.cpu().numpy()
    assert (st == hdg.HDG_ELEM_REFINE).all()
    V, Vh = gc.V.clone(), gc.Vhat.clone()
    code = _code(lambda: hdg.hdg_newton_solve(gc.ctx.handle, V, Vh, hist, gc.case.mass_coef, 1, 1e-10, 3))
    assert code == hdg.HDG_ERR_REFINE
    # the default tolerance: no flags, the mixed outputs within the parity tolerance of FP64
    hdg.hdg_ctx_set_refinement(gc.ctx.handle, 1e-10, True)
    gc.assemble(hist, precision=1)
    assert int(gc.status.abs().sum()) == 0
    S, S64 = gc.S.cpu().numpy(), ref[0].cpu().numpy()
    assert max(rel_fro(S[e], S64[e]) for e in range(S.shape[0])) < 1e-10


def test_invalid_arguments_of_compute_calls():
    gc = GpuCase(CASES["euler2d_p2"])
    hdg = gc.hdg
    V, Vh = gc.V.clone(), gc.Vhat.clone()
    assert _code(lambda: hdg.hdg_newton_step(gc.ctx.handle, V, Vh, gc.V, None, 0.05, 3, 0)) == \
        hdg.HDG_ERR_INVALID_ARG                                                  # bdf_order
    assert _code(lambda: hdg.hdg_newton_step(gc.ctx.handle, V, Vh, gc.V, None, 0.05, 2, 0)) == \
        hdg.HDG_ERR_INVALID_ARG                                                  # BDF2 without V^{n-1}
    assert _code(lambda: hdg.hdg_assemble_condense(gc.ctx.handle, V, Vh, None, 1.0, 5, gc.S, gc.g, gc.recov,
                                                   gc.R)) == hdg.HDG_ERR_INVALID_ARG  # precision
    assert _code(lambda: hdg.hdg_ctx_set_refinement(gc.ctx.handle, -1.0, True)) == hdg.HDG_ERR_INVALID_ARG
    assert _code(lambda: hdg.hdg_ctx_set_trace_solver(gc.ctx.handle, 9, 1e-12, 10)) == hdg.HDG_ERR_INVALID_ARG


def test_unsupported_configuration():
    """3D p = 4 runs on the element-class kernels for Navier-Stokes in the FP64 form only: Euler
    physics there, and the mixed form, say HDG_ERR_UNSUPPORTED."""
    import torch
    from paper_1808_05066_gb300 import hdg
    mesh = hdg.Mesh(3, 1, 0.0, 1.0, 4)
    assert _code(lambda: hdg.Context(mesh, 1.4, 0.1, 0.0, 0.71, 0)) == hdg.HDG_ERR_UNSUPPORTED
    ctx = hdg.Context(mesh, 1.4, 0.1, 1600.0, 0.71, 0)
    i = mesh.info
    buf = {k: torch.zeros(i["len_" + k], dtype=torch.float64, device="cuda") for k in ("V", "g", "S", "recov", "R")}
    Vh = torch.zeros(i["n_trace"], dtype=torch.float64, device="cuda")
    code = _code(lambda: hdg.hdg_assemble_condense(ctx.handle, buf["V"], Vh, None, 0.0, hdg.HDG_PREC_MIXED, buf["S"],
                                                   buf["g"], buf["recov"], buf["R"]))
    assert code == hdg.HDG_ERR_UNSUPPORTED


def test_tcgen05_condensation_wait_timeout(monkeypatch):
    """Every wait of the tcgen05 condensation is bounded. With the test hook that leaves its first
    operand copy unissued (a phase that nothing completes), the waits run out after about a
    second: the kernel sets HDG_ELEM_TIMEOUT, frees its tensor memory and returns, and the
    context stays usable. The FP64 recomputation then replaces the blocks (HDG_ELEM_FP64, the
    FP64 form's outputs bit for bit); without it the Newton solve returns HDG_ERR_TIMEOUT."""
    monkeypatch.setenv("HDG_COND_VARIANT", "3")
    monkeypatch.setenv("HDG_T5_STALL_FIRST_COPY", "1")
    gc = GpuCase(CASES["ns2d_p3"])
    hdg, torch = gc.hdg, gc.torch
    hist = gc.history()
    gc.assemble(hist, precision=0)
    ref = [t.clone() for t in (gc.S, gc.g, gc.recov, gc.R)]
    gc.assemble(hist, precision=1)
    assert (gc.status.cpu().numpy() == hdg.HDG_ELEM_FP64).all()
    for x, y in zip((gc.S, gc.g, gc.recov, gc.R), ref):
        assert torch.equal(x, y)
    hdg.hdg_ctx_set_refinement(gc.ctx.handle, 1e-10, False)
    gc.assemble(hist, precision=1)
    assert (gc.status.cpu().numpy() & hdg.HDG_ELEM_TIMEOUT).all()
    V, Vh = gc.V.clone(), gc.Vhat.clone()
    code = _code(lambda: hdg.hdg_newton_solve(gc.ctx.handle, V, Vh, hist, gc.case.mass_coef, 1, 1e-10, 2))
    assert code == hdg.HDG_ERR_TIMEOUT
    gc.assemble(hist, precision=0)             # the context still works
    assert torch.equal(gc.S, ref[0]) and int(gc.status.abs().sum()) == 0
