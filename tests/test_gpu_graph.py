"""hdg_assemble_condense_graph: the captured launch sequence gives the ordinary call's S, g,
recovery data, residuals and status bit for bit, reads new values from the same buffers,
and captures again when an argument changes. hdg_ctx_graph_replays shows that the graph
really was launched (a failed capture would leave the ordinary path and no replays)."""
import pytest

from hdg_cases import CASES, GpuCase

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("with_status", [True, False])
@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_ordinary_call(precision, with_status):
    import torch

    gc = GpuCase(CASES["ns3d_p2"])
    hdg = gc.hdg
    hist = gc.history()

    def run(fn, S):
        gc.status.zero_()
        fn(gc.ctx.handle, gc.V, gc.Vhat, hist, gc.case.mass_coef, precision, S, gc.g, gc.recov, gc.R,
           gc.status if with_status else None)
        torch.cuda.synchronize()
        return [t.clone() for t in (S, gc.g, gc.recov, gc.R, gc.status)]

    def same(a, b):
        return all(torch.equal(x, y) for x, y in zip(a, b))

    replays = lambda: hdg.hdg_ctx_graph_replays(gc.ctx.handle)
    ref = run(hdg.hdg_assemble_condense, gc.S)
    assert replays() == 0
    for _ in range(3):  # the ordinary call and the capture, then replays
        assert same(run(hdg.hdg_assemble_condense_graph, gc.S), ref)
    assert replays() == 2
    # new values in the same input buffers: the replay reads them
    gc.V.mul_(1.0 + 1e-4)
    ref2 = run(hdg.hdg_assemble_condense, gc.S)
    assert not torch.equal(ref2[0], ref[0])
    assert same(run(hdg.hdg_assemble_condense_graph, gc.S), ref2)
    assert replays() == 3
    # another output buffer: captured again, then replayed
    S2 = torch.empty_like(gc.S)
    for _ in range(2):
        assert same(run(hdg.hdg_assemble_condense_graph, S2), ref2)
    assert replays() == 4
