"""hdg_assemble_condense_noalloc: the FP64 assemble + condense for callers that cannot
allocate device memory during the call (e.g. while a stream is captured into a CUDA
graph, or inside a runtime that owns a fixed arena). Its scratch lives in a static device
array, so this test checks, through the C-ABI, that two calls in a row — on different
inputs, sharing that array — reproduce the ordinary entry point's outputs. The file name
makes pytest collect it last."""
import numpy as np
import pytest

from hdg_cases import CASES, GpuCase, rel_fro

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the parity tolerance of the condensed blocks


@pytest.mark.parametrize("name", ["ns3d_p3", "ns2d_p4"])
def test_noalloc_matches_allocating_entry_point(name):
    torch = pytest.importorskip("torch")
    gc = GpuCase(CASES[name])
    hdg = gc.hdg
    hist = gc.history()
    inputs = [(gc.V.clone(), gc.Vhat.clone()),
              ((gc.V * (1 + 1e-4)).contiguous(), (gc.Vhat * (1 - 1e-4)).contiguous())]
    refs = []
    for V, Vh in inputs:
        gc.V, gc.Vhat = V, Vh
        gc.assemble(hist)
        refs.append([t.clone() for t in (gc.S, gc.g, gc.recov, gc.R)])
    for (V, Vh), ref in zip(inputs, refs):       # two calls in a row
        outs = [torch.full_like(t, float("nan")) for t in ref]
        status = torch.zeros_like(gc.status)
        hdg.hdg_assemble_condense_noalloc(gc.ctx.handle, V, Vh, hist, gc.case.mass_coef, *outs, status)
        torch.cuda.synchronize()
        assert int(status.abs().sum()) == 0
        for o, r in zip(outs, ref):
            o, r = o.cpu().numpy(), r.cpu().numpy()
            assert np.isfinite(o).all()
            assert rel_fro(o, r) <= TOL
