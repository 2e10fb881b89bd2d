"""hdg_assemble_condense_noalloc: the FP64 assemble + condense for callers that cannot
allocate device memory during the call, such as a runtime that owns a fixed memory arena
and forbids further cudaMalloc/cudaFree. Its scratch lives in a static device array shared
by every call, so these tests check, through the C-ABI, that two calls in a row (on
different inputs, sharing that array) reproduce the ordinary entry point's outputs, also on
a mesh with more elements than one pass over the array holds (the array is reused chunk
after chunk within a call). The file name makes pytest collect it last."""
import dataclasses

import numpy as np
import pytest

from hdg_cases import CASES, GpuCase, rel_fro

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the parity tolerance of the condensed blocks

# one ns3d_p3 element needs 60,400 doubles of scratch, so the 64 MiB array holds 138
# elements per chunk: the 4^3 x 6 = 384-element mesh takes three chunks
CHUNKED = dataclasses.replace(CASES["ns3d_p3"], name="ns3d_p3_n4", n=4)


@pytest.mark.parametrize("case", [CASES["ns3d_p3"], CASES["ns2d_p4"], CHUNKED], ids=lambda c: c.name)
def test_noalloc_matches_allocating_entry_point(case):
    torch = pytest.importorskip("torch")
    gc = GpuCase(case)
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
