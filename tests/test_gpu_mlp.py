"""The learned warm start: GPU kernels (BF16 weights, FP32 accumulation) against the
FP64 MLP oracle, and a short BDF2 run where the trained network is compared with the
plain extrapolated start at the same Newton tolerance."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _params_np(params, P):
    """Master weights and the BF16 copy (as float64) from a parameter buffer."""
    import torch
    flat = params.detach()
    master = flat[:P].double().cpu().numpy()
    w16 = flat[3 * P:3 * P + (P + 1) // 2].view(torch.bfloat16)[:P].double().cpu().numpy()
    return master, w16


@pytest.mark.parametrize("sizes", [(64, 64, 16), (48, 32, 12)])
def test_mlp_forward_and_gradient_match_oracle(sizes):
    import torch
    from oracle import mlp as omlp
    from paper_1808_05066_gb300 import hdg
    nin, nh, nout = sizes
    P = hdg.hdg_mlp_param_count(nin, nh, nout)
    assert P == nh * nin + nh + nh * nh + nh + nout * nh + nout
    dev = torch.device("cuda", 0)
    params = torch.empty(((14 * P + 3) // 4,), dtype=torch.float32, device=dev)
    hdg.hdg_mlp_init(params, nin, nh, nout, 11)
    rng = np.random.default_rng(4)
    B = 1000
    x = rng.normal(size=(B, nin)).astype(np.float32)
    t = rng.normal(scale=0.3, size=(B, nout)).astype(np.float32)
    xd, td = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    y = torch.empty((B, nout), dtype=torch.float32, device=dev)
    hdg.hdg_mlp_forward(params, nin, nh, nout, xd, B, y)
    grad = torch.empty(P, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    hdg.hdg_mlp_gradient(params, grad, nin, nh, nout, xd, td, B, loss)
    torch.cuda.synchronize()
    master, w16 = _params_np(params, P)
    assert np.all(np.abs(master - w16) <= 2 ** -8 * np.abs(master) + 1e-30)
    y_o, _ = omlp.forward(w16, x.astype(np.float64), nin, nh, nout)
    g_o = omlp.gradient(w16, x.astype(np.float64), t.astype(np.float64), nin, nh, nout)
    assert np.abs(y.cpu().numpy() - y_o).max() <= 1e-4 * np.abs(y_o).max()
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - g_o) <= 1e-3 * np.linalg.norm(g_o)
    assert abs(float(loss.item()) - omlp.loss(w16, x.astype(np.float64), t.astype(np.float64), nin, nh, nout)) \
        <= 1e-4 * abs(float(loss.item()))
    # one Adam step on the master weights, against the update written out
    hdg.hdg_mlp_train_step(params, grad, nin, nh, nout, xd, td, B, 1e-3, 1, loss)
    torch.cuda.synchronize()
    new_master, _ = _params_np(params, P)
    gg = grad.double().cpu().numpy()
    m = 0.1 * gg
    v = 0.001 * gg * gg
    ref = master - 1e-3 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    assert np.allclose(new_master, ref, rtol=1e-5, atol=1e-7)


def test_learned_warm_start_against_plain_start():
    """BDF2 on the small vortex patch: train on 14 plain steps, then from the same state
    run 6 steps each with the plain extrapolated start, the element-local correction alone
    (trace held at its extrapolation; an ablation) and the network's trace with the local
    recovery. Checked: training lowers the loss; the learned start has a smaller initial
    Newton residual than the plain start and needs no more global Newton updates; every
    run converges to |R| <= 1e-10 and ends in the same state. The ablation numbers are
    printed: on this case the gain over the plain start comes from the local correction,
    and the network's trace correction does not improve on holding the extrapolation."""
    import torch
    from paper_1808_05066_gb300 import hdg
    from paper_1808_05066_gb300.warmstart import Stepper, collect_and_train
    from paper_1808_05066_gb300.workload import DeviceWorkload
    W = DeviceWorkload("ns2d_p3_vortices_small", outputs=False)
    st = Stepper(W, precision=hdg.HDG_PREC_MIXED, tol=1e-10)
    recs, net = collect_and_train(st, 16, skip=2, epochs=60, lr=2e-3)
    assert net.losses[-1] < 0.9 * net.losses[0]
    snap = st.state()
    runs = {}
    for warm in ("plain", "local", "mlp"):
        st.restore(snap)
        runs[warm] = ([st.step(warm, net) for _ in range(6)], st.V.clone())
    gm = {k: float(np.exp(np.mean([np.log(r.res_history[0]) for r in v[0]]))) for k, v in runs.items()}
    upd = {k: sum(r.newton_updates for r in v[0]) for k, v in runs.items()}
    print("initial residual geomean", gm, "newton updates", upd)
    assert all(r.warm == "mlp" for r in runs["mlp"][0])
    assert gm["mlp"] < 0.5 * gm["plain"]
    assert upd["mlp"] <= upd["plain"]
    for k in ("local", "mlp"):
        assert float((runs[k][1] - runs["plain"][1]).norm() / runs["plain"][1].norm()) < 1e-8
