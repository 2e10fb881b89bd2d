"""Implicit time stepping with Newton, with and without the learned warm start.

Orchestration only: every arithmetic step (extrapolation, features, network, training, the
time step with its warm start) is a C-ABI call into libhdg.so.

Time integration is BDF2 (BDF1 for the first step). With the extrapolation
V_e = 2 V^n - V^{n-1}, vhat_e = vhat^n + dvhat^n (dvhat^n = vhat^n - vhat^{n-1}), the
initial guess of step n+1 is
  plain:  (V_e, vhat_e);
  local:  vhat_e, and V from one element-local Newton correction at (V_e, vhat_e) with the
          trace held: assemble+condense, dV = -y (recovery with dvhat = 0);
  mlp:    vhat_m = vhat_e + MLP(face features) in place of the first global trace solve,
          and V from the local recovery dV = -y - X P (vhat_m - vhat_e).
The local and mlp starts are hdg_newton_step's warm start (hdg_warmstart), which also falls
back to the plain solve from (V_e, vhat_e) if the solve from the warm start fails.
The network learns the correction of the extrapolated trace update from the first steps
of the plain solve. The interior residual carries the 1/dt time term and dominates the
Newton residual, so a predicted trace helps only together with the interior it implies;
"local" isolates what the element-local correction alone gives. The Newton solve with the
same tolerance decides the converged state in every case.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import torch

from . import hdg


@dataclass
class StepRecord:
    newton_updates: int
    res_history: list
    trace_iters: int
    wall_ms: float
    warm: str


@dataclass
class Network:
    nin: int
    nh: int
    nout: int
    params: torch.Tensor
    fmean: torch.Tensor
    fstd: torch.Tensor
    tmean: torch.Tensor
    tstd: torch.Tensor
    losses: list = field(default_factory=list)


class Stepper:
    def __init__(self, W, precision=hdg.HDG_PREC_MIXED, tol=1e-10, max_newton=8):
        self.W = W
        self.ctx = W.ctx.handle
        self.prec, self.tol, self.max_newton = precision, tol, max_newton
        self.dt = W.dt
        self.V = W.V.clone()
        self.Vh = W.Vhat.clone()
        self.Vp = None
        self.dvh1 = torch.zeros_like(self.Vh)
        self.dvh2 = torch.zeros_like(self.Vh)
        self.V0 = torch.empty_like(self.V)
        self.Vh0 = torch.empty_like(self.Vh)
        self.n = 0
        i = W.info
        self.F, self.per = i["n_faces"], i["Nf"] * i["m"]

    def state(self):
        return dict(V=self.V.clone(), Vh=self.Vh.clone(), Vp=None if self.Vp is None else self.Vp.clone(),
                    dvh1=self.dvh1.clone(), dvh2=self.dvh2.clone(), n=self.n)

    def restore(self, s):
        self.V, self.Vh = s["V"].clone(), s["Vh"].clone()
        self.Vp = None if s["Vp"] is None else s["Vp"].clone()
        self.dvh1, self.dvh2, self.n = s["dvh1"].clone(), s["dvh2"].clone(), s["n"]

    def features(self, net: Network | None, out: torch.Tensor):
        """Face features of the current state (raw when net is None)."""
        nin = 4 * self.per
        if net is None:
            zeros = torch.zeros(nin, dtype=torch.float32, device=self.V.device)
            ones = torch.ones(nin, dtype=torch.float32, device=self.V.device)
            hdg.hdg_mlp_features(self.ctx, self.V, self.Vh, self.dvh1, self.dvh2, zeros, ones, out)
        else:
            hdg.hdg_mlp_features(self.ctx, self.V, self.Vh, self.dvh1, self.dvh2, net.fmean, net.fstd, out)

    def step(self, warm="plain", net: Network | None = None) -> StepRecord:
        nV, nT = self.V.numel(), self.Vh.numel()
        # initial guess: V_e = 2 V^n - V^{n-1} (V^n on the first step), vhat_e = vhat^n + dvhat^n
        if self.Vp is None:
            order = 1
            self.V0.copy_(self.V)
        else:
            order = 2
            hdg.hdg_axpby(nV, 2.0, self.V, -1.0, self.Vp, self.V0)
        hdg.hdg_axpby(nT, 1.0, self.Vh, 1.0, self.dvh1, self.Vh0)
        ws, used = None, "plain"
        if warm in ("local", "mlp") and self.n >= 2:
            use_net = warm == "mlp" and net is not None
            ws = hdg.make_warmstart(self.Vh, self.dvh1, self.dvh2, net if use_net else None)
            used = "mlp" if use_net else "local"
        V_try, Vh_try = self.V0.clone(), self.Vh0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, rn, rh, tr = hdg.hdg_newton_step(self.ctx, V_try, Vh_try, self.V, self.Vp, self.dt, order, self.prec,
                                             self.tol, self.max_newton, warmstart=ws, history=True)
        torch.cuda.synchronize()
        wall = 1e3 * (time.perf_counter() - t0)
        # advance the histories: dvh2 <- dvh1, dvh1 <- vhat^{n+1} - vhat^n
        self.dvh2.copy_(self.dvh1)
        hdg.hdg_axpby(nT, 1.0, Vh_try, -1.0, self.Vh, self.dvh1)
        self.Vp = self.V
        self.V = V_try
        self.Vh = Vh_try
        self.n += 1
        return StepRecord(it, rh, tr, wall, used)


def collect_and_train(st: Stepper, n_steps: int, skip: int = 2, epochs: int = 30, lr: float = 1e-3,
                      sizes=(None, 64, None), seed: int = 7):
    """Run n_steps plain steps, storing face features and targets, then train the MLP.
    Returns (records, Network)."""
    dev = st.V.device
    per = st.per
    nin, nout = 4 * per, per
    nh = sizes[1] if sizes[1] else (64 if nin == 64 else 32)
    F = st.F
    keep = max(0, n_steps - skip)
    X = torch.empty((keep, F, nin), dtype=torch.float32, device=dev)
    T = torch.empty((keep, F, nout), dtype=torch.float32, device=dev)
    records = []
    for k in range(n_steps):
        if k >= skip:
            st.features(None, X[k - skip])
            vh_old = st.Vh.clone()
            dvh_old = st.dvh1.clone()
        records.append(st.step("plain"))
        if k >= skip:
            hdg.hdg_mlp_target(st.Vh.numel(), st.Vh, vh_old, dvh_old, T[k - skip])
    B = keep * F
    fmean = torch.empty(nin, dtype=torch.float32, device=dev)
    fstd = torch.empty_like(fmean)
    tmean = torch.empty(nout, dtype=torch.float32, device=dev)
    tstd = torch.empty_like(tmean)
    hdg.hdg_mlp_stats(X, B, nin, fmean, fstd)
    hdg.hdg_mlp_stats(T, B, nout, tmean, tstd)
    hdg.hdg_mlp_standardize(X, B, nin, fmean, fstd)
    hdg.hdg_mlp_standardize(T, B, nout, tmean, tstd)
    P = hdg.hdg_mlp_param_count(nin, nh, nout)
    params = torch.empty(((14 * P + 3) // 4,), dtype=torch.float32, device=dev)
    hdg.hdg_mlp_init(params, nin, nh, nout, seed)
    grad = torch.empty(P, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    net = Network(nin, nh, nout, params, fmean, fstd, tmean, tstd)
    step = 0
    for ep in range(epochs):
        tot = 0.0
        for k in range(keep):
            step += 1
            hdg.hdg_mlp_train_step(params, grad, nin, nh, nout, X[k], T[k], F, lr, step, loss)
            tot += float(loss.item()) if k == keep - 1 else 0.0
        net.losses.append(tot)
    return records, net


def experiment(workload="ns2d_p3_vortices", n_train=200, n_apply=200, skip=2, epochs=40, lr=2e-3,
               precision=hdg.HDG_PREC_MIXED, tol=1e-10, dt=None):
    """The learned warm-start experiment: n_train plain steps (training data), training,
    then n_apply steps from the same state with the plain start and with the network.
    Returns a summary dict (Newton updates, initial residuals, wall time per step)."""
    import math

    from .workload import DeviceWorkload
    W = DeviceWorkload(workload, outputs=False)
    if dt is not None:  # a time step other than the workload's (the BDF steps use Stepper.dt)
        W.dt = dt
    st = Stepper(W, precision=precision, tol=tol)
    t0 = time.perf_counter()
    recs, net = collect_and_train(st, n_train, skip=skip, epochs=epochs, lr=lr)
    t_collect_train = time.perf_counter() - t0
    snap = st.state()
    plain = [st.step("plain") for _ in range(n_apply)]
    V_plain = st.V.clone()
    st.restore(snap)
    local = [st.step("local") for _ in range(n_apply)]
    st.restore(snap)
    learned = [st.step("mlp", net) for _ in range(n_apply)]

    def summary(rs):
        return {"steps": len(rs), "newton_updates_per_step": sum(r.newton_updates for r in rs) / len(rs),
                "trace_iters_per_step": sum(r.trace_iters for r in rs) / len(rs),
                "wall_ms_per_step": sum(r.wall_ms for r in rs) / len(rs),
                "initial_residual_geomean": math.exp(sum(math.log(max(r.res_history[0], 1e-300)) for r in rs)
                                                     / len(rs))}

    return {"workload": workload, "elements": W.n_elem, "faces": W.info["n_faces"], "precision": precision,
            "tol": tol, "train_steps": n_train, "skip": skip, "epochs": epochs,
            "network": [net.nin, net.nh, net.nh, net.nout], "train_loss_first_last": [net.losses[0], net.losses[-1]],
            "collect_and_train_s": t_collect_train, "plain": summary(plain), "local": summary(local),
            "learned": summary(learned),
            "final_state_rel_diff": float((st.V - V_plain).norm() / V_plain.norm())}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ns2d_p3_vortices")
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--apply", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--dt", type=float, default=None, help="time step (default: the workload's)")
    a = ap.parse_args()
    print(json.dumps(experiment(a.workload, a.train, a.apply, epochs=a.epochs, dt=a.dt)))
