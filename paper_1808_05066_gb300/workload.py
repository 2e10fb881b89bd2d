"""Device-resident workloads for the C-ABI path.

Builds the named synthetic workload of workloads.py on the GPU: the C-ABI mesh, the
context, the initial entropy variables (closed-form primitive fields at the element and
face nodes, converted by hdg_prim_to_entropy), the trace perturbation, the BDF history
and the output buffers of hdg_assemble_condense. No method arithmetic happens here.
"""
from __future__ import annotations

import math
import sys

import numpy as np
import torch

import workloads as wl

from . import hdg


def _prim(name, spec, x):
    rho, vel, p = wl.primitive_state(name, x)
    return np.concatenate([rho[..., None], vel, p[..., None]], axis=-1)


class DeviceWorkload:
    """State and buffers of one workload on one GPU.

    The time term is BDF2 with both history levels equal to the initial state
    (u^{n-1} = u^n), dt from the workload: mass_coef = 3/(2 dt), history
    c0 = 2/dt, c1 = -1/(2 dt)."""

    def __init__(self, name: str, device: int = 0, n_override: int | None = None, outputs: bool = True):
        spec = dict(wl.WORKLOADS[name])
        if n_override:
            spec["n"] = n_override
        self.name, self.spec = name, spec
        self.dev = torch.device("cuda", device)
        d = spec["dim"]
        E = (2 if d == 2 else 6) * spec["n"] ** d
        self.p_elem = wl.draw_degrees(name, E)
        self.mesh = hdg.Mesh(d, spec["n"], spec["lo"], spec["hi"], spec["p"], p_per_elem=self.p_elem)
        self.ctx = hdg.Context(self.mesh, 1.4, spec["mach"], spec["reynolds"], spec["prandtl"], device)
        self.info = self.mesh.info
        xnode, xfnode, _ = self.mesh.coords()
        self.V = self._entropy(_prim(name, spec, xnode))
        Vh = self._entropy(_prim(name, spec, xfnode))
        eps = spec.get("trace_noise", 0.0)
        if eps:
            Vh = torch.from_numpy(wl.perturb(Vh.cpu().numpy(), eps, spec["seed"])).to(self.dev)
        self.Vhat = Vh.contiguous()
        dt = spec["dt"]
        self.dt = dt
        if spec.get("bdf", 2) == 2:
            self.mass_coef = 1.5 / dt
            c0, c1, V1 = 2.0 / dt, -0.5 / dt, self.V
        else:
            self.mass_coef = 1.0 / dt
            c0, c1, V1 = 1.0 / dt, 0.0, None
        self.hist = torch.empty_like(self.V)
        hdg.hdg_history(self.ctx.handle, self.V, V1, c0, c1, self.hist)
        if outputs:
            self.alloc_outputs()
        torch.cuda.synchronize(self.dev)

    def close(self):
        """Release the device buffers and the context (its internal workspaces)."""
        for k in ("S", "g", "recov", "R", "status", "V", "Vhat", "hist"):
            if hasattr(self, k):
                delattr(self, k)
        self.ctx.close()

    def _entropy(self, prim):
        t = torch.from_numpy(np.ascontiguousarray(prim)).to(self.dev)
        out = torch.empty_like(t)
        hdg.hdg_prim_to_entropy(self.ctx.handle, t, t.numel() // t.shape[-1], out)
        return out

    def alloc_outputs(self):
        i = self.info
        E, nv, nt = i["n_elem"], i["nv"], i["nt"]
        f64 = dict(dtype=torch.float64, device=self.dev)
        if i["mixed"]:   # packed per-element layout
            self.S = torch.empty(i["len_S"], **f64)
            self.g = torch.empty(i["len_g"], **f64)
            self.recov = torch.empty(i["len_recov"], **f64)
            self.R = torch.empty(i["len_R"], **f64)
            self.status = torch.zeros(E, dtype=torch.int32, device=self.dev)
            return
        self.S = torch.empty((E, nt, nt), **f64)
        self.g = torch.empty((E, nt), **f64)
        self.recov = torch.empty((E, nv * nt + nv), **f64)
        self.R = torch.empty((E, nv + nt), **f64)
        self.status = torch.zeros(E, dtype=torch.int32, device=self.dev)

    def assemble(self, precision=hdg.HDG_PREC_FP64, V=None, Vhat=None, stream=None):
        hdg.hdg_assemble_condense(self.ctx.handle, self.V if V is None else V, self.Vhat if Vhat is None else Vhat,
                                  self.hist, self.mass_coef, precision, self.S, self.g, self.recov, self.R,
                                  self.status, stream)

    def assemble_to_host(self, S_host, g_host, precision=hdg.HDG_PREC_FP64, V=None, Vhat=None, stream=None):
        """The same call with S and g delivered to (pinned) host memory, copied chunk by chunk
        while the next chunk computes."""
        hdg.hdg_assemble_condense_host(self.ctx.handle, self.V if V is None else V,
                                       self.Vhat if Vhat is None else Vhat, self.hist, self.mass_coef, precision,
                                       S_host, g_host, self.recov, self.R, self.status, stream)

    @property
    def n_elem(self):
        return self.info["n_elem"]


def bench_workload_name() -> str:
    return "ns3d_p3_tgv"


def flops_per_element(info: dict, viscous: bool, kernel: str) -> float:
    """Useful floating-point operations per element of the FP64 form, counted from the
    loop structure of the kernels (multiply + add = 2 flops):
      assemble: volume contraction per (i, l): NP x [NP x ng x NR + NT' x ng x (NR-1)]
                + the left factor NP x ng x NR x (D+1); face contraction per face and (i, l):
                NFN x NZ x NGF x NRF + NFN x NGF x NRF;
      condense: LU NV^3/3 + solves (NT + 1) NV^2 + Schur NT^2 NV + NT NV."""
    D, M = info["dim"], info["m"]
    NP, NFN, NF, NG, NGF = info["Np"], info["Nf"], info["nF"], info["NG"], info["NGF"]
    NV, NT = info["nv"], info["nt"]
    NZ = NP + NF * NFN
    NR = D + 1 if viscous else 1
    NRF = D + 2 if viscous else 2
    if kernel == "assemble":
        vol = M * M * (NP * (NP * NG * NR + NF * NFN * NG * (NR - 1)) + NP * NG * NR * (D + 1))
        face = NF * M * M * (NFN * NZ * NGF * NRF + NFN * NGF * NRF)
        return 2.0 * (vol + face)
    if kernel == "condense":
        return 2.0 * (NV ** 3 / 3.0 + (NT + 1) * NV ** 2 + NT * NT * NV + NT * NV)
    raise ValueError(kernel)


# FP64 pipe of a GB300: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz (a DFMA probe on the
# same GPU type measured 1.20 TFLOP/s)
FP64_PIPE_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def class_flops_per_element(pk: int, pt: int, nt_own: int) -> float:
    """FP64 flops of one element of the mixed-degree fused kernel (3D Navier-Stokes), counted from
    its loops like flops_per_element: element degree pk (volume rule pk + 1), trace degree pt on
    every face (face rule pt + 1), the face contractions over the element's face nodes (degree pk)
    and the trace nodes (degree pt), and the condensation with the element's own trace size
    nt_own; the projection onto the faces' own spaces is not counted."""
    D, M, NF = 3, 5, 4
    NP = (pk + 1) * (pk + 2) * (pk + 3) // 6
    NFK = (pk + 1) * (pk + 2) // 2
    NFN = (pt + 1) * (pt + 2) // 2
    NG, NGF = (pk + 1) ** 3, (pt + 1) ** 2
    NZ, NV = NP + NF * NFN, NP * M
    NR, NRF = D + 1, D + 2
    vol = M * M * (NP * (NP * NG * NR + NF * NFN * NG * (NR - 1)) + NP * NG * NR * (D + 1))
    face = NF * M * M * ((NFK + NFN) * NZ * NGF * NRF + (NFK + NFN) * NGF * NRF)
    cond = NV ** 3 / 3.0 + (nt_own + 1) * NV ** 2 + nt_own * nt_own * NV + nt_own * NV
    return 2.0 * (vol + face + cond)


SLICES = 6  # exact bf16 slices per operand in the mixed form's tensor-core products


def slice_flops_per_element(info: dict, viscous: bool, kernel: str) -> float:
    """Useful bf16 slice-product flops per element of one mixed-form tensor-core kernel:
    2 x rows x columns x contraction length of every nonzero operator block, times the
    S(S+1)/2 slice products. Tile padding and products a kernel shape adds are not counted, so
    this never exceeds what a kernel executes:
      mixed_assemble: rows (i, l, node) = m^2 NP, contraction NG per operator; the value
                      operator meets the NP interior columns, each of the NR - 1 gradient
                      operators all NZ;
      mixed_face:     per face rows m^2 NFN, contraction NGF; value operator NP columns, trace
                      operator the face's own NFN, each of the NRF - 2 gradient operators all NZ;
      mixed_condense: r0 = B - A' X0 and S = D - C' X: NV + NT rows, NT + 1 right-hand sides,
                      contraction NV."""
    D, M = info["dim"], info["m"]
    NP, NFN, NF, NG, NGF = info["Np"], info["Nf"], info["nF"], info["NG"], info["NGF"]
    NV, NT = info["nv"], info["nt"]
    NZ = NP + NF * NFN
    NR = D + 1 if viscous else 1
    NRF = D + 2 if viscous else 2
    prod = SLICES * (SLICES + 1) // 2
    if kernel == "mixed_assemble":
        return 2.0 * prod * (M * M * NP) * NG * (NP + (NR - 1) * NZ)
    if kernel == "mixed_face":
        return 2.0 * prod * NF * (M * M * NFN) * NGF * (NP + NFN + (NRF - 2) * NZ)
    if kernel == "mixed_condense":
        return 2.0 * prod * (NV + NT) * (NT + 1) * NV
    raise ValueError(kernel)


def algorithmic_bytes_per_element(info: dict, kernel: str) -> int:
    """HBM bytes one element needs moved by a mixed-form kernel (8-byte values):
      mixed_assemble: read the volume point tensors, write A' and B';
      mixed_face:     read the face point tensors, write C' and D', add into A' and B';
      mixed_condense: the method's outputs only: write S, X, y and g (the blocks the assembly
                      parks in HBM for it are this implementation's, not the method's)."""
    D, M = info["dim"], info["m"]
    NP, NFN, NF, NG, NGF = info["Np"], info["Nf"], info["nF"], info["NG"], info["NGF"]
    NV, NT = info["nv"], info["nt"]
    pt_vol = M + D * M + M * M + D * M * M + D * M * M * D
    pt_face = M + 2 * M * M + M * M * D
    if kernel == "mixed_assemble":
        return 8 * (NG * pt_vol + NV * (NV + NT))
    if kernel == "mixed_face":
        return 8 * (NF * NGF * pt_face + NT * (NV + NT) + 2 * NV * (NV + NT))
    if kernel == "mixed_condense":
        return 8 * (NT * NT + NV * NT + NV + NT)
    raise ValueError(kernel)


def method_flops_per_element(info: dict, viscous: bool, kernel: str) -> float:
    """The method's own flops per element of a mixed-form kernel, the same count as the FP64
    form's kernels (flops_per_element): the assembly contractions for mixed_assemble +
    mixed_face (split by the share of their slice products), the LU, solves and Schur product
    for mixed_condense."""
    if kernel == "mixed_condense":
        return flops_per_element(info, viscous, "condense")
    asm = flops_per_element(info, viscous, "assemble")
    v = slice_flops_per_element(info, viscous, "mixed_assemble")
    f = slice_flops_per_element(info, viscous, "mixed_face")
    return asm * (v if kernel == "mixed_assemble" else f) / (v + f)



def main(argv=None):
    """Run a named workload's assemble + condense a few times on cuda:0 and print the time of
    each call (CUDA events): `python -m paper_1808_05066_gb300.workload ns3d_mixed_tgv --n 4`."""
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(wl.WORKLOADS))
    ap.add_argument("--n", type=int, default=None, help="cube / square resolution (default: the workload's)")
    ap.add_argument("--calls", type=int, default=3)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    args = ap.parse_args(argv)
    W = DeviceWorkload(args.name, n_override=args.n)
    prec = hdg.HDG_PREC_MIXED if args.precision == "mixed" else hdg.HDG_PREC_FP64
    E = W.info["n_elem"]
    for k in range(args.calls):
        W.status.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        W.assemble(prec)
        b.record()
        torch.cuda.synchronize(W.dev)
        ms = a.elapsed_time(b)
        print(f"{args.name} E={E} call {k}: {ms:.2f} ms, {E / ms * 1e3:.0f} elem/s, "
              f"flagged elements {int((W.status != 0).sum())}", flush=True)
    W.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
