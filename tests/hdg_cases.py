"""Shared set-up for GPU parity tests: the same seeded workload evaluated once by the
oracle (its own mesh, its own v(u)) and once by the CUDA path (C-ABI mesh, state
conversion by hdg_prim_to_entropy). Only workloads.py is common to both."""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

import workloads as wl


@dataclass
class Case:
    name: str
    dim: int
    n: int
    p: int
    L: float
    mach: float
    reynolds: float
    prandtl: float
    field: str          # "vortex", "vortices16", "tgv"
    noise: float = 1e-3
    seed: int = 11
    mass_coef: float = 20.0
    mu_exponent: float = 0.0   # power-law viscosity exponent (0: constant)
    visc_flux: int = 2         # viscous numerical flux option (Eq. numericalFluxNS_1 / _2)
    scheme: str = "hdg"        # trace space (Sec. 3.4): "hdg", "edg" or "iedg"
    stabilization: str = "slf"  # "slf" (Eq. sLxF) or "s" (Eq. symStab)
    vinf: tuple = (1.0, 0.0)    # free stream of the vortex fields
    psi: float = 5.0            # strength of the single vortex
    bc: tuple = None            # per axis (lo, hi) boundary types; None: periodic

    @property
    def lo(self):
        return 0.0

    def prim(self, x):
        if self.field == "tgv":
            return wl.tgv_field(x * (2 * math.pi / self.L), self.mach)
        if self.field == "vortex":
            return wl.vortex_field(x, [wl.Vortex(self.L / 2, self.L / 2, self.psi)], self.mach, vinf=self.vinf,
                                   period=self.L)
        nv = int(self.field.replace("vortices", ""))
        return wl.vortex_field(x, wl.draw_vortices(nv, self.L, self.seed), self.mach, vinf=self.vinf,
                               period=self.L)


def prim_array(case: Case, x):
    rho, vel, p = case.prim(x)
    return np.concatenate([rho[..., None], vel, p[..., None]], axis=-1)


# ------------------------------------------------------------------ oracle side
def oracle_setup(case: Case):
    from oracle import physics as ph
    from oracle.hdg import Problem, consistent_Q, face_states, interpolate_state
    from oracle.mesh import Mesh
    mesh = Mesh(case.dim, case.n, 0.0, case.L, case.p, bc=case.bc)
    phys = ph.Physics(mach=case.mach, reynolds=case.reynolds, prandtl=case.prandtl, mu_exponent=case.mu_exponent,
                       stabilization=case.stabilization)
    prob = Problem(mesh, phys, viscous_flux_option=case.visc_flux, scheme=case.scheme)
    V, Vh = interpolate_state(prob, case.prim)
    if case.bc is not None:
        prob.boundary_state = face_states(prob, V)     # the unperturbed state at the faces' nodes: v_b
    if case.noise:
        Vh = wl.perturb(Vh, case.noise, case.seed)
    Q = consistent_Q(prob, V, Vh)
    return prob, Q, V, Vh


def oracle_hist(prob, V, case: Case):
    """BDF1 history with V^n = V scaled slightly so the time term is non-trivial."""
    from oracle.hdg import bdf_coefficients
    Vn = V * (1 + 1e-3)
    return np.stack([prob.history_weak(e, [Vn[e]], [case.mass_coef]) for e in range(prob.mesh.E)])


# ------------------------------------------------------------------ GPU side
class GpuCase:
    def __init__(self, case: Case, device=0):
        import torch
        from paper_1808_05066_gb300 import hdg
        self.hdg, self.torch, self.case = hdg, torch, case
        self.mesh = hdg.Mesh(case.dim, case.n, 0.0, case.L, case.p,
                             scheme={"hdg": hdg.HDG_SCHEME_HDG, "edg": hdg.HDG_SCHEME_EDG,
                                     "iedg": hdg.HDG_SCHEME_IEDG}[case.scheme], bc=case.bc)
        self.ctx = hdg.Context(self.mesh, 1.4, case.mach, case.reynolds, case.prandtl, device,
                               mu_exponent=case.mu_exponent, visc_flux=case.visc_flux,
                               stabilization=1 if case.stabilization == "s" else 0)
        self.info = self.mesh.info
        xnode, xfnode, _ = self.mesh.coords()
        dev = torch.device("cuda", device)
        self.dev = dev
        i = self.info
        self.V = self.to_entropy(prim_array(case, xnode))
        Vh = self.to_entropy(prim_array(case, xfnode))
        if case.bc is not None:
            self.Vb = Vh.clone()
            hdg.hdg_ctx_set_boundary_state(self.ctx.handle, self.Vb)
        if case.noise:
            Vh = torch.from_numpy(wl.perturb(Vh.cpu().numpy(), case.noise, case.seed)).to(dev)
        self.Vhat = Vh.contiguous()
        E, nv, nt = i["n_elem"], i["nv"], i["nt"]
        self.S = torch.empty((E, nt, nt), dtype=torch.float64, device=dev)
        self.g = torch.empty((E, nt), dtype=torch.float64, device=dev)
        self.recov = torch.empty((E, nv * nt + nv), dtype=torch.float64, device=dev)
        self.R = torch.empty((E, nv + nt), dtype=torch.float64, device=dev)
        self.status = torch.zeros(E, dtype=torch.int32, device=dev)

    def to_entropy(self, prim):
        t = self.torch.from_numpy(np.ascontiguousarray(prim)).to(self.dev)
        out = self.torch.empty_like(t)
        self.hdg.hdg_prim_to_entropy(self.ctx.handle, t, t.numel() // t.shape[-1], out)
        return out

    def history(self):
        V0 = (self.V * (1 + 1e-3)).contiguous()
        hist = self.torch.empty_like(self.V)
        self.hdg.hdg_history(self.ctx.handle, V0, None, self.case.mass_coef, 0.0, hist)
        return hist

    def assemble(self, hist, precision=0):
        self.status.zero_()
        self.hdg.hdg_assemble_condense(self.ctx.handle, self.V, self.Vhat, hist, self.case.mass_coef, precision,
                                       self.S, self.g, self.recov, self.R, self.status)
        self.torch.cuda.synchronize()


CASES = {
    # the 2D Euler p=2 workload at full size (8x8 periodic [0,10]^2, one vortex)
    "euler2d_p2": Case("euler2d_p2", 2, 8, 2, 10.0, 0.5, 0.0, 0.71, "vortex"),
    "ns2d_p3": Case("ns2d_p3", 2, 3, 3, 3.75, 0.5, 5000.0, 0.71, "vortices16"),
    "ns2d_p4": Case("ns2d_p4", 2, 3, 4, 3.75, 0.3, 1000.0, 0.72, "vortices16"),
    "ns3d_p1": Case("ns3d_p1", 3, 3, 1, 2 * math.pi, 0.1, 1600.0, 0.71, "tgv"),
    "ns3d_p2": Case("ns3d_p2", 3, 2, 2, 2 * math.pi, 0.1, 1600.0, 0.71, "tgv"),
    "ns3d_p3": Case("ns3d_p3", 3, 2, 3, 2 * math.pi, 0.1, 1600.0, 0.71, "tgv"),
}


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
