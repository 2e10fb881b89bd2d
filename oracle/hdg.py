"""Oracle for the entropy-variable hybridized DG local problem and Newton step.

Follows Sec. 3.2 (Euler, Eqs. hDG1-hDG2) and Sec. 3.3 (Navier-Stokes, Eqs.
hDG_NS0-hDG_NS2), with
  * inviscid flux Eq. numericalFlux, sigma = sigma_SLF of Eq. sLxF at v* = vhat
    (the choice of Sec. 5), or sigma_S of Eq. symStab at the same v* (Physics.stabilization),
  * viscous flux Eq. numericalFluxNS_2, G(vhat, q) . n (the choice of Sec. 5),
  * time term (d u(v_h)/dt, w) discretised by BDF: mass_coef (u(v_h), w) - hist,
    hist = sum_j c_j (u(v_h^{n-j}), w) (BDF1 / BDF2; BDF0 = steady),
  * the boundary term <b_h(vhat, v), mu> of Eqs. hDG2 / hDG_NS2 on faces of the boundary
    (the paper leaves b_h open, Sec. 3.2); two are defined:
      BC_STATE  b_h = vhat - v_b: the trace takes a given boundary state v_b (the paper's
                prescribed exact solutions, Secs. 5.1-5.2), v_b given by its values at the
                face nodes (Problem.boundary_state [F, Nf, m], for every trace space); with the
                continuous EDG trace, whose boundary nodes are shared with interior faces, the
                state is imposed strongly instead: the assembled equation of a node on a
                BC_STATE face is vhat - v_b = 0 (assemble_trace, residual_norm);
      BC_SLIP   b_h = fhat(vhat, v; n) + fhat(vhat, R v; -n) (Euler only): the trace residual
                of an interior face whose other side is the element's mirror image, R
                reflecting the momentum components, w -> w - 2 (w . n) n; the converged state
                is the restriction of the mirror-symmetric state on the doubled domain, and
                no mass or energy crosses the wall.

The local Newton system is the plain definition: the dense Jacobian of the local
residuals R_l = (R_q, R_v) and of the element's trace residual R_t, taken by
complex step (exact to rounding, no subtractive cancellation), then
  S = D - C A^{-1} B,  g = R_t - C A^{-1} R_l   (static condensation, Sec. 3.2-3.3)
with A^{-1} applied by LU with partial pivoting (numpy.linalg.solve). The assembled
trace system sum_e P_e^T S_e P_e dvhat = -sum_e P_e^T g_e is solved densely (or by a
sparse direct solve), and the interior update is dx_e = -A^{-1}(R_l + B P_e dvhat).

Interior unknown order: [q (node, component, direction); v (node, component)];
trace order: [local face, face node, component].

Mixed degrees (Mesh(p_elem=...); not in the paper, which uses one degree): element e uses its
own P_{p_e} with the volume rule exact to degree 2 p_e + 1; its faces carry the trace of degree
q_F = max(p_L, p_R) and are integrated with the rule exact to degree 2 PT_e + 1, PT_e = the
largest degree of its faces. V, Q (and the BDF history) are then lists of per-element arrays,
Vhat is [face nodes, m] with the nodes of face F at fnode_off[F] + canonical index, and the
element's trace order is [face, its own face nodes, component].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import physics as ph
from .mesh import BC_PERIODIC, BC_SLIP, BC_STATE, Mesh
from .refel import refel

CSTEP = 1e-30


@dataclass
class ElementTables:
    W: np.ndarray          # [ng] volume weights * |det J|
    phi: np.ndarray        # [ng, Np]
    gphi: np.ndarray       # [ng, Np, d] physical gradients
    Wf: list               # per face [ngf]
    phif: list             # per face [ngf, Np]
    psi: list              # per face [ngf, Nf] trace basis = element basis restricted to the face
    nrm: list              # per face [d] outward unit normal


class Problem:
    """A mesh + physics + the element tables the residual needs."""

    def __init__(self, mesh: Mesh, phys: ph.Physics, viscous_flux_option: int = 2, scheme: str = "hdg"):
        """viscous_flux_option: 2 = ghat = G(vhat, q) . n (Eq. numericalFluxNS_2, used in all of
        Sec. 5), 1 = ghat = G(v, q) . n (Eq. numericalFluxNS_1).
        scheme (Sec. 3.4): "hdg" (E^E_h empty: one trace per face, Vhat [F, Nf, m]), "edg"
        (E^E_h = all faces: a continuous trace, one unknown per skeleton node, Vhat [N, m]) or
        "iedg" (E^E_h = the interior faces: continuous there, one trace per boundary face; on a
        periodic mesh every face is interior, so IEDG is EDG). The element residual is the same for
        all three; only the numbering of the trace unknowns differs."""
        if viscous_flux_option not in (1, 2):
            raise ValueError(viscous_flux_option)
        if scheme not in ("hdg", "edg", "iedg"):
            raise ValueError(scheme)
        self.mesh, self.phys = mesh, phys
        self.viscous_flux_option = viscous_flux_option
        self.scheme = "edg" if scheme == "iedg" else scheme
        bounded = bool(np.any(mesh.face_bc != BC_PERIODIC))
        self.iedg = scheme == "iedg" and bounded
        # EDG on a bounded mesh: a boundary node of the continuous trace is shared with interior
        # faces, so the given state is imposed strongly there (the node's equation is vhat = v_b,
        # Problem.dirichlet_rows); the weak term <vhat - v_b, mu> would be summed with fluxes
        self.edg_dirichlet = scheme == "edg" and bounded
        if self.edg_dirichlet and np.any(mesh.face_bc == BC_SLIP):
            raise ValueError("EDG with boundaries: the given state only")
        if np.any(mesh.face_bc == BC_SLIP) and phys.viscous:
            raise ValueError("the slip boundary is defined for the Euler equations only")
        self.boundary_state = None      # [F, Nf, m] v_b at the canonical face nodes (BC_STATE faces)
        self.mixed = mesh.p_elem is not None
        if self.mixed and self.scheme != "hdg":
            raise ValueError("mixed degrees are built for the HDG trace space")
        if self.scheme == "edg":
            self.n_edg, self.edg_index = mesh.edg_numbering(interior_only=self.iedg)
        ref = mesh.ref
        self.d, self.m = mesh.dim, mesh.dim + 2
        self.Np, self.Nf, self.nF = ref.Np, ref.Nf, ref.nF
        self.viscous = phys.viscous
        if self.mixed:
            self.Nf = mesh.Nf_max
        self.n_i = self.Np * self.m * (1 + (self.d if self.viscous else 0))
        self.n_t = self.nF * self.Nf * self.m
        self._phi = ref.phi(ref.qp)
        self._dphi = ref.dphi(ref.qp)
        self._phif = [ref.phi(x) for x in ref.fqp_ref]
        self._cache = {}

    def dirichlet_nodes(self):
        """EDG on a bounded mesh: (trace nodes on BC_STATE faces [K], their v_b [K, m]) from
        Problem.boundary_state; (None, None) otherwise."""
        if not self.edg_dirichlet:
            return None, None
        vb = {}
        for F in np.flatnonzero(self.mesh.face_bc == BC_STATE):
            e, f = self.mesh.face_elems[F][0]
            for c in range(self.Nf):
                vb.setdefault(int(self.edg_index[e, f, c]), self.boundary_state[F][self.mesh.fnode_map[e, f, c]])
        nodes = np.array(sorted(vb), dtype=np.int64)
        return nodes, np.array([vb[k] for k in nodes])

    def dirichlet_rows(self, Vhat):
        """(rows of the assembled trace system whose equation is vhat - v_b = 0, vhat - v_b there),
        or (None, None)."""
        nodes, vb = self.dirichlet_nodes()
        if nodes is None:
            return None, None
        rows = (nodes[:, None] * self.m + np.arange(self.m)).ravel()
        return rows, (Vhat[nodes] - vb).ravel()

    # -- element sizes (mixed degrees: per element) ----------------------------------------
    def np_e(self, e):
        """Nodes of element e (its own degree)."""
        if self.mixed:
            return refel(self.d, int(self.mesh.p_elem[e])).Np
        return self.Np

    def ni_e(self, e):
        """Interior unknowns of element e: [q;] v."""
        return self.np_e(e) * self.m * (1 + (self.d if self.viscous else 0))

    def trace_mask(self, e):
        """Which entries of the padded local trace [nF, Nf_max, m] are unknowns (mixed degrees:
        face f of element e has the face nodes of its degree q_{e,f}); all of them otherwise."""
        if not self.mixed:
            return np.ones(self.n_t, dtype=bool)
        cnt = self.mesh.face_nnodes[self.mesh.face_of[e]]                  # [nF]
        ok = np.arange(self.Nf)[None, :] < cnt[:, None]
        return np.repeat(ok[:, :, None], self.m, axis=2).ravel()

    def tables(self, e: int) -> ElementTables:
        t = self._cache.get(e)
        if t is not None:
            return t
        mesh, ref = self.mesh, self.mesh.ref
        if self.mixed:
            t = self._mixed_tables(e)
            if len(self._cache) < 64:
                self._cache[e] = t
            return t
        W = ref.qw * abs(mesh.detJ[e])
        gphi = np.einsum("gar,rj->gaj", self._dphi, mesh.Jinv[e])
        Wf, phif, psi, nrm = [], [], [], []
        for f in range(ref.nF):
            Wf.append(ref.fqw * mesh.face_jac[e, f])
            phif.append(self._phif[f])
            psi.append(self._phif[f][:, ref.face_nodes[f]])
            nrm.append(mesh.normal[e, f])
        t = ElementTables(W, self._phi, gphi, Wf, phif, psi, nrm)
        if len(self._cache) < 64:
            self._cache[e] = t
        return t

    def _mixed_tables(self, e):
        """Tables of element e of a mixed-degree mesh: the volume rule and basis of its degree
        p_e (rule exact to degree 2 p_e + 1), on every face the rule exact to degree 2 PT_e + 1
        (PT_e its trace degree) and the nodal trace basis of that face's degree q_{e,f}, padded
        with zero columns to Nf_max."""
        mesh = self.mesh
        pK, PT = int(mesh.p_elem[e]), int(mesh.elem_trace_deg[e])
        rK, rT = refel(self.d, pK), refel(self.d, PT)
        W = rK.qw * abs(mesh.detJ[e])
        phi = rK.phi(rK.qp)
        gphi = np.einsum("gar,rj->gaj", rK.dphi(rK.qp), mesh.Jinv[e])
        Wf, phif, psi, nrm = [], [], [], []
        for f in range(self.nF):
            x = rT.fqp_ref[f]
            rq = refel(self.d, int(mesh.elem_face_deg[e, f]))
            ps = np.zeros((len(x), self.Nf))
            ps[:, :rq.Nf] = rq.phi(x)[:, rq.face_nodes[f]]
            Wf.append(rT.fqw * mesh.face_jac[e, f])
            phif.append(rK.phi(x))
            psi.append(ps)
            nrm.append(mesh.normal[e, f])
        return ElementTables(W, phi, gphi, Wf, phif, psi, nrm)

    # -- gather / scatter between global trace and element-local trace ------------------
    def gather_trace(self, Vhat, e):
        mesh = self.mesh
        if self.mixed:                                                        # padded [nF, Nf_max, m]
            tn = self.trace_node(e)
            return np.where((tn >= 0)[:, :, None], Vhat[np.maximum(tn, 0)], 0.0)
        if self.scheme == "edg":
            return Vhat[self.edg_index[e]]                                    # [nF, Nf, m]
        return Vhat[mesh.face_of[e][:, None], mesh.fnode_map[e]]          # [nF, Nf, m]

    def trace_node(self, e):
        """Global trace node [nF, Nf] of each local face node of element e."""
        mesh = self.mesh
        if self.mixed:                                                        # -1: padding
            fm = mesh.fnode_map_mixed[e]
            return np.where(fm >= 0, mesh.fnode_off[mesh.face_of[e]][:, None] + fm, -1)
        if self.scheme == "edg":
            return self.edg_index[e]
        return mesh.face_of[e][:, None] * self.Nf + mesh.fnode_map[e]

    def trace_index(self, e):
        """Global flat indices of the element's local trace unknowns (f, c, i); with EDG a
        node shared by several local faces appears several times (P_e has repeated columns)."""
        base = self.trace_node(e) * self.m
        idx = (base[:, :, None] + np.arange(self.m)).ravel()
        return idx[self.trace_mask(e)] if self.mixed else idx

    @property
    def n_trace(self):
        if self.mixed:
            return int(self.mesh.fnode_off[-1]) * self.m
        if self.scheme == "edg":
            return self.n_edg * self.m
        return self.mesh.nFaces * self.Nf * self.m

    @property
    def trace_shape(self):
        """Shape of the global Vhat array."""
        if self.mixed:
            return (int(self.mesh.fnode_off[-1]), self.m)
        if self.scheme == "edg":
            return (self.n_edg, self.m)
        return (self.mesh.nFaces, self.Nf, self.m)

    # -- viscous fluxes (Sec. 3.3) ---------------------------------------------------------
    def volume_viscous_flux(self, v, q):
        """G(v_h, q_h) [..., m, d] at volume points, the viscous flux of Eq. hDG_NS1."""
        return ph.viscous_flux(v, q, self.phys)

    def face_viscous_flux(self, vhat, v, q, n):
        """Viscous numerical flux: ghat_h = G(vhat_h, q_h) . n (Eq. numericalFluxNS_2, the option
        used in all of Sec. 5; the interior trace v is not used) or G(v_h, q_h) . n
        (Eq. numericalFluxNS_1; vhat is not used)."""
        state = vhat if self.viscous_flux_option == 2 else v
        return np.einsum("...mj,j->...m", ph.viscous_flux(state, q, self.phys), n)

    # -- residuals ----------------------------------------------------------------------
    def element_residual(self, e, Q, V, Vh, mass_coef=0.0, hist_w=None):
        """Local residuals for a batch [B, ...] of states of element e.

        Q [B, Np, m, d] (None for Euler), V [B, Np, m], Vh [B, nF, Nf, m].
        Returns (Rq [B, Np, m, d] or None, Rv [B, Np, m], Rt [B, nF, Nf, m])."""
        T = self.tables(e)
        g = self.phys.gamma
        v = np.einsum("ga,bam->bgm", T.phi, V)
        u = ph.u_of_v(v, g)
        flux = ph.inviscid_flux_v(v, g)
        Rq = None
        if self.viscous:
            q = np.einsum("ga,bamk->bgmk", T.phi, Q)
            flux = flux + self.volume_viscous_flux(v, q)
            # Eq. hDG_NS0: (q, r) + (v, div r) - <vhat, r.n>
            Rq = (np.einsum("g,ga,bgmk->bamk", T.W, T.phi, q)
                  + np.einsum("g,gak,bgm->bamk", T.W, T.gphi, v))
        # Eq. hDG1 / hDG_NS1: (du/dt, w) - (F + G, grad w) + <fhat + ghat, w>
        Rv = -np.einsum("g,gaj,bgmj->bam", T.W, T.gphi, flux)
        if mass_coef != 0.0:
            Rv = Rv + mass_coef * np.einsum("g,ga,bgm->bam", T.W, T.phi, u)
        if hist_w is not None:
            Rv = Rv - hist_w
        Rt = np.zeros(Vh.shape, dtype=np.result_type(V, Vh))
        for f in range(self.nF):
            vf = np.einsum("ga,bam->bgm", T.phif[f], V)
            vhf = np.einsum("gc,bcm->bgm", T.psi[f], Vh[:, f])
            n = T.nrm[f]
            fh = ph.numerical_flux_inviscid(vhf, vf, n, g, self.phys.stabilization)
            if self.viscous:
                qf = np.einsum("ga,bamk->bgmk", T.phif[f], Q)
                fh = fh + self.face_viscous_flux(vhf, vf, qf, n)
                Rq = Rq - np.einsum("g,ga,bgm,k->bamk", T.Wf[f], T.phif[f], vhf, n)
            Rv = Rv + np.einsum("g,ga,bgm->bam", T.Wf[f], T.phif[f], fh)
            F = self.mesh.face_of[e, f]
            kind = self.mesh.face_bc[F]
            if kind == BC_PERIODIC:
                # Eq. hDG2 / hDG_NS2: element contribution <fhat + ghat, mu>
                Rt[:, f] = np.einsum("g,gc,bgm->bcm", T.Wf[f], T.psi[f], fh)
            elif kind == BC_STATE:          # <vhat - v_b, mu>
                vb = self.boundary_state[F][self.mesh.fnode_map[e, f]]
                vbf = T.psi[f] @ vb
                Rt[:, f] = np.einsum("g,gc,bgm->bcm", T.Wf[f], T.psi[f], vhf - vbf)
            elif kind == BC_SLIP:           # <fhat(vhat, v; n) + fhat(vhat, R v; -n), mu>
                fm = ph.numerical_flux_inviscid(vhf, reflect(vf, n), -n, g, self.phys.stabilization)
                Rt[:, f] = np.einsum("g,gc,bgm->bcm", T.Wf[f], T.psi[f], fh + fm)
            else:
                raise ValueError(kind)
        return Rq, Rv, Rt

    def _pack_l(self, Rq, Rv):
        B = Rv.shape[0]
        if self.viscous:
            return np.concatenate([Rq.reshape(B, -1), Rv.reshape(B, -1)], axis=1)
        return Rv.reshape(B, -1)

    def _unpack_x(self, x, Np):
        B = x.shape[0]
        if self.viscous:
            nq = Np * self.m * self.d
            return (x[:, :nq].reshape(B, Np, self.m, self.d),
                    x[:, nq:].reshape(B, Np, self.m))
        return None, x.reshape(B, Np, self.m)

    def local_residual(self, e, Q, V, Vh, mass_coef=0.0, hist_w=None):
        """Real residuals (R_l [n_i], R_t [n_t]) of element e."""
        Qb = None if Q is None else Q[None]
        Rq, Rv, Rt = self.element_residual(e, Qb, V[None], Vh[None], mass_coef, hist_w)
        Rt = Rt.reshape(-1)
        return self._pack_l(Rq, Rv)[0], (Rt[self.trace_mask(e)] if self.mixed else Rt)

    def local_jacobian(self, e, Q, V, Vh, mass_coef=0.0, hist_w=None):
        """Dense blocks A, B, C, D of d(R_l, R_t)/d(x, vhat) by complex step."""
        ni, nt = self.ni_e(e), self.n_t
        N = ni + nt
        x0 = V.reshape(-1) if Q is None else np.concatenate([Q.reshape(-1), V.reshape(-1)])
        y0 = Vh.reshape(-1)
        X = np.tile(x0.astype(np.complex128), (N, 1))
        Y = np.tile(y0.astype(np.complex128), (N, 1))
        X[np.arange(ni), np.arange(ni)] += 1j * CSTEP
        Y[ni + np.arange(nt), np.arange(nt)] += 1j * CSTEP
        Qb, Vb = self._unpack_x(X, V.shape[0])
        Rq, Rv, Rt = self.element_residual(e, Qb, Vb, Y.reshape((N,) + Vh.shape), mass_coef, hist_w)
        Jl = np.imag(self._pack_l(Rq, Rv)).T / CSTEP          # [ni, N]
        Jt = np.imag(Rt.reshape(N, -1)).T / CSTEP             # [nt, N]
        A, B, C, D = Jl[:, :ni], Jl[:, ni:], Jt[:, :ni], Jt[:, ni:]
        if self.mixed:                                        # drop the padding of the trace
            k = self.trace_mask(e)
            B, C, D = B[:, k], C[k], D[k][:, k]
        return A, B, C, D

    # -- condensation (Sec. 3.2: local elimination of the interior unknowns) -------------
    def condense(self, e, Q, V, Vh, mass_coef=0.0, hist_w=None):
        Rl, Rt = self.local_residual(e, Q, V, Vh, mass_coef, hist_w)
        A, B, C, D = self.local_jacobian(e, Q, V, Vh, mass_coef, hist_w)
        X = solve_equilibrated(A, B)
        y = solve_equilibrated(A, Rl)
        S = D - C @ X
        g = Rt - C @ y
        return dict(S=S, g=g, X=X, y=y, Rl=Rl, Rt=Rt, A=A, B=B, C=C, D=D)

    # -- derived quantities -----------------------------------------------------------------
    def consistent_q(self, e, V, Vh):
        """Q solving Eq. hDG_NS0 exactly for given (v, vhat): M Q = -R_q(Q=0)."""
        T = self.tables(e)
        Np = T.phi.shape[1]
        M = np.einsum("g,ga,gb->ab", T.W, T.phi, T.phi)
        Rq, _, _ = self.element_residual(e, np.zeros((1, Np, self.m, self.d)),
                                         V[None], Vh[None])
        return -np.linalg.solve(M, Rq[0].reshape(Np, -1)).reshape(Np, self.m, self.d)

    def history_weak(self, e, Vs, coefs):
        """hist_w [Np, m] = sum_j c_j (u(v_h^{n-j}), phi_a)_K."""
        T = self.tables(e)
        out = np.zeros((T.phi.shape[1], self.m))
        for Vj, c in zip(Vs, coefs):
            u = ph.u_of_v(T.phi @ Vj, self.phys.gamma)
            out += c * np.einsum("g,ga,gm->am", T.W, T.phi, u)
        return out

    def source_weak(self, e, s_nodes):
        """(s_h, phi_a)_K [Np, m] of a source term s of d u/dt + div(F + G) = s, s_h its nodal
        interpolant (values s_nodes [Np, m] at the element's nodes). The residual takes it with
        the history: R_v = ... - hist - (s_h, w), i.e. hist + source_weak (the paper's Couette
        problem, Sec. 5.2, carries such a source; how it is integrated is not stated)."""
        T = self.tables(e)
        return np.einsum("g,ga,gm->am", T.W, T.phi, T.phi @ s_nodes)

    def entropy_production_terms(self, Q, V):
        """(int rho s, (1/c_v) int (Phi / T + kappa |grad T|^2 / T^2)) of Eq. PiS (Sec. 5.6) with
        Phi = grad V : tau, both from (v_h, q_h) at the volume quadrature points; s = log(p / rho^gamma)
        (Sec. 2.3). Pi_S = d/dt int rho s - the second term is the scheme's own entropy production."""
        phys, g = self.phys, self.phys.gamma
        d = self.d
        tot_s = tot_phys = 0.0
        for e in range(self.mesh.E):
            T = self.tables(e)
            v = T.phi @ V[e]                                    # [ng, m]
            q = np.einsum("ga,amk->gmk", T.phi, Q[e])           # [ng, m, d]
            rho, vel, p = ph.primitives_of_v(v, g)
            tot_s += T.W @ (rho * ph.thermo_entropy(rho, p, g))
            w, vm = v[:, 1:-1], v[:, -1]
            gradV = -q[:, 1:-1, :] / vm[:, None, None] + w[:, :, None] * (q[:, -1, :] / vm[:, None] ** 2)[:, None, :]
            gradT = q[:, -1, :] / (phys.cv * vm[:, None] ** 2)
            Temp = 1.0 / (phys.cv * (-vm))
            fac = phys.viscosity_factor(vm) * np.ones_like(vm)
            mu, kappa = phys.mu * fac, phys.kappa * fac
            div = np.trace(gradV, axis1=1, axis2=2)
            tau = mu[..., None, None] * (gradV + np.swapaxes(gradV, 1, 2)) \
                - (2.0 / 3.0) * (mu * div)[:, None, None] * np.eye(d)
            Phi = np.einsum("gij,gij->g", gradV, tau)
            tot_phys += T.W @ ((Phi / Temp + kappa * np.sum(gradT ** 2, axis=1) / Temp ** 2) / phys.cv)
        return tot_s, tot_phys

    def integrals(self, V):
        """(total u [m], total generalised entropy int H) over the mesh."""
        tot_u = np.zeros(self.m)
        tot_H = 0.0
        for e in range(self.mesh.E):
            T = self.tables(e)
            u = ph.u_of_v(T.phi @ V[e], self.phys.gamma)
            tot_u += T.W @ u
            tot_H += T.W @ ph.entropy_H(u, self.phys.gamma)
        return tot_u, tot_H


def reflect(v, n):
    """The mirror image of the state v in the plane with unit normal n: w = (v_2..v_{d+1})
    -> w - 2 (w . n) n (the velocity V = -w / v_m reflects), v_1 and v_m unchanged."""
    w = v[..., 1:-1]
    w = w - 2.0 * np.sum(w * n, axis=-1)[..., None] * n
    return np.concatenate([v[..., :1], w, v[..., -1:]], axis=-1)


def solve_equilibrated(A, B):
    """A^{-1} B by LU with partial pivoting (numpy.linalg.solve) on the system scaled by powers
    of two, rows by 1/max|row|, then columns by 1/max|column|: X = c (r A c)^{-1} r B. The
    scaling is exact in floating point and does not change X; it matters because the local
    system mixes the q and v unknowns, whose rows differ by orders of magnitude (condition
    number ~6e9 for 3D NS p = 3 at h = 2 pi / 24, against ~6e5 after scaling), and the plain
    FP64 solve then loses about 3e-11 of X."""
    p2 = lambda x: np.exp2(np.round(np.log2(x)))
    r = p2(1.0 / np.abs(A).max(axis=1))
    As = r[:, None] * A
    c = p2(1.0 / np.abs(As).max(axis=0))
    Bs = r[:, None] * B if B.ndim == 2 else r * B
    Y = np.linalg.solve(As * c[None, :], Bs)
    return c[:, None] * Y if Y.ndim == 2 else c * Y


# ---------------------------------------------------------------------------------------
# State initialisation from primitive fields (interpolation at nodes)
# ---------------------------------------------------------------------------------------
def interpolate_state(prob: Problem, prim_fn):
    """V at element nodes and Vhat at the trace nodes (canonical face nodes; EDG: skeleton
    nodes) from prim_fn(x) -> (rho, vel, p)."""
    mesh, g = prob.mesh, prob.phys.gamma
    if prob.mixed:                                   # per-element degrees, trace at face degrees
        V = []
        for e in range(mesh.E):
            rho, vel, p = prim_fn(mesh.elem_nodes(e))
            V.append(ph.v_of_u(ph.u_of_primitives(rho, vel, p, g), g))
        Vhat = np.zeros(prob.trace_shape)
        for F, sides in enumerate(mesh.face_elems):
            e, f = sides[0]
            r = refel(mesh.dim, int(mesh.face_deg[F]))
            x = mesh.X[e, 0] + r.nodes[r.face_nodes[f]] @ mesh.J[e].T
            rho, vel, p = prim_fn(x)
            Vhat[mesh.fnode_off[F]:mesh.fnode_off[F + 1]] = ph.v_of_u(ph.u_of_primitives(rho, vel, p, g), g)
        return V, Vhat
    rho, vel, p = prim_fn(mesh.xnode)
    V = ph.v_of_u(ph.u_of_primitives(rho, vel, p, g), g)
    fn = np.array(mesh.ref.face_nodes)
    if prob.scheme == "edg":
        # a node's value from its first appearance over (element, local face, face node): periodic
        # copies of a node can differ by the field's own periodic tail (~1e-11 for the vortex)
        ids, first = np.unique(prob.edg_index.reshape(-1), return_index=True)
        Vhat = np.zeros(prob.trace_shape)
        Vhat[ids] = V[:, fn, :].reshape(-1, prob.m)[first]
        return V, Vhat
    return V, face_states(prob, V)


def face_states(prob: Problem, V):
    """[F, Nf, m]: the element nodal values V at every face's canonical nodes, taken from the
    face's first side (one degree): the HDG trace of an interpolated state, and the boundary
    state v_b (Problem.boundary_state) of the BC_STATE faces of any trace space."""
    fn = np.array(prob.mesh.ref.face_nodes)
    owner = np.array([sides[0] for sides in prob.mesh.face_elems])     # [F, 2] (e, f)
    return V[owner[:, 0][:, None], fn[owner[:, 1]]]


def bdf_coefficients(order: int, dt: float):
    """(mass_coef, history coefficients) of BDF1 / BDF2; order 0 = steady."""
    if order == 0:
        return 0.0, []
    if order == 1:
        return 1.0 / dt, [1.0 / dt]
    if order == 2:
        return 1.5 / dt, [2.0 / dt, -0.5 / dt]
    raise ValueError(order)


@dataclass
class NewtonResult:
    Q: np.ndarray | None
    V: np.ndarray
    Vhat: np.ndarray
    res_norms: list = field(default_factory=list)
    iters: int = 0


def assemble_trace(prob: Problem, locs, Vhat=None):
    """Assembled trace matrix (sparse CSR) and right-hand side -sum P^T g; on the rows of a
    strongly imposed state (EDG with boundaries; Vhat required) the identity and v_b - vhat."""
    n = prob.n_trace
    rows, cols, vals = [], [], []
    rhs = np.zeros(n)
    for e, L in enumerate(locs):
        gi = prob.trace_index(e)
        rows.append(np.repeat(gi, gi.size))
        cols.append(np.tile(gi, gi.size))
        vals.append(L["S"].ravel())
        np.add.at(rhs, gi, -L["g"])
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    drows, dres = prob.dirichlet_rows(Vhat) if prob.edg_dirichlet else (None, None)
    if drows is not None:
        keep = np.ones(n)
        keep[drows] = 0.0
        K = sp.diags(keep) @ K + sp.diags(1.0 - keep)
        rhs[drows] = -dres
        K = K.tocsr()
    return K, rhs


def solve_trace(K, rhs, dense_max=12000):
    if K.shape[0] <= dense_max:
        return np.linalg.solve(K.toarray(), rhs)
    return spla.spsolve(K.tocsc(), rhs)


def residual_norm(prob: Problem, locs, Vhat=None):
    """sqrt(sum_e |R_l,e|^2 + |sum_e P_e^T R_t,e|^2), the assembled trace residual being
    vhat - v_b on the rows of a strongly imposed state (EDG with boundaries; Vhat required)."""
    rt = np.zeros(prob.n_trace)
    s = 0.0
    for e, L in enumerate(locs):
        s += float(L["Rl"] @ L["Rl"])
        np.add.at(rt, prob.trace_index(e), L["Rt"])
    if prob.edg_dirichlet:
        drows, dres = prob.dirichlet_rows(Vhat)
        rt[drows] = dres
    return math.sqrt(s + float(rt @ rt))


def newton_iteration(prob: Problem, Q, V, Vhat, mass_coef, hist):
    """One full Newton iteration: condense every element, solve the trace system,
    recover the interior. Returns (Q', V', Vhat', residual norm before the update,
    dvhat, per-element local data)."""
    E = prob.mesh.E
    locs = []
    for e in range(E):
        Qe = None if Q is None else Q[e]
        locs.append(prob.condense(e, Qe, V[e], prob.gather_trace(Vhat, e), mass_coef,
                                  None if hist is None else hist[e]))
    rn = residual_norm(prob, locs, Vhat)
    K, rhs = assemble_trace(prob, locs, Vhat)
    dvh = solve_trace(K, rhs)
    Vhat_new = Vhat + dvh.reshape(Vhat.shape)
    cp = lambda A: [a.copy() for a in A] if isinstance(A, list) else A.copy()
    Qn = None if Q is None else cp(Q)
    Vn = cp(V)
    for e, L in enumerate(locs):
        dx = -(L["y"] + L["X"] @ dvh[prob.trace_index(e)])
        if Q is None:
            Vn[e] += dx.reshape(V[e].shape)
        else:
            nq = Q[e].size
            Qn[e] += dx[:nq].reshape(Q[e].shape)
            Vn[e] += dx[nq:].reshape(V[e].shape)
    return Qn, Vn, Vhat_new, rn, dvh, locs


def newton_solve(prob: Problem, Q, V, Vhat, mass_coef=0.0, hist=None, tol=1e-10, max_it=10):
    """Undamped Newton with the exact Jacobian; converged when
    |R| <= tol * max(1, |R_0|)."""
    res = NewtonResult(Q, V, Vhat)
    r0 = None
    for it in range(max_it + 1):
        Qn, Vn, Vhn, rn, _dvh, _ = newton_iteration(prob, res.Q, res.V, res.Vhat, mass_coef, hist)
        res.res_norms.append(rn)
        if r0 is None:
            r0 = rn
        if rn <= tol * max(1.0, r0) or it == max_it:
            break
        res.Q, res.V, res.Vhat = Qn, Vn, Vhn
        res.iters = it + 1
    return res


def time_step(prob: Problem, Q, V, Vhat, Vhist, order, dt, tol=1e-10, max_it=10):
    """One BDF step from history states Vhist = [V^n, V^{n-1}, ...]."""
    mass_coef, coefs = bdf_coefficients(order, dt)
    hist = [prob.history_weak(e, [Vj[e] for Vj in Vhist[:len(coefs)]], coefs) for e in range(prob.mesh.E)]
    if not prob.mixed:
        hist = np.stack(hist)
    return newton_solve(prob, Q, V, Vhat, mass_coef, hist, tol, max_it)


def dirk3_tableau():
    """Butcher tableau (A [3x3], b, c) of the three-stage, third-order, L-stable DIRK(3,3)
    method of Alexander used in Sec. 5. The diagonal g is the root in (1/6, 1/2) of
    g^3 - 3 g^2 + 3 g / 2 - 1/6 = 0 (the condition for third order with L-stability);
    c_2 = (1 + g)/2, b_1 = -(6 g^2 - 16 g + 1)/4, b_2 = (6 g^2 - 20 g + 5)/4, b_3 = g, and the
    last row of A equals b (stiffly accurate)."""
    lo, hi = 1.0 / 6.0, 0.5
    f = lambda x: x ** 3 - 3.0 * x * x + 1.5 * x - 1.0 / 6.0
    for _ in range(200):                       # bisection: f(1/6) > 0 > f(1/2)
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    g = 0.5 * (lo + hi)
    c2 = 0.5 * (1.0 + g)
    b1 = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0
    b2 = (6.0 * g * g - 20.0 * g + 5.0) / 4.0
    A = np.array([[g, 0.0, 0.0], [c2 - g, g, 0.0], [b1, b2, g]])
    return A, A[2].copy(), np.array([g, c2, 1.0])


def dirk3_step(prob: Problem, Q, V, Vhat, dt, tol=1e-10, max_it=10):
    """One DIRK(3,3) step from level n (V, Vhat) (Sec. 5). Stage i solves the discrete
    equations with the time term
        (u_i - u_n, w) / (dt a_ii) - sum_{j<i} (a_ij / a_ii) (k_j, w),
    i.e. mass_coef = 1 / (dt a_ii) and hist_i = (u_n, w) / (dt a_ii) + sum_{j<i} (a_ij/a_ii) (k_j, w),
    where the weak stage derivatives follow from the stage equations themselves:
        (k_j, w) = (u_j - u_n, w) / (dt a_jj) - sum_{l<j} (a_jl / a_jj) (k_l, w).
    Each stage starts Newton from the previous stage's state; the method is stiffly accurate,
    so u_{n+1} = u_3. Returns (NewtonResult of the last stage, Newton updates per stage)."""
    A, _, _ = dirk3_tableau()
    E = prob.mesh.E
    # per-element weak forms: one array [E, Np, m], or (mixed degrees) a list of [Np_e, m] arrays
    weak = lambda Vs: (lambda L: L if prob.mixed else np.stack(L))(
        [prob.history_weak(e, [Vs[e]], [1.0]) for e in range(E)])
    lin = lambda a, X, b, Y: ([a * x + b * y for x, y in zip(X, Y)] if prob.mixed else a * X + b * Y)
    Un = weak(V)
    ks = []
    cur = NewtonResult(Q, V, Vhat)
    iters = []
    for i in range(3):
        aii = A[i, i]
        hist = [u / (dt * aii) for u in Un] if prob.mixed else Un / (dt * aii)
        for j in range(i):
            hist = lin(1.0, hist, A[i, j] / aii, ks[j])
        res = newton_solve(prob, cur.Q, cur.V, cur.Vhat, 1.0 / (dt * aii), hist, tol, max_it)
        iters.append(res.iters)
        Ui = weak(res.V)
        k = [(u - un) / (dt * aii) for u, un in zip(Ui, Un)] if prob.mixed else (Ui - Un) / (dt * aii)
        for j in range(i):
            k = lin(1.0, k, -(A[i, j] / aii), ks[j])
        ks.append(k)
        cur = res
    return cur, iters


def consistent_Q(prob: Problem, V, Vhat):
    if not prob.viscous:
        return None
    Q = [prob.consistent_q(e, V[e], prob.gather_trace(Vhat, e)) for e in range(prob.mesh.E)]
    return Q if prob.mixed else np.stack(Q)
