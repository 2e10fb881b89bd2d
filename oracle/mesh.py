"""Periodic simplex meshes for the oracle (Sec. 3.1.1 mesh; Sec. 3.4 counting).

The paper uses triangles from split Cartesian grids and tetrahedral meshes with
about 2 N_v triangles or 6 N_v tetrahedra (Sec. 3.4). The split is not printed;
the reading used here is the Kuhn (Freudenthal) split along the main diagonal,
identical in every cell, which is conforming under periodic identification:

* 2D cell (i, j), index c = j n + i; triangles (00,10,11) and (00,11,01); e = 2c + t.
* 3D cell (i, j, k), c = (k n + j) n + i; for each axis permutation s (lexicographic
  order) the tetrahedron 0, e_s0, e_s0 + e_s1, (1,1,1); when its determinant is
  negative vertices 1 and 2 are swapped; e = 6c + t.

A face is the set of element vertices other than local vertex f. Faces are keyed by
(min vertex mod n on periodic axes, offsets of the other two vertices), so periodic
copies coincide even for n = 1.

Boundaries (the term b_h of Eqs. hDG2 / hDG_NS2, Sec. 3.2): an axis is periodic (the
default) or bounded on both sides; each side of a bounded axis carries a boundary type
(BC_STATE or BC_SLIP, see oracle.hdg). A face with one side lies on such a side; it is
owned by its element. Global faces are numbered in order of first appearance over
(element, local face); the first element is the owner and its local face-node
order is the face's canonical node order. Face nodes of the other element are
matched by integer node coordinates (units h/p) relative to the face's smallest
vertex, which periodic copies share.

Mixed degrees (the paper uses one degree k everywhere; this extension is not in it): with
p_elem given, element e carries P_{p_e}, and the trace on a face carries the larger degree of
its two sides, q_F = max(p_L, p_R). Element e then has face degrees q_{e,f} = q_F of its faces
and a trace degree PT_e = max_f q_{e,f} >= p_e. The trace unknowns are the face nodes of degree
q_F (the face nodes of the degree-q_F reference element on that face), numbered face by face
(fnode_off), in the owner's local order; the other side is matched by integer node coordinates
in units h/q_F. Mixed degrees are built for periodic meshes.
"""
from __future__ import annotations

import itertools

import numpy as np

from .refel import refel

BC_PERIODIC, BC_STATE, BC_SLIP = 0, 1, 2
BC_NAMES = {"periodic": BC_PERIODIC, "state": BC_STATE, "slip": BC_SLIP}


class Mesh:
    def __init__(self, dim: int, n: int, lo: float, hi: float, p: int, deg: int | None = None,
                 bc=None, verts=None, p_elem=None):
        """bc: per axis a pair (lo side, hi side) of "periodic", "state" or "slip" (default:
        all periodic); an axis is periodic on both sides or on neither.
        verts: lattice vertex coordinates [E, d+1, d] of the elements on [0, n]^d, positively
        oriented (default: the Kuhn split of the n^d grid).
        p_elem: degree of every element [E] (mixed degrees; p is then ignored and the largest
        degree takes its place in the uniform arrays)."""
        if p_elem is not None:
            p_elem = np.asarray(p_elem, dtype=np.int64)
            if p_elem.ndim != 1 or p_elem.min() < 1:
                raise ValueError("p_elem: one degree >= 1 per element")
            if deg is not None or bc is not None:
                raise ValueError("mixed degrees: periodic meshes with the default rules only")
            p = int(p_elem.max())
        self.dim, self.n, self.p = dim, n, p
        bc = bc if bc is not None else [("periodic", "periodic")] * dim
        self.bc = np.array([[BC_NAMES[s] for s in pair] for pair in bc], dtype=np.int64)   # [dim, 2]
        if self.bc.shape != (dim, 2) or np.any((self.bc[:, 0] == 0) != (self.bc[:, 1] == 0)):
            raise ValueError("bc: an axis is periodic on both sides or on neither")
        self.periodic = self.bc[:, 0] == BC_PERIODIC
        self.lo, self.hi = float(lo), float(hi)
        self.h = (self.hi - self.lo) / n
        self.ref = refel(dim, p, deg)
        ref = self.ref
        if dim == 2:
            cell = np.array([[(0, 0), (1, 0), (1, 1)], [(0, 0), (1, 1), (0, 1)]], dtype=np.int64)
            jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
            origin = np.stack([ii.ravel(), jj.ravel()], axis=-1)              # cells, x fastest
        else:
            tets = []
            for s in itertools.permutations(range(3)):
                P = [np.zeros(3, int)]
                P.append(P[0] + np.eye(3, dtype=int)[s[0]])
                P.append(P[1] + np.eye(3, dtype=int)[s[1]])
                P.append(np.ones(3, int))
                if np.linalg.det(np.array([P[1], P[2], P[3]], float)) < 0:
                    P[1], P[2] = P[2], P[1]
                tets.append(P)
            cell = np.array(tets, dtype=np.int64)                              # [6, 4, 3]
            kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
            origin = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=-1)
        if verts is None:
            verts = (origin[:, None, None, :] + cell[None]).reshape(-1, cell.shape[1], dim)
        verts = np.asarray(verts, dtype=np.int64)
        self.L = verts.astype(np.int64)              # [E, nF, dim]
        self.E = len(verts)
        self.X = self.lo + self.h * self.L.astype(np.float64)
        X0 = self.X[:, 0, :]
        self.J = np.transpose(self.X[:, 1:, :] - X0[:, None, :], (0, 2, 1))   # [E, dim, dim], columns
        self.detJ = np.linalg.det(self.J)
        self.Jinv = np.linalg.inv(self.J)
        # node coordinates
        self.xnode = X0[:, None, :] + np.einsum("erc,ac->ear", self.J, ref.nodes)
        idx = np.array(ref.idx, dtype=np.int64)
        self.Nint = (p * self.L[:, 0, None, :]
                     + np.einsum("erc,ac->ear", (self.L[:, 1:, :] - self.L[:, 0:1, :]).transpose(0, 2, 1), idx))
        self._faces()
        self._face_geometry()
        self.p_elem = None
        if p_elem is not None:
            if len(p_elem) != self.E:
                raise ValueError("p_elem: one degree per element")
            self.p_elem = p_elem
            self._mixed_faces()

    # -- topology -------------------------------------------------------------------
    def _encode(self, arr):
        """Integers -> one int64 per row, monotone in the lexicographic row order."""
        W = 4 * (self.n * self.p + 8)
        out = np.zeros(arr.shape[:-1], dtype=np.int64)
        for r in range(arr.shape[-1]):
            out = out * W + (arr[..., r] + W // 2)
        return out

    def _faces(self):
        ref, n, p, E = self.ref, self.n, self.p, self.E
        nF, Nf = ref.nF, ref.Nf
        # vertices of every (element, local face), sorted lexicographically
        fv = self.L[:, np.array(ref.face_verts), :]                        # [E, nF, nF-1, d]
        order = np.argsort(self._encode(fv), axis=-1, kind="stable")
        fv = np.take_along_axis(fv, order[..., None], axis=2)
        A = fv[:, :, 0, :]                                                 # smallest vertex
        Ak = np.where(self.periodic, A % n, A)
        key = np.concatenate([Ak, (fv[:, :, 1:, :] - A[:, :, None, :]).reshape(E, nF, -1)], axis=-1)
        key = key.reshape(E * nF, -1)
        _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
        inv = inv.reshape(-1)
        rank = np.empty(len(first), dtype=np.int64)                        # first-appearance order
        rank[np.argsort(first, kind="stable")] = np.arange(len(first))
        face_of = rank[inv]
        self.face_of = face_of.reshape(E, nF)
        self.nFaces = len(first)
        srt = np.argsort(face_of, kind="stable")                           # sides in appearance order
        counts = np.bincount(face_of, minlength=self.nFaces)
        assert np.all((counts == 1) | (counts == 2))
        starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
        flat = [srt[s:s + c] for s, c in zip(starts, counts)]               # flat (e * nF + f)
        self.face_elems = [[(int(a // nF), int(a % nF)) for a in fl] for fl in flat]
        # boundary faces: every vertex on one side of a bounded axis
        self.face_bc = np.zeros(self.nFaces, dtype=np.int64)
        self.face_wall = np.full((self.nFaces, 2), -1, dtype=np.int64)    # (axis, side)
        for F in np.nonzero(counts == 1)[0]:
            a0 = flat[F][0]
            v = fv[a0 // nF, a0 % nF]                                      # [nF-1, d]
            hit = [(r, s) for r in range(self.dim) if not self.periodic[r] for s in (0, 1)
                   if np.all(v[:, r] == (0 if s == 0 else n))]
            assert len(hit) == 1, "a face with one side lies on one side of a bounded axis"
            self.face_wall[F] = hit[0]
            self.face_bc[F] = self.bc[hit[0]]
        sides = np.array([fl for fl in flat if len(fl) == 2]).reshape(-1, 2)
        owners = np.array([fl[0] for fl in flat])
        # face-node keys: node position (units h/p) relative to the face's smallest vertex;
        # periodic copies of a face differ by a translation, so both sides share the keys
        fn = np.array(ref.face_nodes)                                      # [nF, Nf]
        KN = self.Nint[:, fn, :] - p * A[:, :, None, :]                     # [E, nF, Nf, d]
        codes = self._encode(KN).reshape(E * nF, Nf)
        c0, c1 = codes[sides[:, 0]], codes[sides[:, 1]]
        o0, o1 = np.argsort(c0, axis=1), np.argsort(c1, axis=1)
        assert np.array_equal(np.take_along_axis(c0, o0, 1), np.take_along_axis(c1, o1, 1))
        assert np.all(np.diff(np.take_along_axis(c0, o0, 1), axis=1) > 0)
        fmap = np.zeros((E * nF, Nf), dtype=np.int64)
        fmap[owners] = np.arange(Nf)                                       # owner: canonical order
        m1 = np.zeros_like(c1)
        np.put_along_axis(m1, o1, o0, axis=1)
        fmap[sides[:, 1]] = m1
        self.fnode_map = fmap.reshape(E, nF, Nf)

    def _mixed_faces(self):
        """Face degrees q_F = max(p_L, p_R), the trace degree of every element and the face-node
        maps at degree q_F (owner order canonical, the other side matched by node coordinates)."""
        dim, nF, E = self.dim, self.ref.nF, self.E
        pe = self.p_elem
        self.face_deg = np.array([max(int(pe[e]) for e, _f in sides) for sides in self.face_elems],
                                 dtype=np.int64)
        self.elem_face_deg = self.face_deg[self.face_of]                  # [E, nF]
        self.elem_trace_deg = self.elem_face_deg.max(axis=1)              # [E]
        nf = {q: refel(dim, q).Nf for q in range(1, self.p + 1)}
        self.face_nnodes = np.array([nf[int(q)] for q in self.face_deg], dtype=np.int64)
        self.fnode_off = np.concatenate([[0], np.cumsum(self.face_nnodes)]).astype(np.int64)
        self.Nf_max = max(nf[int(q)] for q in self.face_deg)
        fmap = np.full((E, nF, self.Nf_max), -1, dtype=np.int64)
        fv_all = self.ref.face_verts
        for F, sides in enumerate(self.face_elems):
            q = int(self.face_deg[F])
            r = refel(dim, q)
            idx = np.array(r.idx, dtype=np.int64)
            codes = []
            for (e, f) in sides:
                L = self.L[e]
                Nq = q * L[0] + idx @ (L[1:] - L[0])                      # degree-q lattice of e
                fv = L[fv_all[f]]
                A = fv[np.argmin(self._encode(fv))]                        # smallest face vertex
                codes.append(self._encode(Nq[r.face_nodes[f]] - q * A))
            e0, f0 = sides[0]
            fmap[e0, f0, :r.Nf] = np.arange(r.Nf)
            if len(sides) == 2:
                c0, c1 = codes
                o0, o1 = np.argsort(c0), np.argsort(c1)
                assert np.array_equal(c0[o0], c1[o1])
                m1 = np.empty(r.Nf, dtype=np.int64)
                m1[o1] = o0
                e1, f1 = sides[1]
                fmap[e1, f1, :r.Nf] = m1
        self.fnode_map_mixed = fmap

    def elem_nodes(self, e):
        """Physical coordinates [Np_e, d] of the nodes of element e at its own degree."""
        r = refel(self.dim, int(self.p_elem[e])) if self.p_elem is not None else self.ref
        return self.X[e, 0] + r.nodes @ self.J[e].T

    def _face_geometry(self):
        ref, dim = self.ref, self.dim
        nF = ref.nF
        self.normal = np.zeros((self.E, nF, dim))
        self.face_jac = np.zeros((self.E, nF))
        pm = 1.0 if dim == 2 else 0.5                # measure of the parameter simplex
        for f in range(nF):
            Y = self.X[:, ref.face_verts[f]]         # [E, dim, dim]
            opp = self.X[:, f]
            if dim == 2:
                t = Y[:, 1] - Y[:, 0]
                nv = np.stack([t[:, 1], -t[:, 0]], axis=-1)
                area = np.linalg.norm(t, axis=-1)
            else:
                nv = np.cross(Y[:, 1] - Y[:, 0], Y[:, 2] - Y[:, 0])
                area = 0.5 * np.linalg.norm(nv, axis=-1)
            nv = nv / np.linalg.norm(nv, axis=-1, keepdims=True)
            flip = np.sum(nv * (opp - Y[:, 0]), axis=-1) > 0
            nv[flip] = -nv[flip]
            self.normal[:, f] = nv
            self.face_jac[:, f] = area / pm

    # -- counting (Sec. 3.4, Eqs. dof / nnz, Tables t:dofs / t:nnz) ------------------
    @property
    def n_vertices(self):
        return self.n ** self.dim

    def trace_dof_hdg(self):
        return self.nFaces * self.ref.Nf

    def trace_block_nnz_hdg(self):
        """Number of scalar-per-component nonzeros of the HDG trace Jacobian / m^2."""
        nb = 0
        for F, sides in enumerate(self.face_elems):
            coupled = set()
            for (e, _f) in sides:
                coupled.update(int(x) for x in self.face_of[e])
            nb += len(coupled)
        return nb * self.ref.Nf ** 2

    def _trace_nodes_edg(self):
        period = self.n * self.p
        ids = {}
        elem_nodes = []
        ref = self.ref
        for e in range(self.E):
            s = set()
            for f in range(ref.nF):
                for a in ref.face_nodes[f]:
                    key = tuple(np.where(self.periodic, self.Nint[e, a] % period, self.Nint[e, a]))
                    if key not in ids:
                        ids[key] = len(ids)
                    s.add(ids[key])
            elem_nodes.append(s)
        return ids, elem_nodes

    def edg_numbering(self, interior_only: bool = False):
        """The continuous trace spaces of Sec. 3.4: one unknown per skeleton node, numbered in
        order of first appearance over (element, local face, face node). EDG (E^E_h = all faces):
        a node is shared by every face through it. IEDG (interior_only; E^E_h = the interior
        faces): the trace is continuous on the interior faces only, so each node of a face on the
        boundary is its own unknown, shared with no other face (on a periodic mesh every face is
        interior and IEDG is EDG). Returns (number of nodes, index [E, nF, Nf] of every local face
        node)."""
        period = self.n * self.p
        nF, Nf = self.ref.nF, self.ref.Nf
        fn = np.array(self.ref.face_nodes)                                  # [nF, Nf]
        keys = np.where(self.periodic, self.Nint[:, fn, :] % period, self.Nint[:, fn, :])  # [E, nF, Nf, d]
        ids = {}
        index = np.zeros((self.E, nF, Nf), dtype=np.int64)
        for e in range(self.E):
            for f in range(nF):
                own = interior_only and self.face_bc[self.face_of[e, f]] != 0
                for c in range(Nf):
                    key = ("face", e, f, c) if own else tuple(keys[e, f, c])
                    if key not in ids:
                        ids[key] = len(ids)
                    index[e, f, c] = ids[key]
        return len(ids), index

    def trace_dof_edg(self):
        ids, _ = self._trace_nodes_edg()
        return len(ids)

    def trace_nnz_edg(self):
        ids, elem_nodes = self._trace_nodes_edg()
        nbr = [set() for _ in range(len(ids))]
        for s in elem_nodes:
            for a in s:
                nbr[a].update(s)
        return sum(len(x) for x in nbr)

    def dof_dg(self):
        return self.E * self.ref.Np

    def nnz_dg(self):
        return self.E * (1 + self.ref.nF) * self.ref.Np ** 2
