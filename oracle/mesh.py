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
(min vertex mod n, offsets of the other two vertices), so periodic copies coincide
even for n = 1. Global faces are numbered in order of first appearance over
(element, local face); the first element is the owner and its local face-node
order is the face's canonical node order. Face nodes of the other element are
matched by integer node coordinates (units h/p) relative to the face's smallest
vertex, which periodic copies share.
"""
from __future__ import annotations

import itertools

import numpy as np

from .refel import refel


class Mesh:
    def __init__(self, dim: int, n: int, lo: float, hi: float, p: int, deg: int | None = None):
        self.dim, self.n, self.p = dim, n, p
        self.lo, self.hi = float(lo), float(hi)
        self.h = (self.hi - self.lo) / n
        self.ref = refel(dim, p, deg)
        ref = self.ref
        verts = []                                   # integer lattice coords per element
        if dim == 2:
            tris = [[(0, 0), (1, 0), (1, 1)], [(0, 0), (1, 1), (0, 1)]]
            for j in range(n):
                for i in range(n):
                    for t in tris:
                        verts.append([(i + a, j + b) for a, b in t])
        else:
            perms = list(itertools.permutations(range(3)))
            for k in range(n):
                for j in range(n):
                    for i in range(n):
                        for s in perms:
                            P = [np.zeros(3, int)]
                            P.append(P[0] + np.eye(3, dtype=int)[s[0]])
                            P.append(P[1] + np.eye(3, dtype=int)[s[1]])
                            P.append(np.ones(3, int))
                            if np.linalg.det(np.array([P[1], P[2], P[3]], float)) < 0:
                                P[1], P[2] = P[2], P[1]
                            verts.append([tuple(np.array((i, j, k)) + q) for q in P])
        self.L = np.array(verts, dtype=np.int64)     # [E, nF, dim]
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

    # -- topology -------------------------------------------------------------------
    def _face_key(self, e, f):
        vs = sorted(tuple(v) for k, v in enumerate(self.L[e]) if k != f)
        A = np.array(vs[0])
        return (tuple(A % self.n),) + tuple(tuple(np.array(v) - A) for v in vs[1:])

    def _faces(self):
        ref, n, p = self.ref, self.n, self.p
        nF = ref.nF
        key2id = {}
        self.face_of = np.zeros((self.E, nF), dtype=np.int64)
        self.face_elems = []
        for e in range(self.E):
            for f in range(nF):
                k = self._face_key(e, f)
                if k not in key2id:
                    key2id[k] = len(self.face_elems)
                    self.face_elems.append([(e, f)])
                else:
                    self.face_elems[key2id[k]].append((e, f))
                self.face_of[e, f] = key2id[k]
        self.nFaces = len(self.face_elems)
        assert all(len(s) == 2 for s in self.face_elems), "periodic mesh: every face has two sides"
        self.fnode_map = np.zeros((self.E, nF, ref.Nf), dtype=np.int64)
        for F, sides in enumerate(self.face_elems):
            e0, f0 = sides[0]
            canon = [self._face_node_key(e0, f0, a) for a in ref.face_nodes[f0]]
            pos = {c: i for i, c in enumerate(canon)}
            assert len(pos) == ref.Nf
            for (e, f) in sides:
                for c, a in enumerate(ref.face_nodes[f]):
                    self.fnode_map[e, f, c] = pos[self._face_node_key(e, f, a)]

    def _face_node_key(self, e, f, a):
        """Node position (units h/p) relative to the face's smallest vertex: periodic
        copies of a face differ by a translation, so the key is the same on both sides."""
        A = min(tuple(v) for k, v in enumerate(self.L[e]) if k != f)
        return tuple(self.Nint[e, a] - self.p * np.array(A))

    def _face_geometry(self):
        ref, dim = self.ref, self.dim
        nF = ref.nF
        self.normal = np.zeros((self.E, nF, dim))
        self.face_jac = np.zeros((self.E, nF))
        pm = 1.0 if dim == 2 else 0.5                # measure of the parameter simplex
        for e in range(self.E):
            for f in range(nF):
                Y = self.X[e, ref.face_verts[f]]
                opp = self.X[e, f]
                if dim == 2:
                    t = Y[1] - Y[0]
                    nv = np.array([t[1], -t[0]])
                    area = np.linalg.norm(t)
                else:
                    c = np.cross(Y[1] - Y[0], Y[2] - Y[0])
                    nv = c
                    area = 0.5 * np.linalg.norm(c)
                nv = nv / np.linalg.norm(nv)
                if np.dot(nv, opp - Y[0]) > 0:
                    nv = -nv
                self.normal[e, f] = nv
                self.face_jac[e, f] = area / pm

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
                    key = tuple(self.Nint[e, a] % period)
                    if key not in ids:
                        ids[key] = len(ids)
                    s.add(ids[key])
            elem_nodes.append(s)
        return ids, elem_nodes

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
