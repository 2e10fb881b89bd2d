"""Reference simplex for the oracle (Sec. 3.1.2 spaces; quadrature and basis are
not fixed by the paper, see the readings listed in the oracle header).

* Gauss-Jacobi rules by Golub-Welsch (eigen-decomposition of the Jacobi matrix of
  the three-term recurrence), collapsed (Duffy) onto the triangle / tetrahedron,
  k = ceil((deg+1)/2) points per direction, exact for total degree 2k-1.
* Nodal Lagrange basis of P_p on equispaced nodes, lexicographic (i fastest),
  obtained by inverting a plain monomial Vandermonde matrix.
* Local face f is the face opposite reference vertex f.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np


def gauss_jacobi(n: int, alpha: float, beta: float):
    """n-point Gauss-Jacobi rule on [-1, 1] for the weight (1-x)^alpha (1+x)^beta."""
    ab = alpha + beta
    diag = np.empty(n)
    diag[0] = (beta - alpha) / (ab + 2.0)
    for i in range(1, n):
        diag[i] = (beta ** 2 - alpha ** 2) / ((2 * i + ab) * (2 * i + ab + 2))
    off = np.empty(max(n - 1, 0))
    for i in range(1, n):
        num = 4.0 * i * (i + alpha) * (i + beta) * (i + ab)
        den = (2 * i + ab) ** 2 * (2 * i + ab + 1) * (2 * i + ab - 1)
        off[i - 1] = math.sqrt(num / den)
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, vec = np.linalg.eigh(T)
    mu0 = 2.0 ** (ab + 1) * math.gamma(alpha + 1) * math.gamma(beta + 1) / math.gamma(ab + 2)
    w = mu0 * vec[0, :] ** 2
    return x, w


def simplex_rule(dim: int, deg: int):
    """Quadrature on the reference simplex {r_i >= 0, sum r_i <= 1}.

    Returns points [n, dim] and weights [n] (weights sum to 1/dim!).
    dim = 1 is the unit interval [0, 1].
    """
    k = max(1, math.ceil((deg + 1) / 2))
    if dim == 1:
        a, wa = gauss_jacobi(k, 0.0, 0.0)
        return ((a + 1) / 2)[:, None], wa / 2
    if dim == 2:
        a, wa = gauss_jacobi(k, 0.0, 0.0)
        b, wb = gauss_jacobi(k, 1.0, 0.0)
        pts, wts = [], []
        for j in range(k):
            for i in range(k):
                s = (1 + b[j]) / 2
                r = (1 + a[i]) / 2 * (1 - s)
                pts.append((r, s))
                wts.append(wa[i] * wb[j] / 8.0)
        return np.array(pts), np.array(wts)
    if dim == 3:
        a, wa = gauss_jacobi(k, 0.0, 0.0)
        b, wb = gauss_jacobi(k, 1.0, 0.0)
        c, wc = gauss_jacobi(k, 2.0, 0.0)
        pts, wts = [], []
        for l in range(k):
            for j in range(k):
                for i in range(k):
                    t = (1 + c[l]) / 2
                    s = (1 + b[j]) / 2 * (1 - t)
                    r = (1 + a[i]) / 2 * (1 - s - t)
                    pts.append((r, s, t))
                    wts.append(wa[i] * wb[j] * wc[l] / 64.0)
        return np.array(pts), np.array(wts)
    raise ValueError(dim)


def lattice(dim: int, p: int):
    """Multi-indices (i, j[, k]) with total <= p, i fastest."""
    out = []
    if dim == 1:
        return [(i,) for i in range(p + 1)]
    if dim == 2:
        for j in range(p + 1):
            for i in range(p + 1 - j):
                out.append((i, j))
        return out
    for k in range(p + 1):
        for j in range(p + 1 - k):
            for i in range(p + 1 - k - j):
                out.append((i, j, k))
    return out


def ref_vertices(dim: int) -> np.ndarray:
    return np.vstack([np.zeros(dim), np.eye(dim)])


class RefElement:
    """Nodal P_p Lagrange element on the reference simplex with its rules."""

    def __init__(self, dim: int, p: int, deg: int | None = None):
        self.dim, self.p = dim, p
        self.deg = 2 * p + 1 if deg is None else deg
        self.idx = lattice(dim, p)
        self.nodes = np.array(self.idx, dtype=np.float64) / p
        self.Np = len(self.idx)
        mono = np.array(self.idx)                         # exponents, same lattice
        self.mono = mono
        Vm = self._monomials(self.nodes)                  # [node, mono]
        self.coef = np.linalg.inv(Vm)                     # phi_a = sum_m coef[m,a] x^m
        self.qp, self.qw = simplex_rule(dim, self.deg)
        self.fqp, self.fqw = simplex_rule(dim - 1, self.deg) if dim > 1 else (None, None)
        self.nF = dim + 1
        # face f opposite vertex f: node membership and (sorted) local face nodes
        self.face_nodes = []
        for f in range(self.nF):
            if f == 0:
                mask = [sum(ix) == p for ix in self.idx]
            else:
                mask = [ix[f - 1] == 0 for ix in self.idx]
            self.face_nodes.append([a for a, mk in enumerate(mask) if mk])
        self.Nf = len(self.face_nodes[0])
        rv = ref_vertices(dim)
        self.face_verts = [[v for v in range(self.nF) if v != f] for f in range(self.nF)]
        # reference face quadrature points mapped into the element
        self.fqp_ref = []
        for f in range(self.nF):
            Y = rv[self.face_verts[f]]
            pts = Y[0] + self.fqp @ (Y[1:] - Y[0])
            self.fqp_ref.append(pts)

    def _monomials(self, x):
        x = np.atleast_2d(x)
        out = np.ones((x.shape[0], len(self.mono)))
        for m, e in enumerate(self.mono):
            for r in range(self.dim):
                out[:, m] *= x[:, r] ** e[r]
        return out

    def _monomial_grads(self, x):
        x = np.atleast_2d(x)
        out = np.zeros((x.shape[0], len(self.mono), self.dim))
        for m, e in enumerate(self.mono):
            for r in range(self.dim):
                if e[r] == 0:
                    continue
                g = e[r] * x[:, r] ** (e[r] - 1)
                for s in range(self.dim):
                    if s != r:
                        g = g * x[:, s] ** e[s]
                out[:, m, r] = g
        return out

    def phi(self, x):
        """Basis values [npts, Np]."""
        return self._monomials(x) @ self.coef

    def dphi(self, x):
        """Reference gradients [npts, Np, dim]."""
        return np.einsum("qmr,ma->qar", self._monomial_grads(x), self.coef)


@lru_cache(maxsize=None)
def refel(dim: int, p: int, deg: int | None = None) -> RefElement:
    return RefElement(dim, p, deg)
