"""Pins of the oracle's reference element and mesh against closed forms, library
routines and the paper's counting tables (Sec. 3.4, Tables t:dofs and t:nnz)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.mesh import Mesh
from oracle.refel import RefElement, gauss_jacobi, lattice, simplex_rule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dof_nnz_tables.txt")


def test_gauss_legendre_matches_library():
    for n in range(1, 8):
        x, w = gauss_jacobi(n, 0.0, 0.0)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(np.sort(x), np.sort(xr), atol=1e-14)
        assert np.allclose(w[np.argsort(x)], wr[np.argsort(xr)], atol=1e-14)


@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_gauss_jacobi_exactness(alpha):
    # int_{-1}^{1} (1-x)^alpha x^k dx, by the binomial expansion of x = 1 - (1-x)
    for n in range(1, 7):
        x, w = gauss_jacobi(n, alpha, 0.0)
        for k in range(2 * n):
            a = int(alpha)
            exact = float(sum(Fraction(math.comb(k, j) * (-1) ** j * 2 ** (a + j + 1), a + j + 1)
                              for j in range(k + 1)))
            assert abs(np.dot(w, x ** k) - exact) < 1e-12 * max(1, abs(exact))


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_simplex_rule_exact_to_2k_minus_1(dim):
    # int over the unit simplex of prod r_i^{a_i} = prod a_i! / (sum a_i + dim)!
    for deg in range(0, 10):
        pts, wts = simplex_rule(dim, deg)
        k = math.ceil((deg + 1) / 2)
        top = 2 * k - 1
        for a in lattice(dim, top):
            exact = math.prod(math.factorial(t) for t in a) / math.factorial(sum(a) + dim)
            got = np.dot(wts, np.prod(pts ** np.array(a), axis=1))
            assert abs(got - exact) < 1e-14, (dim, deg, a)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 3), (3, 4)])
def test_lagrange_basis(dim, p):
    ref = RefElement(dim, p)
    assert ref.Np == math.comb(p + dim, dim)
    assert np.allclose(ref.phi(ref.nodes), np.eye(ref.Np), atol=1e-11)
    rng = np.random.default_rng(0)
    x = rng.dirichlet(np.ones(dim + 1), size=20)[:, 1:]
    assert np.allclose(ref.phi(x).sum(1), 1.0, atol=1e-12)
    assert np.allclose(ref.dphi(x).sum(1), 0.0, atol=1e-10)
    # reproduces a degree-p polynomial and its gradient
    c = rng.normal(size=dim)
    P = lambda y: (1.0 + y @ c) ** p
    dP = lambda y: p * (1.0 + y @ c)[:, None] ** (p - 1) * c
    assert np.allclose(ref.phi(x) @ P(ref.nodes), P(x), atol=1e-11)
    assert np.allclose(np.einsum("qar,a->qr", ref.dphi(x), P(ref.nodes)), dP(x), atol=1e-9)
    # face f = face opposite vertex f; its nodes have barycentric coordinate f equal to 0
    bary = np.hstack([1 - ref.nodes.sum(1, keepdims=True), ref.nodes])
    for f in range(ref.nF):
        assert len(ref.face_nodes[f]) == math.comb(p + dim - 1, dim - 1)
        assert np.allclose(bary[ref.face_nodes[f], f], 0.0)
        assert np.allclose(np.hstack([1 - ref.fqp_ref[f].sum(1, keepdims=True), ref.fqp_ref[f]])[:, f], 0.0)
        # element basis functions of off-face nodes vanish on the face
        off = [a for a in range(ref.Np) if a not in ref.face_nodes[f]]
        assert np.allclose(ref.phi(ref.fqp_ref[f])[:, off], 0.0, atol=1e-12)


@pytest.mark.parametrize("dim,n,p", [(2, 3, 2), (3, 2, 2), (3, 1, 1)])
def test_mesh_geometry_and_faces(dim, n, p):
    L = 2.0
    m = Mesh(dim, n, 0.0, L, p)
    assert m.E == (2 if dim == 2 else 6) * n ** dim
    assert m.nFaces == (3 if dim == 2 else 12) * n ** dim
    assert abs(np.abs(m.detJ).sum() / math.factorial(dim) - L ** dim) < 1e-12
    assert np.all(m.detJ > 0)
    period = n * p
    for F, sides in enumerate(m.face_elems):
        (e0, f0), (e1, f1) = sides
        assert np.allclose(m.normal[e0, f0], -m.normal[e1, f1], atol=1e-14)
        assert abs(m.face_jac[e0, f0] - m.face_jac[e1, f1]) < 1e-14
        a0 = [m.Nint[e0, a] for a in m.ref.face_nodes[f0]]
        a1 = [m.Nint[e1, a] for a in m.ref.face_nodes[f1]]
        for c in range(m.ref.Nf):
            c0 = np.where(m.fnode_map[e0, f0] == c)[0][0]
            c1 = np.where(m.fnode_map[e1, f1] == c)[0][0]
            d = a0[c0] - a1[c1]                          # copies differ by a period shift
            assert np.all(d % period == 0)
            if c == 0:
                shift = d
            assert np.array_equal(d, shift)
        assert np.array_equal(m.fnode_map[e0, f0], np.arange(m.ref.Nf))
    # divergence theorem per element: sum_f |F| n_F = 0
    pm = 1.0 if dim == 2 else 0.5
    for e in range(m.E):
        assert np.allclose((m.face_jac[e][:, None] * pm * m.normal[e]).sum(0), 0.0, atol=1e-13)


def _golden():
    rows = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            tab, meth, dim, *vals = line.split()
            rows[(tab, meth, int(dim))] = [int(v) for v in vals]
    return rows


@pytest.mark.parametrize("dim", [2, 3])
def test_dof_nnz_tables(dim):
    """Counts on a Kuhn-split periodic mesh reproduce Tables t:dofs and t:nnz exactly."""
    g = _golden()
    n = 4 if dim == 2 else 3
    for k in range(1, 6):
        m = Mesh(dim, n, 0.0, 1.0, k)
        Nv = m.n_vertices
        assert m.trace_dof_hdg() == g[("dof", "HDG", dim)][k - 1] * Nv
        assert m.trace_block_nnz_hdg() == g[("nnz", "HDG", dim)][k - 1] * Nv
        assert m.trace_dof_edg() == g[("dof", "EDG", dim)][k - 1] * Nv
        assert m.trace_nnz_edg() == g[("nnz", "EDG", dim)][k - 1] * Nv
        assert m.dof_dg() == g[("dof", "DG", dim)][k - 1] * Nv
        assert m.nnz_dg() == g[("nnz", "DG", dim)][k - 1] * Nv
