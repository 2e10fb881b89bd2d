"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
symbol include/hdg.h declares, rejects invalid arguments, and its mesh (an independent
C++ implementation of the numbering rules) agrees with the oracle's mesh."""
import os
import re

import numpy as np
import pytest

from oracle.mesh import Mesh as OMesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1808_05066_gb300 import hdg
    return hdg


def test_library_exports_every_declared_symbol():
    hdg = _lib()
    with open(os.path.join(ROOT, "include", "hdg.h")) as fh:
        text = fh.read()
    declared = set(re.findall(r"^\s*(?:int64_t|int|void|const char\*)\s+(hdg_\w+)\s*\(", text, re.M))
    assert declared, "no declarations parsed"
    assert declared == set(hdg.EXPORTED)
    for name in declared:
        assert hasattr(hdg._lib, name), name


def test_invalid_arguments_are_rejected():
    hdg = _lib()
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_mesh_create(2, [0, 4], [0, 0], [1, 1], 2)
    assert ei.value.code == hdg.HDG_ERR_INVALID_ARG
    with pytest.raises(hdg.HdgError):
        hdg.hdg_mesh_create(4, [2, 2, 2], [0, 0, 0], [1, 1, 1], 2)
    with pytest.raises(hdg.HdgError):
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 0)
    with pytest.raises(hdg.HdgError) as ei:     # unknown trace space
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 2, scheme=7)
    assert ei.value.code == hdg.HDG_ERR_INVALID_ARG
    with pytest.raises(hdg.HdgError) as ei:     # a degree outside 1..4 in p_per_elem
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 2, p_per_elem=np.array([2] * 7 + [9], np.int8))
    assert ei.value.code == hdg.HDG_ERR_INVALID_ARG
    with pytest.raises(hdg.HdgError) as ei:     # an axis periodic on one side only
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 2, bc=[("periodic", "state"), ("periodic", "periodic")])
    assert ei.value.code == hdg.HDG_ERR_INVALID_ARG
    with pytest.raises(hdg.HdgError) as ei:     # an unknown boundary type
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 2, bc=[(5, 5), (0, 0)])
    assert ei.value.code == hdg.HDG_ERR_INVALID_ARG
    with pytest.raises(hdg.HdgError) as ei:     # EDG with boundaries takes the given state only
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 2, scheme=hdg.HDG_SCHEME_EDG,
                            bc=[("state", "state"), ("slip", "slip")])
    assert ei.value.code == hdg.HDG_ERR_UNSUPPORTED
    m = hdg.Mesh(2, 2, 0.0, 1.0, 3, bc=[("slip", "slip"), ("periodic", "periodic")])
    with pytest.raises(hdg.HdgError) as ei:     # the slip wall is defined for the Euler equations only
        hdg.hdg_ctx_create(m.handle, 1.4, 0.3, 100.0, 0.72, 0)
    assert ei.value.code == hdg.HDG_ERR_UNSUPPORTED


@pytest.mark.parametrize("dim,n,p", [(2, 3, 2), (2, 2, 4), (3, 2, 3), (3, 1, 2)])
def test_edg_numbering_matches_oracle(dim, n, p):
    """The C++ EDG / IEDG numbering of the skeleton nodes (Sec. 3.4) equals the oracle's, node for
    node, and its size is the oracle's count (Table t:dofs)."""
    from oracle.hdg import Problem
    from oracle import physics as ph
    hdg = _lib()
    o = OMesh(dim, n, 0.0, 2.0, p)
    prob = Problem(o, ph.Physics(), scheme="edg")
    for scheme in (hdg.HDG_SCHEME_EDG, hdg.HDG_SCHEME_IEDG):
        m = hdg.Mesh(dim, n, 0.0, 2.0, p, scheme=scheme)
        assert m.info["scheme"] == scheme and m.info["n_trace_nodes"] == prob.n_edg == o.trace_dof_edg()
        assert m.info["n_trace"] == prob.n_trace
        assert np.array_equal(m.trace_map(), prob.edg_index)
        _, xt, _ = m.coords()
        assert xt.shape == (prob.n_edg, dim)
    # the HDG trace map is face * Nf + canonical node
    h = hdg.Mesh(dim, n, 0.0, 2.0, p)
    assert np.array_equal(h.trace_map(), o.face_of[:, :, None] * o.ref.Nf + o.fnode_map)


@pytest.mark.parametrize("dim,n,p,bc,scheme", [(2, 3, 2, [("state", "state"), ("state", "state")], "iedg"),
                                               (2, 3, 2, [("state", "state"), ("state", "state")], "edg"),
                                               (2, 2, 3, [("periodic", "periodic"), ("state", "state")], "iedg"),
                                               (3, 2, 2, [("state", "state"), ("periodic", "periodic"), ("slip", "slip")],
                                                "iedg"),
                                               (3, 2, 2, [("state", "state"), ("periodic", "periodic"),
                                                          ("state", "state")], "edg")])
def test_iedg_numbering_on_bounded_meshes_matches_oracle(dim, n, p, bc, scheme):
    """On a bounded mesh the C++ IEDG numbering (continuous on the interior faces, each boundary
    face with nodes of its own) and EDG numbering (continuous everywhere; bounded axes not wrapped)
    equal the oracle's node for node, and the trace nodes' coordinates are those of the element
    nodes they copy (up to the period on periodic axes)."""
    from oracle.hdg import Problem
    from oracle import physics as ph
    hdg = _lib()
    o = OMesh(dim, n, 0.0, 2.0, p, bc=bc)
    prob = Problem(o, ph.Physics(), scheme=scheme)
    m = hdg.Mesh(dim, n, 0.0, 2.0, p, scheme=hdg.HDG_SCHEME_IEDG if scheme == "iedg" else hdg.HDG_SCHEME_EDG, bc=bc)
    assert m.info["n_trace_nodes"] == prob.n_edg and m.info["n_trace"] == prob.n_trace
    tmap = m.trace_map()
    assert np.array_equal(tmap, prob.edg_index)
    _, xt, _ = m.coords()
    fn = np.array(o.ref.face_nodes)
    d = xt[tmap] - o.xnode[:, fn, :]
    d = np.where(o.periodic, d - 2.0 * np.round(d / 2.0), d)
    assert np.abs(d).max() <= 1e-13


def test_mixed_degree_variants_that_are_not_built():
    """Meshes of mixed degree are built periodic, HDG, with the default rules; EDG or bounded
    axes with mixed degrees say so with HDG_ERR_UNSUPPORTED, degrees outside 1..4 are invalid."""
    hdg = _lib()
    pe = np.array([2] * 7 + [3], np.int8)
    m = hdg.Mesh(2, 2, 0.0, 1.0, 0, p_per_elem=pe)
    assert m.info["mixed"] == 1 and m.info["p"] == 3 and m.info["p_min"] == 2
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 2, p_per_elem=pe, scheme=hdg.HDG_SCHEME_EDG)
    assert ei.value.code == hdg.HDG_ERR_UNSUPPORTED
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 2, p_per_elem=pe, bc=[("state", "state"), ("periodic", "periodic")])
    assert ei.value.code == hdg.HDG_ERR_UNSUPPORTED
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 2, p_per_elem=np.array([2] * 7 + [5], np.int8))
    assert ei.value.code == hdg.HDG_ERR_INVALID_ARG
    # a per-element array of one degree is the uniform mesh
    m = hdg.Mesh(3, 1, 0.0, 1.0, 2, p_per_elem=np.full(6, 2, np.int8))
    assert m.info["n_elem"] == 6 and m.info["p"] == 2 and m.info["mixed"] == 0


@pytest.mark.parametrize("dim,n,degs", [(3, 1, (1, 2, 3, 4)), (3, 2, (1, 2, 3, 4)), (2, 3, (1, 2, 3))])
def test_mixed_degree_mesh_matches_oracle(dim, n, degs):
    """Face degrees max(p_L, p_R), trace-node numbering, trace map, packed layout and node
    coordinates of the library's mixed-degree mesh against the oracle's."""
    from oracle import physics as ph
    from oracle.hdg import Problem
    from oracle.refel import refel
    hdg = _lib()
    E = (2 * n * n) if dim == 2 else 6 * n ** 3
    pe = np.random.default_rng(4 + n).choice(degs, size=E).astype(np.int8)
    L = 2.5
    m = hdg.Mesh(dim, n, 0.0, L, 0, p_per_elem=pe)
    o = OMesh(dim, n, 0.0, L, 0, p_elem=pe)
    prob = Problem(o, ph.Physics(mach=0.3, reynolds=100.0, prandtl=0.71))
    lay, tn = m.layout(), m.trace_map()
    face_of, _, _ = m.topology()
    assert np.array_equal(face_of, o.face_of)
    assert np.array_equal(lay["elem_p"], pe)
    assert np.array_equal(lay["face_deg"], o.face_deg)
    assert np.array_equal(lay["face_node_off"], o.fnode_off)
    assert m.info["n_trace_nodes"] == o.fnode_off[-1]
    xnode, xfnode, _ = m.coords()
    for e in range(E):
        t = prob.trace_node(e)
        assert np.array_equal(tn[e][:, :t.shape[1]], t)
        assert np.all(tn[e][:, t.shape[1]:] == -1)
        nv, nt = prob.np_e(e) * (dim + 2), int(prob.trace_mask(e).sum())
        assert lay["voff"][e + 1] - lay["voff"][e] == nv and lay["toff"][e + 1] - lay["toff"][e] == nt
        assert lay["soff"][e + 1] - lay["soff"][e] == nt * nt
        assert lay["roff"][e + 1] - lay["roff"][e] == nv * nt + nv
        assert lay["Roff"][e + 1] - lay["Roff"][e] == nv + nt
        a = lay["voff"][e] // (dim + 2)
        assert np.allclose(xnode[a:a + prob.np_e(e)], o.elem_nodes(e), atol=1e-13)
    for F, sides in enumerate(o.face_elems):
        e, f = sides[0]
        r = refel(dim, int(o.face_deg[F]))
        x = o.X[e, 0] + r.nodes[r.face_nodes[f]] @ o.J[e].T
        assert np.allclose(xfnode[o.fnode_off[F]:o.fnode_off[F + 1]], x, atol=1e-13)


_BOUNDED = {2: [("state", "slip"), ("periodic", "periodic")],
            3: [("periodic", "periodic"), ("slip", "slip"), ("state", "state")]}


@pytest.mark.parametrize("bounded", [False, True])
@pytest.mark.parametrize("dim,n,p", [(2, 3, 2), (2, 2, 4), (3, 2, 3), (3, 1, 1), (3, 3, 2)])
def test_mesh_matches_oracle(dim, n, p, bounded):
    """Topology, face types and geometry of the library's mesh against the oracle's, periodic
    and with bounded axes (one-sided faces on the walls)."""
    hdg = _lib()
    L = 2.5
    bc = _BOUNDED[dim] if bounded else None
    m = hdg.Mesh(dim, n, 0.0, L, p, bc=bc)
    o = OMesh(dim, n, 0.0, L, p, bc=bc)
    info = m.info
    assert info["n_elem"] == o.E and info["n_faces"] == o.nFaces
    assert info["Np"] == o.ref.Np and info["Nf"] == o.ref.Nf
    assert info["NG"] == len(o.ref.qw) and info["NGF"] == len(o.ref.fqw)
    assert info["n_boundary_faces"] == int(np.sum(o.face_bc != 0)) and (info["n_boundary_faces"] > 0) == bounded
    face_of, fnode_map, face_side = m.topology()
    assert np.array_equal(face_of, o.face_of)
    assert np.array_equal(fnode_map, o.fnode_map)
    sides = np.array([[e * o.ref.nF + f for (e, f) in s] + [-1] * (2 - len(s)) for s in o.face_elems])
    assert np.array_equal(face_side, sides)
    assert np.array_equal(m.face_bc(), o.face_bc)
    xnode, xfnode, geo = m.coords()
    assert np.allclose(xnode, o.xnode, atol=1e-13)
    d = dim
    assert np.allclose(geo[:, :d * d].reshape(-1, d, d), o.Jinv, atol=1e-12)
    assert np.allclose(geo[:, d * d], np.abs(o.detJ), atol=1e-13)
    for f in range(d + 1):
        base = d * d + 1 + f * (d + 1)
        assert np.allclose(geo[:, base:base + d], o.normal[:, f], atol=1e-13)
        assert np.allclose(geo[:, base + d], o.face_jac[:, f], atol=1e-13)
    for F, sd in enumerate(o.face_elems):
        e, f = sd[0]
        assert np.allclose(xfnode[F], o.xnode[e, o.ref.face_nodes[f]], atol=1e-13)


def test_physics_arguments_are_checked():
    """Invalid physics (power-law exponent outside 0..4, unknown viscous-flux option or
    stabilization matrix) is rejected
    before any device is touched."""
    hdg = _lib()
    m = hdg.Mesh(2, 2, 0.0, 1.0, 2)
    for kw in (dict(mu_exponent=-0.5), dict(mu_exponent=9.0), dict(visc_flux=3),
               dict(stabilization=2)):
        with pytest.raises(hdg.HdgError) as ei:
            hdg.hdg_ctx_create(m.handle, 1.4, 0.3, 100.0, 0.72, 0, **kw)
        assert ei.value.code == hdg.HDG_ERR_INVALID_ARG


@pytest.mark.parametrize("dim,p", [(2, 3), (3, 2), (3, 4)])
def test_layout_of_one_degree_is_the_uniform_stride(dim, p):
    """For a mesh of one degree the packed layout is the uniform one (also for 3D p = 4, which
    runs on the element-class kernels): offsets e * nv, e * nt, e * nt^2, ..., faces of degree p
    with Nf nodes each."""
    hdg = _lib()
    m = hdg.Mesh(dim, 2, 0.0, 1.0, p)
    i, lay = m.info, m.layout()
    E, F, nv, nt, Nf = i["n_elem"], i["n_faces"], i["nv"], i["nt"], i["Nf"]
    e = np.arange(E + 1)
    assert i["mixed"] == 0 and i["p"] == p
    assert np.array_equal(lay["voff"], e * nv) and np.array_equal(lay["toff"], e * nt)
    assert np.array_equal(lay["soff"], e * nt * nt) and np.array_equal(lay["roff"], e * (nv * nt + nv))
    assert np.array_equal(lay["Roff"], e * (nv + nt))
    assert np.all(lay["elem_p"] == p) and np.all(lay["face_deg"] == p)
    assert np.array_equal(lay["face_node_off"], np.arange(F + 1) * Nf)
    assert i["len_S"] == E * nt * nt and i["n_trace_nodes"] == F * Nf
    assert np.array_equal(m.trace_map(), OMesh(dim, 2, 0.0, 1.0, p).face_of[:, :, None] * Nf
                          + OMesh(dim, 2, 0.0, 1.0, p).fnode_map)
