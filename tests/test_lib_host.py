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
    with pytest.raises(hdg.HdgError) as ei:     # boundaries are built for the HDG trace space only
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 2, scheme=hdg.HDG_SCHEME_EDG,
                            bc=[("state", "state"), ("periodic", "periodic")])
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


def test_unbuilt_variants_are_reported():
    """The boundary's argument for meshes of mixed degree exists; such meshes are not built and
    say so with HDG_ERR_UNSUPPORTED."""
    hdg = _lib()
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_mesh_create(2, [2, 2], [0, 0], [1, 1], 2, p_per_elem=np.array([2] * 7 + [3], np.int8))
    assert ei.value.code == hdg.HDG_ERR_UNSUPPORTED
    # a per-element array of one degree is the uniform mesh
    m = hdg.Mesh(3, 1, 0.0, 1.0, 2, p_per_elem=np.full(6, 2, np.int8))
    assert m.info["n_elem"] == 6 and m.info["p"] == 2


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
