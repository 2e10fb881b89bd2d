"""ctypes binding of include/hdg.h: the same entry points, argument marshalling only.

Device buffers are passed as torch CUDA tensors (or raw integer addresses); streams as
torch.cuda.Stream / raw handles (None = the current torch stream). All numerical work
runs in libhdg.so; if the library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_int32, c_int64, c_void_p

import numpy as np

from . import _build

HDG_OK = 0
HDG_ERR_INVALID_ARG = 1
HDG_ERR_NONPHYSICAL = 2
HDG_ERR_SINGULAR = 3
HDG_ERR_REFINE = 4
HDG_ERR_NOT_CONVERGED = 5
HDG_ERR_TIMEOUT = 6
HDG_ERR_CUDA = 7
HDG_ERR_UNSUPPORTED = 8
HDG_PREC_FP64 = 0
HDG_PREC_MIXED = 1
HDG_SOLVER_AUTO = 0
HDG_SOLVER_GMRES = 1
HDG_SOLVER_DENSE = 2
HDG_SCHEME_HDG = 0
HDG_SCHEME_EDG = 1
HDG_SCHEME_IEDG = 2
HDG_ELEM_NONPHYSICAL = 1
HDG_ELEM_SINGULAR = 2
HDG_ELEM_REFINE = 4
HDG_ELEM_FP64 = 8
HDG_ELEM_TIMEOUT = 16

EXPORTED = [
    "hdg_mesh_create", "hdg_mesh_destroy", "hdg_mesh_get_info", "hdg_mesh_copy_topology",
    "hdg_mesh_copy_coords", "hdg_ctx_create", "hdg_ctx_destroy", "hdg_prim_to_entropy",
    "hdg_history", "hdg_add_source", "hdg_assemble_condense", "hdg_trace_solve", "hdg_recover_interior",
    "hdg_trace_matvec", "hdg_residual_norm", "hdg_newton_step", "hdg_profile_enable",
    "hdg_profile_reset", "hdg_profile_read", "hdg_last_error", "hdg_assemble_condense_noalloc",
    "hdg_mlp_param_count", "hdg_mlp_init", "hdg_mlp_features", "hdg_mlp_forward", "hdg_mlp_gradient",
    "hdg_mlp_train_step", "hdg_mlp_apply_trace", "hdg_mlp_stats", "hdg_mlp_standardize", "hdg_mlp_target",
    "hdg_axpby", "hdg_assemble_condense_host", "hdg_assemble_condense_graph", "hdg_newton_solve",
    "hdg_ctx_set_refinement", "hdg_ctx_graph_replays", "hdg_ctx_set_trace_solver", "hdg_dirk3_step",
    "hdg_entropy_production", "hdg_mesh_copy_trace_map", "hdg_mesh_copy_face_bc", "hdg_ctx_set_boundary_state",
    "hdg_mesh_copy_layout", "hdg_ctx_trace_cycles",
]
HDG_BC_PERIODIC = 0
HDG_BC_STATE = 1
HDG_BC_SLIP = 2
_BC_NAMES = {"periodic": HDG_BC_PERIODIC, "state": HDG_BC_STATE, "slip": HDG_BC_SLIP}
HDG_KERNEL_POINTWISE = 0
HDG_KERNEL_ASSEMBLE = 1
HDG_KERNEL_CONDENSE = 2
HDG_KERNEL_MIXED_ASSEMBLE = 3
HDG_KERNEL_MIXED_CONDENSE = 4
HDG_KERNEL_TRACE = 5
HDG_KERNEL_OTHER = 6
HDG_KERNEL_MIXED_PREP = 7
HDG_KERNEL_MIXED_FACE = 8
HDG_KERNEL_MIXED_OPERATORS = 9
HDG_KERNEL_PCLASS = 10
HDG_KERNEL_CLASSES = 11


class HdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hdg error {code}: {msg}")
        self.code = code


class hdg_physics(ctypes.Structure):
    _fields_ = [("gamma", c_double), ("mach", c_double), ("reynolds", c_double), ("prandtl", c_double),
                ("mu_exponent", c_double), ("visc_flux", c_int32),
                ("stabilization", c_int32)]


class hdg_warmstart(ctypes.Structure):
    _fields_ = [("params", c_void_p), ("nin", c_int), ("nh", c_int), ("nout", c_int),
                ("feat_mean", c_void_p), ("feat_std", c_void_p), ("tmean", c_void_p), ("tscale", c_void_p),
                ("vhat_n", c_void_p), ("dvhat1", c_void_p), ("dvhat2", c_void_p)]


class hdg_mesh_info(ctypes.Structure):
    _fields_ = [("dim", c_int32), ("p", c_int32), ("quad_points", c_int32), ("m", c_int32),
                ("Np", c_int32), ("Nf", c_int32), ("nF", c_int32), ("NG", c_int32), ("NGF", c_int32),
                ("nv", c_int32), ("nt", c_int32), ("geo_stride", c_int32),
                ("n_elem", c_int64), ("n_faces", c_int64), ("n_trace", c_int64),
                ("scheme", c_int32), ("n_trace_nodes", c_int64), ("n_boundary_faces", c_int64),
                ("mixed", c_int32), ("p_min", c_int32), ("len_V", c_int64), ("len_g", c_int64), ("len_S", c_int64),
                ("len_recov", c_int64), ("len_R", c_int64)]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "hdg_mesh_create": (c_int, [c_int, POINTER(c_int64), POINTER(c_double), POINTER(c_double), c_void_p, c_int,
                                    c_int, c_int, c_void_p, POINTER(c_void_p)]),
        "hdg_mesh_copy_face_bc": (c_int, [P, P]),
        "hdg_ctx_set_boundary_state": (c_int, [P, P, P]),
        "hdg_mesh_destroy": (None, [P]),
        "hdg_mesh_get_info": (c_int, [P, POINTER(hdg_mesh_info)]),
        "hdg_mesh_copy_topology": (c_int, [P, P, P, P]),
        "hdg_mesh_copy_coords": (c_int, [P, P, P, P]),
        "hdg_ctx_create": (c_int, [P, POINTER(hdg_physics), c_int, POINTER(c_void_p)]),
        "hdg_ctx_destroy": (None, [P]),
        "hdg_prim_to_entropy": (c_int, [P, P, c_int64, P, P]),
        "hdg_history": (c_int, [P, P, P, c_double, c_double, P, P]),
        "hdg_add_source": (c_int, [P, P, c_double, P, P]),
        "hdg_assemble_condense": (c_int, [P, P, P, P, c_double, c_int, P, P, P, P, P, P]),
        "hdg_trace_solve": (c_int, [P, P, P, P, c_int, c_double, c_int, POINTER(c_int), POINTER(c_double), P]),
        "hdg_recover_interior": (c_int, [P, P, P, P, P]),
        "hdg_trace_matvec": (c_int, [P, P, P, P, P]),
        "hdg_residual_norm": (c_int, [P, P, POINTER(c_double), P]),
        "hdg_newton_solve": (c_int, [P, P, P, P, c_double, c_int, c_double, c_int, POINTER(c_int),
                                     POINTER(c_double), POINTER(c_double), POINTER(c_int), P]),
        "hdg_newton_step": (c_int, [P, P, P, P, P, c_double, c_int, c_int, c_double, c_int, POINTER(hdg_warmstart),
                                    POINTER(c_int), POINTER(c_double), POINTER(c_double), POINTER(c_int), P]),
        "hdg_ctx_set_refinement": (c_int, [P, c_double, c_int]),
        "hdg_ctx_graph_replays": (c_int, [P, POINTER(c_int64)]),
        "hdg_ctx_trace_cycles": (c_int, [P, POINTER(c_int64), POINTER(c_int64)]),
        "hdg_ctx_set_trace_solver": (c_int, [P, c_int, c_double, c_int]),
        "hdg_entropy_production": (c_int, [P, P, P, POINTER(c_double), POINTER(c_double), P]),
        "hdg_mesh_copy_trace_map": (c_int, [P, P]),
        "hdg_mesh_copy_layout": (c_int, [P, P, P, P, P, P, P, P, P]),
        "hdg_dirk3_step": (c_int, [P, P, P, P, c_double, c_int, c_double, c_int, POINTER(c_int), POINTER(c_double),
                                   POINTER(c_int), P]),
        "hdg_mlp_param_count": (c_int64, [c_int, c_int, c_int]),
        "hdg_mlp_init": (c_int, [P, c_int, c_int, c_int, ctypes.c_uint64, P]),
        "hdg_mlp_features": (c_int, [P, P, P, P, P, P, P, P, P]),
        "hdg_mlp_forward": (c_int, [P, c_int, c_int, c_int, P, c_int64, P, P]),
        "hdg_mlp_gradient": (c_int, [P, P, c_int, c_int, c_int, P, P, c_int64, P, P]),
        "hdg_mlp_train_step": (c_int, [P, P, c_int, c_int, c_int, P, P, c_int64, ctypes.c_float, c_int, P, P]),
        "hdg_mlp_apply_trace": (c_int, [P, P, P, P, P, P, P, P]),
        "hdg_mlp_stats": (c_int, [P, c_int64, c_int, P, P, P]),
        "hdg_mlp_standardize": (c_int, [P, c_int64, c_int, P, P, P]),
        "hdg_mlp_target": (c_int, [c_int64, P, P, P, P, P]),
        "hdg_axpby": (c_int, [c_int64, c_double, P, c_double, P, P, P]),
        "hdg_profile_enable": (c_int, [P, c_int]),
        "hdg_profile_reset": (c_int, [P]),
        "hdg_profile_read": (c_int, [P, c_int, POINTER(c_int64), POINTER(c_double)]),
        "hdg_last_error": (ctypes.c_char_p, []),
        "hdg_assemble_condense_noalloc": (c_int, [P, P, P, P, c_double, P, P, P, P, P, P]),
        "hdg_assemble_condense_host": (c_int, [P, P, P, P, c_double, c_int, P, P, P, P, P, P]),
        "hdg_assemble_condense_graph": (c_int, [P, P, P, P, c_double, c_int, P, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
LIB_PATH = _build.LIB


def _check(code):
    if code != HDG_OK:
        raise HdgError(code, _lib.hdg_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------------ raw entry points
def _bc_array(dim, bc):
    """None, or per axis a pair (lo, hi) of HDG_BC_* codes or names -> int32 [2 dim]."""
    if bc is None:
        return None
    out = [(_BC_NAMES[s] if isinstance(s, str) else int(s)) for pair in bc for s in pair]
    if len(out) != 2 * dim:
        raise ValueError("bc: one (lo, hi) pair per axis")
    return np.array(out, dtype=np.int32)


def hdg_mesh_create(dim, n, lo, hi, p, quad_points=0, p_per_elem=None, scheme=HDG_SCHEME_HDG, bc=None):
    """p_per_elem: None (uniform p) or an int8 array [E] of per-element degrees; bc: None (periodic)
    or per axis a (lo, hi) pair of boundary types ("periodic", "state", "slip" or HDG_BC_*)."""
    n3 = (c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    lo3 = (c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
    hi3 = (c_double * 3)(*(list(hi) + [1.0] * (3 - len(hi))))
    pe = None if p_per_elem is None else np.ascontiguousarray(p_per_elem, dtype=np.int8)
    bca = _bc_array(dim, bc)
    h = c_void_p()
    _check(_lib.hdg_mesh_create(dim, n3, lo3, hi3, _ptr(pe), p, scheme, quad_points, _ptr(bca), byref(h)))
    return h.value


def hdg_mesh_copy_face_bc(mesh):
    i = hdg_mesh_get_info(mesh)
    out = np.zeros(i["n_faces"], np.int8)
    _check(_lib.hdg_mesh_copy_face_bc(mesh, _ptr(out)))
    return out


def hdg_ctx_set_boundary_state(ctx, Vb, stream=None):
    """Vb: device tensor in the trace layout [F][Nf][m] (read on the HDG_BC_STATE faces)."""
    _check(_lib.hdg_ctx_set_boundary_state(ctx, _ptr(Vb), _stream(stream)))


def hdg_mesh_destroy(mesh):
    _lib.hdg_mesh_destroy(mesh)


def hdg_mesh_get_info(mesh):
    info = hdg_mesh_info()
    _check(_lib.hdg_mesh_get_info(mesh, byref(info)))
    return {k: getattr(info, k) for k, _ in hdg_mesh_info._fields_}


def hdg_mesh_copy_topology(mesh):
    i = hdg_mesh_get_info(mesh)
    face_of = np.zeros((i["n_elem"], i["nF"]), np.int32)
    fnode_map = np.zeros((i["n_elem"], i["nF"], i["Nf"]), np.int32)
    face_side = np.zeros((i["n_faces"], 2), np.int32)
    _check(_lib.hdg_mesh_copy_topology(mesh, _ptr(face_of), _ptr(fnode_map), _ptr(face_side)))
    return face_of, fnode_map, face_side


def hdg_mesh_copy_trace_map(mesh):
    i = hdg_mesh_get_info(mesh)
    tnode = np.zeros((i["n_elem"], i["nF"], i["Nf"]), np.int32)
    _check(_lib.hdg_mesh_copy_trace_map(mesh, _ptr(tnode)))
    return tnode


def hdg_mesh_copy_layout(mesh):
    """Packed per-element layout: dict of offsets [E + 1] (voff, toff, soff, roff, Roff), elem_p [E],
    face_deg [F], face_node_off [F + 1] (host arrays)."""
    i = hdg_mesh_get_info(mesh)
    E, F = i["n_elem"], i["n_faces"]
    out = {k: np.zeros(E + 1, np.int64) for k in ("voff", "toff", "soff", "roff", "Roff")}
    out["elem_p"] = np.zeros(E, np.int8)
    out["face_deg"] = np.zeros(F, np.int8)
    out["face_node_off"] = np.zeros(F + 1, np.int64)
    _check(_lib.hdg_mesh_copy_layout(mesh, *[_ptr(out[k]) for k in ("voff", "toff", "soff", "roff", "Roff", "elem_p",
                                                                     "face_deg", "face_node_off")]))
    return out


def hdg_mesh_copy_coords(mesh):
    """(xnode [E][Np][dim], trace-node coordinates ([F][Nf][dim] HDG, [N][dim] EDG), geo)."""
    i = hdg_mesh_get_info(mesh)
    if i["mixed"]:   # packed: element nodes at each element's degree, trace nodes at each face's
        xnode = np.zeros((i["len_V"] // i["m"], i["dim"]))
        xfnode = np.zeros((i["n_trace_nodes"], i["dim"]))
        geo = np.zeros((i["n_elem"], i["geo_stride"]))
        _check(_lib.hdg_mesh_copy_coords(mesh, _ptr(xnode), _ptr(xfnode), _ptr(geo)))
        return xnode, xfnode, geo
    xnode = np.zeros((i["n_elem"], i["Np"], i["dim"]))
    if i["scheme"] == HDG_SCHEME_HDG:
        xfnode = np.zeros((i["n_faces"], i["Nf"], i["dim"]))
    else:
        xfnode = np.zeros((i["n_trace_nodes"], i["dim"]))
    geo = np.zeros((i["n_elem"], i["geo_stride"]))
    _check(_lib.hdg_mesh_copy_coords(mesh, _ptr(xnode), _ptr(xfnode), _ptr(geo)))
    return xnode, xfnode, geo


def hdg_ctx_create(mesh, gamma=1.4, mach=0.5, reynolds=0.0, prandtl=0.71, device=0, mu_exponent=0.0, visc_flux=2,
                   stabilization=0):
    ph = hdg_physics(gamma, mach, reynolds, prandtl, mu_exponent, visc_flux, stabilization)
    h = c_void_p()
    _check(_lib.hdg_ctx_create(mesh, byref(ph), device, byref(h)))
    return h.value


def hdg_ctx_destroy(ctx):
    _lib.hdg_ctx_destroy(ctx)


def hdg_prim_to_entropy(ctx, prim, n_points, v, stream=None):
    _check(_lib.hdg_prim_to_entropy(ctx, _ptr(prim), n_points, _ptr(v), _stream(stream)))


def hdg_history(ctx, V0, V1, c0, c1, hist, stream=None):
    _check(_lib.hdg_history(ctx, _ptr(V0), _ptr(V1), c0, c1, _ptr(hist), _stream(stream)))


def hdg_add_source(ctx, src, c, hist, stream=None):
    _check(_lib.hdg_add_source(ctx, _ptr(src), c, _ptr(hist), _stream(stream)))


def hdg_assemble_condense(ctx, V, Vhat, hist, mass_coef, precision, S, g, recov, R, elem_status=None,
                          stream=None):
    _check(_lib.hdg_assemble_condense(ctx, _ptr(V), _ptr(Vhat), _ptr(hist), mass_coef, precision, _ptr(S),
                                      _ptr(g), _ptr(recov), _ptr(R), _ptr(elem_status), _stream(stream)))


def hdg_assemble_condense_graph(ctx, V, Vhat, hist, mass_coef, precision, S, g, recov, R, elem_status=None,
                                stream=None):
    """hdg_assemble_condense replayed as a CUDA graph after its first call with these arguments."""
    _check(_lib.hdg_assemble_condense_graph(ctx, _ptr(V), _ptr(Vhat), _ptr(hist), mass_coef, precision, _ptr(S),
                                            _ptr(g), _ptr(recov), _ptr(R), _ptr(elem_status), _stream(stream)))


def hdg_assemble_condense_host(ctx, V, Vhat, hist, mass_coef, precision, S_host, g_host, recov, R,
                               elem_status=None, stream=None):
    """hdg_assemble_condense with S and g written to host memory (S_host, g_host: CPU tensors,
    pinned for the copies to overlap the kernels); complete once the stream is synchronised."""
    _check(_lib.hdg_assemble_condense_host(ctx, _ptr(V), _ptr(Vhat), _ptr(hist), mass_coef, precision,
                                           _ptr(S_host), _ptr(g_host), _ptr(recov), _ptr(R), _ptr(elem_status),
                                           _stream(stream)))


def hdg_assemble_condense_noalloc(ctx, V, Vhat, hist, mass_coef, S, g, recov, R, elem_status, stream=None):
    """FP64 assemble + condense that allocates no device memory (scratch in a static
    64 MiB device array); for callers that cannot allocate during the call."""
    _check(_lib.hdg_assemble_condense_noalloc(ctx, _ptr(V), _ptr(Vhat), _ptr(hist), mass_coef, _ptr(S), _ptr(g),
                                              _ptr(recov), _ptr(R), _ptr(elem_status), _stream(stream)))


def hdg_entropy_production(ctx, V, Vhat, stream=None):
    """(int rho s, physical entropy production) of Eq. PiS from (v_h, q_h)."""
    a, b = c_double(), c_double()
    _check(_lib.hdg_entropy_production(ctx, _ptr(V), _ptr(Vhat), byref(a), byref(b), _stream(stream)))
    return a.value, b.value


def hdg_trace_solve(ctx, S, g, dVhat, method=HDG_SOLVER_AUTO, rtol=1e-12, max_it=600, stream=None):
    it = c_int()
    res = c_double()
    _check(_lib.hdg_trace_solve(ctx, _ptr(S), _ptr(g), _ptr(dVhat), method, rtol, max_it, byref(it), byref(res),
                                _stream(stream)))
    return it.value, res.value


def hdg_recover_interior(ctx, recov, dVhat, dV, stream=None):
    _check(_lib.hdg_recover_interior(ctx, _ptr(recov), _ptr(dVhat), _ptr(dV), _stream(stream)))


def hdg_trace_matvec(ctx, S, x, y, stream=None):
    _check(_lib.hdg_trace_matvec(ctx, _ptr(S), _ptr(x), _ptr(y), _stream(stream)))


def hdg_residual_norm(ctx, R, stream=None):
    out = c_double()
    _check(_lib.hdg_residual_norm(ctx, _ptr(R), byref(out), _stream(stream)))
    return out.value


def hdg_newton_solve(ctx, V, Vhat, hist, mass_coef, precision=HDG_PREC_FP64, tol=1e-10, max_newton=10,
                     stream=None, history=False):
    """Returns (updates, final residual norm) or, with history=True,
    (updates, final norm, residual norms before each update, trace-solver iterations)."""
    it = c_int()
    res = c_double()
    hist_buf = (c_double * (max_newton + 1))()
    tr = c_int()
    _check(_lib.hdg_newton_solve(ctx, _ptr(V), _ptr(Vhat), _ptr(hist), mass_coef, precision, tol, max_newton,
                                 byref(it), byref(res), hist_buf, byref(tr), _stream(stream)))
    if history:
        return it.value, res.value, list(hist_buf)[:it.value + 1], tr.value
    return it.value, res.value


def make_warmstart(vhat_n, dvhat1, dvhat2, net=None):
    """hdg_warmstart from device tensors; net: object with params, nin, nh, nout, fmean, fstd,
    tmean, tstd (None: the element-local start alone)."""
    w = hdg_warmstart()
    w.vhat_n, w.dvhat1, w.dvhat2 = _ptr(vhat_n), _ptr(dvhat1), _ptr(dvhat2)
    if net is not None:
        w.params = _ptr(net.params)
        w.nin, w.nh, w.nout = net.nin, net.nh, net.nout
        w.feat_mean, w.feat_std = _ptr(net.fmean), _ptr(net.fstd)
        w.tmean, w.tscale = _ptr(net.tmean), _ptr(net.tstd)
    return w


def hdg_newton_step(ctx, V, Vhat, V_n, V_nm1, dt, bdf_order, precision=HDG_PREC_FP64, tol=1e-10, max_newton=10,
                    warmstart=None, stream=None, history=False):
    """One BDF time step (bdf_order 0, 1, 2) from the initial guess (V, Vhat), updated in place.
    warmstart: an hdg_warmstart (make_warmstart) or None. Returns as hdg_newton_solve."""
    it = c_int()
    res = c_double()
    hist_buf = (c_double * (max_newton + 1))()
    tr = c_int()
    _check(_lib.hdg_newton_step(ctx, _ptr(V), _ptr(Vhat), _ptr(V_n), _ptr(V_nm1), dt, bdf_order, precision, tol,
                                max_newton, None if warmstart is None else byref(warmstart), byref(it), byref(res),
                                hist_buf, byref(tr), _stream(stream)))
    if history:
        return it.value, res.value, list(hist_buf)[:it.value + 1], tr.value
    return it.value, res.value


def hdg_dirk3_step(ctx, V, Vhat, V_n, dt, precision=HDG_PREC_FP64, tol=1e-10, max_newton=10, stream=None):
    """One DIRK(3,3) step; (V, Vhat) in: first stage's guess, out: level n+1.
    Returns (Newton updates per stage [3], final residual norm, trace-solver iterations)."""
    its = (c_int * 3)()
    res = c_double()
    tr = c_int()
    _check(_lib.hdg_dirk3_step(ctx, _ptr(V), _ptr(Vhat), _ptr(V_n), dt, precision, tol, max_newton, its, byref(res),
                               byref(tr), _stream(stream)))
    return list(its), res.value, tr.value


def hdg_ctx_set_refinement(ctx, tol=1e-10, fp64_fallback=True):
    _check(_lib.hdg_ctx_set_refinement(ctx, tol, 1 if fp64_fallback else 0))


def hdg_ctx_set_trace_solver(ctx, method=HDG_SOLVER_AUTO, rtol=1e-12, max_it=600):
    """rtol = 0: inexact Newton (Eisenstat-Walker forcing terms)."""
    _check(_lib.hdg_ctx_set_trace_solver(ctx, method, rtol, max_it))


def hdg_ctx_graph_replays(ctx):
    n = c_int64()
    _check(_lib.hdg_ctx_graph_replays(ctx, byref(n)))
    return n.value


def hdg_ctx_trace_cycles(ctx):
    """(GMRES restart cycles so far, of them replayed as a CUDA graph)."""
    c, r = c_int64(), c_int64()
    _check(_lib.hdg_ctx_trace_cycles(ctx, byref(c), byref(r)))
    return c.value, r.value


def hdg_axpby(n, a, x, b, y, out, stream=None):
    _check(_lib.hdg_axpby(n, a, _ptr(x), b, _ptr(y), _ptr(out), _stream(stream)))


def hdg_mlp_param_count(nin, nh, nout):
    return int(_lib.hdg_mlp_param_count(nin, nh, nout))


def hdg_mlp_init(params, nin, nh, nout, seed, stream=None):
    _check(_lib.hdg_mlp_init(_ptr(params), nin, nh, nout, seed, _stream(stream)))


def hdg_mlp_features(ctx, V, Vhat, dvhat1, dvhat2, mean, std, feat, stream=None):
    _check(_lib.hdg_mlp_features(ctx, _ptr(V), _ptr(Vhat), _ptr(dvhat1), _ptr(dvhat2), _ptr(mean), _ptr(std),
                                 _ptr(feat), _stream(stream)))


def hdg_mlp_stats(x, B, n, mean, std, stream=None):
    _check(_lib.hdg_mlp_stats(_ptr(x), B, n, _ptr(mean), _ptr(std), _stream(stream)))


def hdg_mlp_standardize(x, B, n, mean, std, stream=None):
    _check(_lib.hdg_mlp_standardize(_ptr(x), B, n, _ptr(mean), _ptr(std), _stream(stream)))


def hdg_mlp_target(n, vhat_next, vhat, dvhat1, out, stream=None):
    _check(_lib.hdg_mlp_target(n, _ptr(vhat_next), _ptr(vhat), _ptr(dvhat1), _ptr(out), _stream(stream)))


def hdg_mlp_forward(params, nin, nh, nout, x, B, y, stream=None):
    _check(_lib.hdg_mlp_forward(_ptr(params), nin, nh, nout, _ptr(x), B, _ptr(y), _stream(stream)))


def hdg_mlp_gradient(params, grad, nin, nh, nout, x, target, B, loss, stream=None):
    _check(_lib.hdg_mlp_gradient(_ptr(params), _ptr(grad), nin, nh, nout, _ptr(x), _ptr(target), B, _ptr(loss),
                                 _stream(stream)))


def hdg_mlp_train_step(params, grad, nin, nh, nout, x, target, B, lr, step, loss, stream=None):
    _check(_lib.hdg_mlp_train_step(_ptr(params), _ptr(grad), nin, nh, nout, _ptr(x), _ptr(target), B, lr, step,
                                   _ptr(loss), _stream(stream)))


def hdg_mlp_apply_trace(ctx, Vhat, dvhat1, pred, tmean, tscale, Vhat_out, stream=None):
    _check(_lib.hdg_mlp_apply_trace(ctx, _ptr(Vhat), _ptr(dvhat1), _ptr(pred), _ptr(tmean), _ptr(tscale),
                                    _ptr(Vhat_out), _stream(stream)))


def hdg_profile_enable(ctx, on=True):
    _check(_lib.hdg_profile_enable(ctx, 1 if on else 0))


def hdg_profile_reset(ctx):
    _check(_lib.hdg_profile_reset(ctx))


def hdg_profile_read(ctx, kernel_class=-1):
    n = c_int64()
    ms = c_double()
    _check(_lib.hdg_profile_read(ctx, kernel_class, byref(n), byref(ms)))
    return n.value, ms.value


# ------------------------------------------------------------------ thin owners
class Mesh:
    """Owns an hdg_mesh_t; exposes its info and host copies of its tables."""

    def __init__(self, dim, n, lo, hi, p, quad_points=0, p_per_elem=None, scheme=HDG_SCHEME_HDG, bc=None):
        n = [n] * dim if np.isscalar(n) else list(n)
        lo = [lo] * dim if np.isscalar(lo) else list(lo)
        hi = [hi] * dim if np.isscalar(hi) else list(hi)
        self.handle = hdg_mesh_create(dim, n, lo, hi, p, quad_points, p_per_elem, scheme, bc)
        self.info = hdg_mesh_get_info(self.handle)

    def topology(self):
        return hdg_mesh_copy_topology(self.handle)

    def face_bc(self):
        return hdg_mesh_copy_face_bc(self.handle)

    def trace_map(self):
        return hdg_mesh_copy_trace_map(self.handle)

    def layout(self):
        return hdg_mesh_copy_layout(self.handle)

    def coords(self):
        return hdg_mesh_copy_coords(self.handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            hdg_mesh_destroy(h)
            self.handle = None


class Context:
    """Owns an hdg_ctx_t bound to a Mesh (kept alive by this object)."""

    def __init__(self, mesh: Mesh, gamma=1.4, mach=0.5, reynolds=0.0, prandtl=0.71, device=0, mu_exponent=0.0,
                 visc_flux=2, stabilization=0):
        self.mesh = mesh
        self.handle = hdg_ctx_create(mesh.handle, gamma, mach, reynolds, prandtl, device, mu_exponent, visc_flux,
                                     stabilization)
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            hdg_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()
