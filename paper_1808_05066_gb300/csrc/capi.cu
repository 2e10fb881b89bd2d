// C-ABI entry points (include/hdg.h): argument checks, context set-up, device table
// upload, and the Newton-step driver. All numerical work runs in the kernels of
// assemble_fp64.cu, assemble_mixed.cu and trace.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.hpp"

namespace hdg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t err, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(err);
  return HDG_ERR_CUDA;
}

}  // namespace hdg

using hdg::set_error;

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

template <class T>
int upload(T** dst, const std::vector<T>& src) {
  HDG_CK(cudaMalloc(dst, sizeof(T) * std::max<size_t>(1, src.size())));
  if (!src.empty()) HDG_CK(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return HDG_OK;
}

}  // namespace

namespace hdg {

double* chunk_S(hdg_ctx* c, double* S, int64_t e0, cudaStream_t s, int* rc) {
  *rc = HDG_OK;
  if (!c->sink_host) return S;
  const size_t per = (size_t)c->NT * c->NT;
  if (c->Sbuf_chunk < c->chunk) {  // first use, or a larger chunk: (re)allocate the ring
    cudaStreamSynchronize(c->copy_stream);
    for (double*& b : c->d_Sbuf) {
      if (b) cudaFree(b);
      b = nullptr;
    }
    c->Sbuf_chunk = 0;
    for (int k = 0; k < c->sink_bufs; ++k) {
      double*& b = c->d_Sbuf[k];
      if (cudaMalloc(&b, sizeof(double) * per * c->chunk) != cudaSuccess) {
        set_error("hdg_assemble_condense_host: cannot allocate the chunk buffers of S");
        *rc = HDG_ERR_CUDA;
        return nullptr;
      }
    }
    c->Sbuf_chunk = c->chunk;
  }
  const int b = c->sink_idx % c->sink_bufs;
  if (c->sink_idx >= c->sink_bufs && cudaStreamWaitEvent(s, c->ev_copied[b], 0) != cudaSuccess) {  // copied out
    *rc = HDG_ERR_CUDA;
    return nullptr;
  }
  // the kernels index S by the global element: shift the buffer's address by e0 elements
  return reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(c->d_Sbuf[b]) - (uintptr_t)(e0 * per * sizeof(double)));
}

int chunk_done(hdg_ctx* c, int64_t e0, int64_t ne, cudaStream_t s) {
  if (!c->sink_host) return HDG_OK;
  const int b = c->sink_idx % c->sink_bufs;
  const size_t per = (size_t)c->NT * c->NT;
  HDG_CK(cudaEventRecord(c->ev_done[b], s));
  HDG_CK(cudaStreamWaitEvent(c->copy_stream, c->ev_done[b], 0));
  HDG_CK(cudaMemcpyAsync(c->sink_host + e0 * per, c->d_Sbuf[b], sizeof(double) * per * ne, cudaMemcpyDeviceToHost,
                         c->copy_stream));
  HDG_CK(cudaEventRecord(c->ev_copied[b], c->copy_stream));
  ++c->sink_idx;
  return HDG_OK;
}

}  // namespace hdg

extern "C" {

const char* hdg_last_error(void) { return hdg::g_last_error.c_str(); }

int hdg_mesh_create(int dim, const int64_t n[3], const double lo[3], const double hi[3], const int8_t* p_per_elem,
                    int p, int scheme, int quad_points, const int32_t* bc, hdg_mesh_t* out) {
  if (!out || !n || !lo || !hi) {
    set_error("hdg_mesh_create: null argument");
    return HDG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (scheme != HDG_SCHEME_HDG && scheme != HDG_SCHEME_EDG && scheme != HDG_SCHEME_IEDG) {
    set_error("hdg_mesh_create: unknown scheme");
    return HDG_ERR_INVALID_ARG;
  }
  bool mixed = false;
  if (p_per_elem) {  // one degree per element; all equal: the uniform mesh of that degree
    if (dim < 2 || dim > 3) {
      set_error("hdg_mesh_create: invalid mesh arguments");
      return HDG_ERR_INVALID_ARG;
    }
    int64_t E = dim == 2 ? 2 : 6;
    for (int d = 0; d < dim; ++d) E *= n[d] > 0 ? n[d] : 0;
    int pmin = 99, pmax = 0;
    for (int64_t e = 0; e < E; ++e) {
      if (p_per_elem[e] < 1 || p_per_elem[e] > 4) {
        set_error("hdg_mesh_create: element degrees must lie in 1..4");
        return HDG_ERR_INVALID_ARG;
      }
      pmin = std::min<int>(pmin, p_per_elem[e]);
      pmax = std::max<int>(pmax, p_per_elem[e]);
    }
    if (E > 0) p = pmax;
    mixed = pmin != pmax;
    if (mixed) {
      bool periodic = true;
      for (int d = 0; bc && d < 2 * dim; ++d) periodic = periodic && bc[d] == HDG_BC_PERIODIC;
      if (scheme != HDG_SCHEME_HDG || !periodic || (quad_points != 0 && quad_points != p + 1)) {
        set_error("hdg_mesh_create: meshes of mixed degree are built periodic, HDG, with the default rules");
        return HDG_ERR_UNSUPPORTED;
      }
    }
  }
  bool slip = false;
  for (int d = 0; bc && d < 2 * dim && d < 6; ++d) slip = slip || bc[d] == HDG_BC_SLIP;
  if (slip && scheme == HDG_SCHEME_EDG) {
    // an EDG node on the boundary is shared with interior faces: the given state is imposed
    // strongly there; the slip wall is built for the HDG and IEDG trace spaces
    set_error("hdg_mesh_create: EDG with boundaries takes the given state (HDG_BC_STATE) only");
    return HDG_ERR_UNSUPPORTED;
  }
  if (quad_points == 0) quad_points = p + 1;
  auto* m = new hdg_mesh();
  int rc = hdg::build_mesh(dim, n, lo, hi, p, quad_points, m->m, bc);
  if (rc != 0) {
    delete m;
    set_error("hdg_mesh_create: invalid mesh arguments (code " + std::to_string(rc) + ")");
    return HDG_ERR_INVALID_ARG;
  }
  m->m.scheme = scheme;
  // IEDG differs from EDG only on a bounded mesh (on a periodic one every face is interior)
  if (scheme != HDG_SCHEME_HDG) hdg::build_edg(m->m, scheme == HDG_SCHEME_IEDG);
  // 3D p = 4 has no uniform kernels: a periodic HDG mesh of that one degree is served by the
  // element-class kernels too (its packed layout is the uniform one)
  bool periodic = true;
  for (int d = 0; bc && d < 2 * dim; ++d) periodic = periodic && bc[d] == HDG_BC_PERIODIC;
  std::vector<int8_t> all4;
  const int8_t* pe = p_per_elem;
  if (!mixed && dim == 3 && p == 4 && scheme == HDG_SCHEME_HDG && periodic && quad_points == p + 1) {
    all4.assign(m->m.E, (int8_t)4);
    pe = all4.data();
    mixed = true;
  }
  if (mixed && (rc = hdg::build_mixed(m->m, pe)) != 0) {
    delete m;
    set_error("hdg_mesh_create: mixed-degree face matching failed (code " + std::to_string(rc) + ")");
    return HDG_ERR_INVALID_ARG;
  }
  *out = m;
  return HDG_OK;
}

void hdg_mesh_destroy(hdg_mesh_t mesh) { delete mesh; }

int hdg_mesh_get_info(hdg_mesh_t mesh, hdg_mesh_info* out) {
  if (!mesh || !out) {
    set_error("hdg_mesh_get_info: null argument");
    return HDG_ERR_INVALID_ARG;
  }
  const hdg::Mesh& m = mesh->m;
  out->dim = m.dim;
  out->p = m.p;
  out->quad_points = m.K;
  out->m = m.dim + 2;
  out->Np = m.ref.Np;
  out->Nf = m.ref.Nf;
  out->nF = m.ref.nF;
  out->NG = m.ref.NG;
  out->NGF = m.ref.NGF;
  out->nv = m.ref.Np * (m.dim + 2);
  out->nt = m.ref.nF * m.ref.Nf * (m.dim + 2);
  out->geo_stride = m.geo_stride;
  out->n_elem = m.E;
  out->n_faces = m.nFaces;
  out->scheme = m.scheme;
  out->n_trace_nodes = m.scheme == HDG_SCHEME_HDG ? m.nFaces * m.ref.Nf : m.n_edg;
  out->n_trace = out->n_trace_nodes * (m.dim + 2);
  out->n_boundary_faces = m.n_boundary;
  out->mixed = 0;
  if (!m.pe.empty()) {
    out->p_min = *std::min_element(m.pe.begin(), m.pe.end());
    out->mixed = out->p_min != m.p ? 1 : 0;
    out->n_trace_nodes = m.fnoff.back();
    out->n_trace = out->n_trace_nodes * (m.dim + 2);
    out->len_V = m.voff.back();
    out->len_g = m.toff.back();
    out->len_S = m.soff.back();
    out->len_recov = m.roff.back();
    out->len_R = m.Roff.back();
  } else {
    out->p_min = m.p;
    out->len_V = m.E * out->nv;
    out->len_g = m.E * out->nt;
    out->len_S = m.E * (int64_t)out->nt * out->nt;
    out->len_recov = m.E * ((int64_t)out->nv * out->nt + out->nv);
    out->len_R = m.E * (int64_t)(out->nv + out->nt);
  }
  return HDG_OK;
}

int hdg_mesh_copy_layout(hdg_mesh_t mesh, int64_t* voff, int64_t* toff, int64_t* soff, int64_t* roff, int64_t* Roff,
                         int8_t* elem_p, int8_t* face_deg, int64_t* face_node_off) {
  if (!mesh) {
    set_error("hdg_mesh_copy_layout: null mesh");
    return HDG_ERR_INVALID_ARG;
  }
  const hdg::Mesh& m = mesh->m;
  const int M = m.dim + 2;
  const int64_t nv = (int64_t)m.ref.Np * M, nt = (int64_t)m.ref.nF * m.ref.Nf * M;
  const bool mx = !m.pe.empty();
  for (int64_t e = 0; e <= m.E; ++e) {
    if (voff) voff[e] = mx ? m.voff[e] : e * nv;
    if (toff) toff[e] = mx ? m.toff[e] : e * nt;
    if (soff) soff[e] = mx ? m.soff[e] : e * nt * nt;
    if (roff) roff[e] = mx ? m.roff[e] : e * (nv * nt + nv);
    if (Roff) Roff[e] = mx ? m.Roff[e] : e * (nv + nt);
    if (elem_p && e < m.E) elem_p[e] = mx ? m.pe[e] : (int8_t)m.p;
  }
  for (int64_t F = 0; F <= m.nFaces; ++F) {
    if (face_deg && F < m.nFaces) face_deg[F] = mx ? m.fdeg[F] : (int8_t)m.p;
    if (face_node_off) face_node_off[F] = mx ? m.fnoff[F] : F * m.ref.Nf;
  }
  return HDG_OK;
}

int hdg_mesh_copy_face_bc(hdg_mesh_t mesh, int8_t* face_bc) {
  if (!mesh || !face_bc) {
    set_error("hdg_mesh_copy_face_bc: null argument");
    return HDG_ERR_INVALID_ARG;
  }
  std::memcpy(face_bc, mesh->m.face_bc.data(), mesh->m.face_bc.size());
  return HDG_OK;
}

int hdg_mesh_copy_trace_map(hdg_mesh_t mesh, int32_t* tnode) {
  if (!mesh || !tnode) {
    set_error("hdg_mesh_copy_trace_map: null argument");
    return HDG_ERR_INVALID_ARG;
  }
  const hdg::Mesh& m = mesh->m;
  const int nF = m.ref.nF, Nf = m.ref.Nf;
  for (int64_t e = 0; e < m.E; ++e)
    for (int f = 0; f < nF; ++f)
      for (int c = 0; c < Nf; ++c) {
        const int64_t i = (e * nF + f) * Nf + c;
        if (!m.pe.empty())
          tnode[i] = m.fnode_mix[i] < 0 ? -1 : (int32_t)(m.fnoff[m.face_of[e * nF + f]] + m.fnode_mix[i]);
        else
          tnode[i] = m.scheme == HDG_SCHEME_HDG ? m.face_of[e * nF + f] * Nf + m.fnode_map[i] : m.edg_index[i];
      }
  return HDG_OK;
}

int hdg_mesh_copy_topology(hdg_mesh_t mesh, int32_t* face_of, int32_t* fnode_map, int32_t* face_side) {
  if (!mesh) {
    set_error("hdg_mesh_copy_topology: null mesh");
    return HDG_ERR_INVALID_ARG;
  }
  const hdg::Mesh& m = mesh->m;
  if (face_of) std::memcpy(face_of, m.face_of.data(), sizeof(int32_t) * m.face_of.size());
  if (fnode_map) std::memcpy(fnode_map, m.fnode_map.data(), sizeof(int32_t) * m.fnode_map.size());
  if (face_side) std::memcpy(face_side, m.face_side.data(), sizeof(int32_t) * m.face_side.size());
  return HDG_OK;
}

int hdg_mesh_copy_coords(hdg_mesh_t mesh, double* xnode, double* xfnode, double* geo) {
  if (!mesh) {
    set_error("hdg_mesh_copy_coords: null mesh");
    return HDG_ERR_INVALID_ARG;
  }
  const hdg::Mesh& m = mesh->m;
  const bool mx = !m.pe.empty();
  if (xnode) {
    const std::vector<double>& x = mx ? m.xnode_mix : m.xnode;
    std::memcpy(xnode, x.data(), sizeof(double) * x.size());
  }
  if (xfnode) {
    const std::vector<double>& x = mx ? m.xfnode_mix : m.scheme == HDG_SCHEME_HDG ? m.xfnode : m.xedg;
    std::memcpy(xfnode, x.data(), sizeof(double) * x.size());
  }
  if (geo) std::memcpy(geo, m.geo.data(), sizeof(double) * m.geo.size());
  return HDG_OK;
}

int hdg_ctx_create(hdg_mesh_t mesh, const hdg_physics* phys, int device, hdg_ctx_t* out) {
  if (!mesh || !phys || !out) {
    set_error("hdg_ctx_create: null argument");
    return HDG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!(phys->gamma > 1.0) || !(phys->mach > 0.0) || phys->reynolds < 0.0 || !(phys->prandtl > 0.0) ||
      !(phys->mu_exponent >= 0.0 && phys->mu_exponent <= 4.0) || phys->visc_flux < 0 || phys->visc_flux > 2 ||
      (phys->stabilization != HDG_STAB_SLF && phys->stabilization != HDG_STAB_S)) {
    set_error("hdg_ctx_create: invalid physics parameters");
    return HDG_ERR_INVALID_ARG;
  }
  const hdg::Mesh& m = mesh->m;
  const bool visc = phys->reynolds > 0.0;
  if (m.pe.empty() && !hdg::config_supported(m.dim, m.p, m.K, visc)) {
    set_error("hdg_ctx_create: (dim, p, quad_points, physics) not compiled in");
    return HDG_ERR_UNSUPPORTED;
  }
  if (visc)
    for (int8_t k : m.face_bc)
      if (k == HDG_BC_SLIP) {
        set_error("hdg_ctx_create: the slip wall is defined for the Euler equations only");
        return HDG_ERR_UNSUPPORTED;
      }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    set_error("hdg_ctx_create: no such CUDA device");
    return HDG_ERR_CUDA;
  }
  DeviceGuard guard(device);
  auto* c = new hdg_ctx();
  c->mesh = mesh;
  c->device = device;
  c->visc = visc;
  const double g = phys->gamma;
  c->ph.gamma = g;
  c->ph.cv = 1.0 / (g * (g - 1.0) * phys->mach * phys->mach);
  c->ph.mu = visc ? 1.0 / phys->reynolds : 0.0;
  c->ph.kappa = g * c->ph.cv * c->ph.mu / phys->prandtl;
  c->ph.mu_exp = visc ? phys->mu_exponent : 0.0;
  c->ph.gflux = phys->visc_flux == 1 ? 1 : 2;
  c->ph.stab = phys->stabilization;
  c->dim = m.dim;
  c->p = m.p;
  c->K = m.K;
  c->M = m.dim + 2;
  c->NP = m.ref.Np;
  c->NFN = m.ref.Nf;
  c->NF = m.ref.nF;
  c->NG = m.ref.NG;
  c->NGF = m.ref.NGF;
  c->NV = c->NP * c->M;
  c->NT = c->NF * c->NFN * c->M;
  c->GEO = m.geo_stride;
  c->E = m.E;
  c->F = m.nFaces;
  c->scheme = m.scheme == HDG_SCHEME_HDG ? 0 : 1;
  c->n_tnodes = m.scheme == HDG_SCHEME_HDG ? m.nFaces * m.ref.Nf : m.n_edg;
  c->ntrace = c->n_tnodes * c->M;
  if (const char* av = std::getenv("HDG_ASM_VARIANT")) {  // force a tile shape (tests)
    long v = std::strtol(av, nullptr, 10);
    if (v >= 0 && v < 4) c->asm_variant = c->face_variant = (int)v;
  }
  if (const char* cv = std::getenv("HDG_COND_VARIANT")) {  // force a condensation shape (tests)
    long v = std::strtol(cv, nullptr, 10);
    if (v >= 0 && v < 4) c->cond_variant = (int)v;
  }
  if (const char* st = std::getenv("HDG_T5_STALL_FIRST_COPY")) c->t5_stall = std::strtol(st, nullptr, 10) != 0;
  if (const char* sb = std::getenv("HDG_SINK_BUFFERS")) {  // device buffers of the host-sink ring
    long v = std::strtol(sb, nullptr, 10);
    if (v >= 2 && v <= hdg_ctx::kSinkMax) c->sink_bufs = (int)v;
  }
  if (const char* ch = std::getenv("HDG_ELEMENT_CHUNK")) {
    long v = std::strtol(ch, nullptr, 10);
    if (v > 0) c->chunk = std::min<int64_t>(v, c->E);
  }
  if (!m.pe.empty()) {  // mixed degrees: class tables, packed layout and work queue only
    c->n_tnodes = m.fnoff.back();
    c->ntrace = c->n_tnodes * c->M;
    int rc = HDG_OK;
    if ((rc = upload(&c->d_geo, m.geo)) || (rc = hdg::pclass_setup(c))) {
      hdg_ctx_destroy(c);
      return rc;
    }
    *out = c;
    return HDG_OK;
  }

  hdg::RefTables T = hdg::make_tables(m.ref);
  std::vector<double> tab;
  size_t off[8];
  const std::vector<double>* parts[8] = {&T.W, &T.Phi, &T.dPhi, &T.PL, &T.WF, &T.PhiF, &T.dPhiF, &T.PLF};
  for (int i = 0; i < 8; ++i) {
    off[i] = tab.size();
    tab.insert(tab.end(), parts[i]->begin(), parts[i]->end());
  }
  std::vector<int> itab(T.fnodes);
  const size_t npos_off = itab.size();
  std::vector<int> nodepos(c->NF * c->NP, -1);
  for (int f = 0; f < c->NF; ++f)
    for (int cc = 0; cc < c->NFN; ++cc) nodepos[f * c->NP + T.fnodes[f * c->NFN + cc]] = cc;
  itab.insert(itab.end(), nodepos.begin(), nodepos.end());

  // element -> canonical face node; face sides
  std::vector<int> tgidx(c->E * c->NF * c->NFN);
  for (int64_t e = 0; e < c->E; ++e)
    for (int f = 0; f < c->NF; ++f)
      for (int cc = 0; cc < c->NFN; ++cc) {
        const int64_t i = (e * c->NF + f) * c->NFN + cc;
        tgidx[i] = c->scheme ? m.edg_index[i] : m.face_of[e * c->NF + f] * c->NFN + m.fnode_map[i];
      }
  // every local occurrence (e NF NFN + local face node) of each trace node, grouped by node (the
  // EDG trace operator and its node-block preconditioner gather through it)
  std::vector<int> tr_ptr(c->n_tnodes + 1, 0), tr_occ(tgidx.size());
  for (int t : tgidx) ++tr_ptr[t + 1];
  for (int64_t t = 0; t < c->n_tnodes; ++t) tr_ptr[t + 1] += tr_ptr[t];
  {
    std::vector<int> fill(tr_ptr.begin(), tr_ptr.end() - 1);
    for (size_t i = 0; i < tgidx.size(); ++i) tr_occ[fill[tgidx[i]]++] = (int)i;
  }
  std::vector<int> fs_elem(2 * c->F), fs_loc(2 * c->F * c->NFN, 0);
  for (int64_t F = 0; F < c->F; ++F)
    for (int sd = 0; sd < 2; ++sd) {
      int32_t ef = m.face_side[2 * F + sd];
      if (ef < 0) {  // the missing side of a boundary face
        fs_elem[2 * F + sd] = -1;
        continue;
      }
      int64_t e = ef / c->NF;
      int f = ef % c->NF;
      fs_elem[2 * F + sd] = (int)e;
      for (int cc = 0; cc < c->NFN; ++cc) {
        int canon = m.fnode_map[(e * c->NF + f) * c->NFN + cc];
        fs_loc[(2 * F + sd) * c->NFN + canon] = f * c->NFN + cc;
      }
    }
  // boundary faces in ascending e NF + f, with their types
  std::vector<int> bkind;
  for (int64_t e = 0; e < c->E; ++e)
    for (int f = 0; f < c->NF; ++f) {
      const int8_t k = m.face_bc[m.face_of[e * c->NF + f]];
      if (k == HDG_BC_PERIODIC) continue;
      c->h_bface.push_back((int)(e * c->NF + f));
      bkind.push_back(k);
      if (k == HDG_BC_STATE) c->has_state_bc = true;
    }
  int rc = HDG_OK;
  if (!c->h_bface.empty() && ((rc = upload(&c->d_bface, c->h_bface)) || (rc = upload(&c->d_bkind, bkind)))) {
    hdg_ctx_destroy(c);
    return rc;
  }
  if (m.scheme == HDG_SCHEME_EDG && !c->h_bface.empty()) {
    // the continuous EDG trace takes the state strongly at the nodes of its BC_STATE faces
    const int per = c->NF * c->NFN;
    std::vector<char> on_state(m.n_edg, 0), seen(m.n_edg, 0);
    for (size_t k = 0; k < c->h_bface.size(); ++k)
      if (bkind[k] == HDG_BC_STATE)
        for (int cc = 0; cc < c->NFN; ++cc) on_state[m.edg_index[(int64_t)c->h_bface[k] * c->NFN + cc]] = 1;
    std::vector<int> first;
    for (int64_t i = 0; i < c->E * per; ++i) {
      const int32_t node = m.edg_index[i];
      if (!on_state[node]) continue;
      c->h_dir.push_back((int)i);
      first.push_back(seen[node] ? 0 : 1);
      seen[node] = 1;
    }
    if (!c->h_dir.empty() && ((rc = upload(&c->d_dir, c->h_dir)) || (rc = upload(&c->d_dir_first, first)))) {
      hdg_ctx_destroy(c);
      return rc;
    }
  }
  if ((rc = upload(&c->d_tab, tab)) || (rc = upload(&c->d_itab, itab)) || (rc = upload(&c->d_tgidx, tgidx)) ||
      (rc = upload(&c->d_geo, m.geo)) || (rc = upload(&c->d_fs_elem, fs_elem)) || (rc = upload(&c->d_fs_loc, fs_loc)) ||
      (rc = upload(&c->d_tr_ptr, tr_ptr)) || (rc = upload(&c->d_tr_occ, tr_occ))) {
    hdg_ctx_destroy(c);
    return rc;
  }
  c->tab_size = tab.size();
  c->T.W = c->d_tab + off[0];
  c->T.Phi = c->d_tab + off[1];
  c->T.dPhi = c->d_tab + off[2];
  c->T.PL = c->d_tab + off[3];
  c->T.WF = c->d_tab + off[4];
  c->T.PhiF = c->d_tab + off[5];
  c->T.dPhiF = c->d_tab + off[6];
  c->T.PLF = c->d_tab + off[7];
  c->T.fnodes = c->d_itab;
  c->T.nodepos = c->d_itab + npos_off;
  *out = c;
  return HDG_OK;
}

void hdg_ctx_destroy(hdg_ctx_t c) {
  if (!c) return;
  DeviceGuard guard(c->device);
  void* bufs[] = {c->d_tab, c->d_tab_df, c->d_itab, c->d_tgidx, c->d_geo, c->d_fs_elem, c->d_fs_loc, c->d_scr,
                  c->d_sw, c->d_pc, c->d_dense, c->d_dpiv, c->d_red, c->d_S,
                  c->d_g, c->d_recov, c->d_R, c->d_dV, c->d_dVh, c->d_status, c->d_hist, c->d_V0,
                  c->d_Vh0, c->d_feat, c->d_pred, c->d_dirk, c->d_ent, c->d_tr_ptr, c->d_tr_occ, c->d_pcn,
                  c->d_bface, c->d_bkind, c->d_vb, c->d_mv_err, c->d_Sdf, c->d_dir, c->d_dir_first};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->h_red) cudaFreeHost(c->h_red);
  if (c->d_gm) cudaFree(c->d_gm);
  if (c->h_gm) cudaFreeHost(c->h_gm);
  if (c->gm_graph) cudaGraphExecDestroy(c->gm_graph);
  if (c->gm_stream) cudaStreamDestroy(c->gm_stream);
  if (c->lu_graph_exec) cudaGraphExecDestroy(c->lu_graph_exec);
  if (c->ac_graph) cudaGraphExecDestroy(c->ac_graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
    for (int b = 0; b < hdg_ctx::kSinkMax; ++b) {
      if (c->ev_done[b]) cudaEventDestroy(c->ev_done[b]);
      if (c->ev_copied[b]) cudaEventDestroy(c->ev_copied[b]);
      if (c->d_Sbuf[b]) cudaFree(c->d_Sbuf[b]);
    }
  }
  for (auto& r : c->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  hdg::pclass_free(c->pm);
  delete c;
}

// Array lengths (doubles) of the compute calls: uniform strides, or the packed per-element layout
// of a mixed-degree mesh
static int64_t len_S(const hdg_ctx* c) { return c->pm ? c->mesh->m.soff.back() : c->E * (int64_t)c->NT * c->NT; }
static int64_t len_g(const hdg_ctx* c) { return c->pm ? c->mesh->m.toff.back() : c->E * (int64_t)c->NT; }
static int64_t len_recov(const hdg_ctx* c) {
  return c->pm ? c->mesh->m.roff.back() : c->E * ((int64_t)c->NV * c->NT + c->NV);
}
static int64_t len_R(const hdg_ctx* c) { return c->pm ? c->mesh->m.Roff.back() : c->E * (int64_t)(c->NV + c->NT); }
static int64_t len_V(const hdg_ctx* c) { return c->pm ? c->mesh->m.voff.back() : c->E * (int64_t)c->NV; }

// Calls not built for meshes whose elements differ in degree
#define HDG_UNIFORM_ONLY(ctx, name)                                                      \
  do {                                                                                   \
    if ((ctx)->pm) {                                                                     \
      set_error(std::string(name) + ": not built for meshes of mixed degree");           \
      return HDG_ERR_UNSUPPORTED;                                                        \
    }                                                                                    \
  } while (0)

#define HDG_REQUIRE(cond, msg)  \
  do {                          \
    if (!(cond)) {              \
      set_error(msg);           \
      return HDG_ERR_INVALID_ARG; \
    }                           \
  } while (0)

int hdg_ctx_set_boundary_state(hdg_ctx_t ctx, const double* Vb, void* stream) {
  HDG_REQUIRE(ctx && Vb, "hdg_ctx_set_boundary_state: null argument");
  HDG_UNIFORM_ONLY(ctx, "hdg_ctx_set_boundary_state");
  DeviceGuard guard(ctx->device);
  if (!ctx->d_vb) HDG_CK(cudaMalloc(&ctx->d_vb, sizeof(double) * ctx->ntrace));
  HDG_CK(cudaMemcpyAsync(ctx->d_vb, Vb, sizeof(double) * ctx->ntrace, cudaMemcpyDeviceToDevice,
                         (cudaStream_t)stream));
  ctx->vb_set = true;
  return HDG_OK;
}

int hdg_prim_to_entropy(hdg_ctx_t ctx, const double* prim, int64_t n_points, double* v, void* stream) {
  HDG_REQUIRE(ctx && prim && v && n_points >= 0, "hdg_prim_to_entropy: invalid argument");
  DeviceGuard guard(ctx->device);
  return hdg::launch_prim_to_entropy(ctx, prim, n_points, v, (cudaStream_t)stream);
}

int hdg_history(hdg_ctx_t ctx, const double* V0, const double* V1, double c0, double c1, double* hist,
                void* stream) {
  HDG_REQUIRE(ctx && V0 && hist, "hdg_history: invalid argument");
  DeviceGuard guard(ctx->device);
  return hdg::launch_history(ctx, V0, V1, c0, c1, hist, (cudaStream_t)stream);
}

int hdg_add_source(hdg_ctx_t ctx, const double* src, double c, double* hist, void* stream) {
  HDG_REQUIRE(ctx && src && hist && std::isfinite(c), "hdg_add_source: invalid argument");
  HDG_UNIFORM_ONLY(ctx, "hdg_add_source");
  DeviceGuard guard(ctx->device);
  return hdg::launch_source_weak(ctx, src, c, hist, (cudaStream_t)stream);
}

int hdg_assemble_condense(hdg_ctx_t ctx, const double* V, const double* Vhat, const double* hist, double mass_coef,
                          int precision, double* S, double* g, double* recov, double* R, int32_t* elem_status,
                          void* stream) {
  HDG_REQUIRE(ctx && V && Vhat && S && g && recov && R, "hdg_assemble_condense: null argument");
  HDG_REQUIRE(precision == HDG_PREC_FP64 || precision == HDG_PREC_MIXED, "hdg_assemble_condense: precision");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* st = elem_status;
  if (!st) {
    if (!ctx->d_status) HDG_CK(cudaMalloc(&ctx->d_status, sizeof(int32_t) * ctx->E));
    HDG_CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t) * ctx->E, s));
    st = ctx->d_status;
  }
  if (ctx->pm) {
    if (precision != HDG_PREC_FP64) {
      set_error("hdg_assemble_condense: meshes of mixed degree are built for the FP64 form");
      return HDG_ERR_UNSUPPORTED;
    }
    return hdg::assemble_condense_pclass(ctx, V, Vhat, hist, mass_coef, S, g, recov, R, st, s);
  }
  if (precision == HDG_PREC_MIXED)
    return hdg::assemble_condense_mixed(ctx, V, Vhat, hist, mass_coef, S, g, recov, R, st, s);
  return hdg::assemble_condense_fp64(ctx, V, Vhat, hist, mass_coef, S, g, recov, R, st, s);
}


int hdg_assemble_condense_graph(hdg_ctx_t ctx, const double* V, const double* Vhat, const double* hist,
                                double mass_coef, int precision, double* S, double* g, double* recov, double* R,
                                int32_t* elem_status, void* stream) {
  HDG_REQUIRE(ctx && V && Vhat && S && g && recov && R, "hdg_assemble_condense_graph: null argument");
  HDG_UNIFORM_ONLY(ctx, "hdg_assemble_condense_graph");
  HDG_REQUIRE(precision == HDG_PREC_FP64 || precision == HDG_PREC_MIXED, "hdg_assemble_condense_graph: precision");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  using Key = hdg_ctx::GraphKey;
  Key k;
  const void* args[9] = {V, Vhat, hist, S, g, recov, R, elem_status, ctx->d_status};
  for (int i = 0; i < 9; ++i) k.p[i] = args[i];
  k.mass_coef = mass_coef;
  k.precision = precision;
  k.scratch = ctx->d_scr;
  k.chunk = ctx->chunk;
  if (ctx->ac_graph && ctx->ac_key == k) {  // replay
    HDG_CK(cudaGraphLaunch(ctx->ac_graph, s));
    ++ctx->ac_replays;
    for (int c = 0; c < HDG_KERNEL_CLASSES; ++c) ctx->launches[c] += ctx->ac_launches[c];
    return HDG_OK;
  }
  // an ordinary call computes this call's result (and tunes and allocates what the sequence
  // needs); the same sequence is then captured, without running, on a private stream
  int rc = hdg_assemble_condense(ctx, V, Vhat, hist, mass_coef, precision, S, g, recov, R, elem_status, stream);
  if (rc != HDG_OK || ctx->ac_graph_failed) return rc;
  k.p[8] = ctx->d_status;
  k.scratch = ctx->d_scr;
  k.chunk = ctx->chunk;
  if (!ctx->cap_stream) HDG_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  int64_t before[HDG_KERNEL_CLASSES];
  for (int c = 0; c < HDG_KERNEL_CLASSES; ++c) before[c] = ctx->launches[c];
  const bool prof = ctx->prof;
  ctx->prof = false;  // no timing events inside the graph
  cudaGraph_t graph = nullptr;
  int rc2 = HDG_OK;
  cudaError_t err = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (err == cudaSuccess) {
    rc2 = hdg_assemble_condense(ctx, V, Vhat, hist, mass_coef, precision, S, g, recov, R, elem_status,
                                ctx->cap_stream);
    err = cudaStreamEndCapture(ctx->cap_stream, &graph);
  }
  ctx->prof = prof;
  for (int c = 0; c < HDG_KERNEL_CLASSES; ++c) {
    ctx->ac_launches[c] = ctx->launches[c] - before[c];
    ctx->launches[c] = before[c];
  }
  cudaGraphExec_t exec = nullptr;
  if (err == cudaSuccess && rc2 == HDG_OK && graph) err = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (err != cudaSuccess || rc2 != HDG_OK || !exec) {  // keep the ordinary path from now on
    if (exec) cudaGraphExecDestroy(exec);
    cudaGetLastError();
    ctx->ac_graph_failed = true;
    return HDG_OK;
  }
  if (ctx->ac_graph) cudaGraphExecDestroy(ctx->ac_graph);
  ctx->ac_graph = exec;
  ctx->ac_key = k;
  return HDG_OK;
}

int hdg_assemble_condense_host(hdg_ctx_t ctx, const double* V, const double* Vhat, const double* hist,
                               double mass_coef, int precision, double* S_host, double* g_host, double* recov,
                               double* R, int32_t* elem_status, void* stream) {
  HDG_REQUIRE(ctx && V && Vhat && S_host && g_host && recov && R, "hdg_assemble_condense_host: null argument");
  HDG_UNIFORM_ONLY(ctx, "hdg_assemble_condense_host");
  HDG_REQUIRE(precision == HDG_PREC_FP64 || precision == HDG_PREC_MIXED, "hdg_assemble_condense_host: precision");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!ctx->copy_stream) {
    HDG_CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    for (int b = 0; b < ctx->sink_bufs; ++b) {
      HDG_CK(cudaEventCreateWithFlags(&ctx->ev_done[b], cudaEventDisableTiming));
      HDG_CK(cudaEventCreateWithFlags(&ctx->ev_copied[b], cudaEventDisableTiming));
    }
  }
  if (!ctx->d_g) HDG_CK(cudaMalloc(&ctx->d_g, sizeof(double) * ctx->E * ctx->NT));
  int32_t* st = elem_status;
  if (!st) {
    if (!ctx->d_status) HDG_CK(cudaMalloc(&ctx->d_status, sizeof(int32_t) * ctx->E));
    HDG_CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t) * ctx->E, s));
    st = ctx->d_status;
  }
  ctx->sink_host = S_host;
  ctx->sink_idx = 0;
  int rc = precision == HDG_PREC_MIXED
               ? hdg::assemble_condense_mixed(ctx, V, Vhat, hist, mass_coef, nullptr, ctx->d_g, recov, R, st, s)
               : hdg::assemble_condense_fp64(ctx, V, Vhat, hist, mass_coef, nullptr, ctx->d_g, recov, R, st, s);
  const int used = ctx->sink_idx;
  ctx->sink_host = nullptr;
  if (rc) return rc;
  HDG_CK(cudaMemcpyAsync(g_host, ctx->d_g, sizeof(double) * ctx->E * ctx->NT, cudaMemcpyDeviceToHost, s));
  for (int b = 0; b < ctx->sink_bufs && b < used; ++b) HDG_CK(cudaStreamWaitEvent(s, ctx->ev_copied[b], 0));
  return HDG_OK;
}

int hdg_entropy_production(hdg_ctx_t ctx, const double* V, const double* Vhat, double* int_rho_s, double* production,
                           void* stream) {
  HDG_REQUIRE(ctx && V && Vhat && int_rho_s && production, "hdg_entropy_production: null argument");
  HDG_UNIFORM_ONLY(ctx, "hdg_entropy_production");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!ctx->d_ent) HDG_CK(cudaMalloc(&ctx->d_ent, 2 * sizeof(double)));
  HDG_CK(cudaMemsetAsync(ctx->d_ent, 0, 2 * sizeof(double), s));
  if (int rc = hdg::entropy_terms(ctx, V, Vhat, ctx->d_ent, s)) return rc;
  double h[2];
  HDG_CK(cudaMemcpyAsync(h, ctx->d_ent, sizeof(h), cudaMemcpyDeviceToHost, s));
  HDG_CK(cudaStreamSynchronize(s));
  *int_rho_s = h[0];
  *production = h[1];
  return HDG_OK;
}

int hdg_trace_solve(hdg_ctx_t ctx, const double* S, const double* g, double* dVhat, int method, double rtol,
                    int max_it, int* iters, double* final_res, void* stream) {
  HDG_REQUIRE(ctx && S && g && dVhat && iters && final_res, "hdg_trace_solve: null argument");
  HDG_REQUIRE(method >= HDG_SOLVER_AUTO && method <= HDG_SOLVER_DENSE && rtol > 0.0 && max_it > 0,
              "hdg_trace_solve: invalid method / tolerance");
  DeviceGuard guard(ctx->device);
  return hdg::trace_solve(ctx, S, g, dVhat, method, rtol, max_it, iters, final_res, (cudaStream_t)stream);
}

int hdg_recover_interior(hdg_ctx_t ctx, const double* recov, const double* dVhat, double* dV, void* stream) {
  HDG_REQUIRE(ctx && recov && dVhat && dV, "hdg_recover_interior: null argument");
  DeviceGuard guard(ctx->device);
  return hdg::launch_recover(ctx, recov, dVhat, dV, (cudaStream_t)stream);
}

int hdg_trace_matvec(hdg_ctx_t ctx, const double* S, const double* x, double* y, void* stream) {
  HDG_REQUIRE(ctx && S && x && y, "hdg_trace_matvec: null argument");
  DeviceGuard guard(ctx->device);
  double* work = nullptr;
  HDG_CK(cudaMallocAsync(&work, sizeof(double) * len_g(ctx), (cudaStream_t)stream));
  int rc = hdg::launch_trace_matvec(ctx, S, x, y, work, (cudaStream_t)stream);
  cudaFreeAsync(work, (cudaStream_t)stream);
  return rc;
}

int hdg_residual_norm(hdg_ctx_t ctx, const double* R, double* norm, void* stream) {
  HDG_REQUIRE(ctx && R && norm, "hdg_residual_norm: null argument");
  DeviceGuard guard(ctx->device);
  return hdg::residual_norm(ctx, R, norm, (cudaStream_t)stream);
}

int hdg_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, void* stream) {
  HDG_REQUIRE(n >= 0 && x && y && out, "hdg_axpby: invalid argument");
  return hdg::launch_axpby(n, a, x, b, y, out, (cudaStream_t)stream);
}

int hdg_ctx_set_refinement(hdg_ctx_t ctx, double tol, int fp64_fallback) {
  HDG_REQUIRE(ctx && tol >= 0.0 && tol < 1.0, "hdg_ctx_set_refinement: invalid argument");
  ctx->refine_tol = tol;
  ctx->refine_fallback = fp64_fallback != 0;
  if (ctx->ac_graph) {  // the captured launch sequence depends on both settings
    cudaGraphExecDestroy(ctx->ac_graph);
    ctx->ac_graph = nullptr;
    ctx->ac_key = hdg_ctx::GraphKey{};
  }
  return HDG_OK;
}

int hdg_ctx_set_trace_solver(hdg_ctx_t ctx, int method, double rtol, int max_it) {
  HDG_REQUIRE(ctx && method >= HDG_SOLVER_AUTO && method <= HDG_SOLVER_DENSE && rtol >= 0.0 && rtol < 1.0 &&
                  max_it > 0,
              "hdg_ctx_set_trace_solver: invalid argument");
  ctx->newton_solver = method;
  ctx->newton_rtol = rtol;
  ctx->newton_max_it = max_it;
  return HDG_OK;
}

int hdg_ctx_trace_cycles(hdg_ctx_t ctx, int64_t* cycles, int64_t* replays) {
  HDG_REQUIRE(ctx && cycles && replays, "hdg_ctx_trace_cycles: null argument");
  *cycles = ctx->gm_cycles;
  *replays = ctx->gm_replays;
  return HDG_OK;
}

int hdg_ctx_graph_replays(hdg_ctx_t ctx, int64_t* replays) {
  HDG_REQUIRE(ctx && replays, "hdg_ctx_graph_replays: null argument");
  *replays = ctx->ac_replays;
  return HDG_OK;
}

int hdg_profile_enable(hdg_ctx_t ctx, int on) {
  HDG_REQUIRE(ctx, "hdg_profile_enable: null context");
  ctx->prof = on != 0;
  return HDG_OK;
}

static int drain_profile(hdg_ctx_t ctx) {
  for (auto& r : ctx->pending) {
    HDG_CK(cudaEventSynchronize(r.b));
    float ms = 0.f;
    HDG_CK(cudaEventElapsedTime(&ms, r.a, r.b));
    ctx->prof_ms[r.cls] += ms;
    ctx->prof_n[r.cls] += 1;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  ctx->pending.clear();
  return HDG_OK;
}

int hdg_profile_reset(hdg_ctx_t ctx) {
  HDG_REQUIRE(ctx, "hdg_profile_reset: null context");
  DeviceGuard guard(ctx->device);
  int rc = drain_profile(ctx);
  for (int k = 0; k < HDG_KERNEL_CLASSES; ++k) {
    ctx->prof_ms[k] = 0.0;
    ctx->prof_n[k] = 0;
    ctx->launches[k] = 0;
  }
  return rc;
}

int hdg_profile_read(hdg_ctx_t ctx, int kernel_class, int64_t* launches, double* total_ms) {
  HDG_REQUIRE(ctx && launches && total_ms && kernel_class >= -1 && kernel_class < HDG_KERNEL_CLASSES,
              "hdg_profile_read: invalid argument");
  DeviceGuard guard(ctx->device);
  int rc = drain_profile(ctx);
  if (rc) return rc;
  *launches = 0;
  *total_ms = 0.0;
  for (int k = 0; k < HDG_KERNEL_CLASSES; ++k)
    if (kernel_class < 0 || k == kernel_class) {
      *launches += ctx->launches[k];
      *total_ms += ctx->prof_ms[k];
    }
  return HDG_OK;
}

int hdg_newton_solve(hdg_ctx_t ctx, double* V, double* Vhat, const double* hist, double mass_coef, int precision,
                     double tol, int max_newton, int* newton_iters, double* res_norm, double* res_history,
                     int* trace_iters, void* stream) {
  HDG_REQUIRE(ctx && V && Vhat && newton_iters && res_norm && tol > 0.0 && max_newton >= 0,
              "hdg_newton_solve: invalid argument");
  HDG_REQUIRE(precision == HDG_PREC_FP64 || precision == HDG_PREC_MIXED, "hdg_newton_solve: precision");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t E = ctx->E;
  if (!ctx->d_S) {
    HDG_CK(cudaMalloc(&ctx->d_S, sizeof(double) * len_S(ctx)));
    if (!ctx->d_g) HDG_CK(cudaMalloc(&ctx->d_g, sizeof(double) * len_g(ctx)));
    HDG_CK(cudaMalloc(&ctx->d_recov, sizeof(double) * len_recov(ctx)));
    HDG_CK(cudaMalloc(&ctx->d_R, sizeof(double) * len_R(ctx)));
    HDG_CK(cudaMalloc(&ctx->d_dV, sizeof(double) * len_V(ctx)));
    HDG_CK(cudaMalloc(&ctx->d_dVh, sizeof(double) * ctx->ntrace));
  }
  if (!ctx->d_status) HDG_CK(cudaMalloc(&ctx->d_status, sizeof(int32_t) * E));
  std::vector<int32_t> hstat;
  double r0 = -1.0, rn = 0.0, r_prev = -1.0, eta = 0.1;
  *newton_iters = 0;
  if (trace_iters) *trace_iters = 0;
  for (int it = 0;; ++it) {
    HDG_CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t) * E, s));
    // one degree: the assemble + condense launch sequence is captured on the first iteration and
    // replayed on the others (its arguments do not change within the solve); mixed degrees: one
    // persistent launch
    int rc = ctx->pm ? hdg_assemble_condense(ctx, V, Vhat, hist, mass_coef, precision, ctx->d_S, ctx->d_g,
                                             ctx->d_recov, ctx->d_R, ctx->d_status, s)
                     : hdg_assemble_condense_graph(ctx, V, Vhat, hist, mass_coef, precision, ctx->d_S, ctx->d_g,
                                                   ctx->d_recov, ctx->d_R, ctx->d_status, s);
    if (rc) return rc;
    rc = hdg::residual_norm(ctx, ctx->d_R, &rn, s);
    if (rc) return rc;
    hstat.resize(E);
    HDG_CK(cudaMemcpyAsync(hstat.data(), ctx->d_status, sizeof(int32_t) * E, cudaMemcpyDeviceToHost, s));
    HDG_CK(cudaStreamSynchronize(s));
    int bits = 0;
    for (int32_t b : hstat) bits |= b;
    *res_norm = rn;
    if (res_history) res_history[it] = rn;
    if (bits & HDG_ELEM_NONPHYSICAL) {
      set_error("hdg_newton_solve: non-physical state");
      return HDG_ERR_NONPHYSICAL;
    }
    if (bits & HDG_ELEM_SINGULAR) {
      set_error("hdg_newton_solve: singular element matrix");
      return HDG_ERR_SINGULAR;
    }
    if (bits & HDG_ELEM_TIMEOUT) {  // only with the FP64 recomputation switched off
      set_error("hdg_newton_solve: a bounded wait in the element condensation gave up");
      return HDG_ERR_TIMEOUT;
    }
    if (bits & HDG_ELEM_REFINE) {  // only with the FP64 recomputation switched off
      set_error("hdg_newton_solve: iterative refinement of an element block missed its tolerance");
      return HDG_ERR_REFINE;
    }
    if (r0 < 0.0) r0 = rn;
    if (rn <= tol * std::max(1.0, r0)) return HDG_OK;
    if (it >= max_newton) {
      set_error("hdg_newton_solve: Newton did not converge");
      return HDG_ERR_NOT_CONVERGED;
    }
    // relative tolerance of the trace solve: fixed, or (newton_rtol == 0) the Eisenstat-Walker
    // forcing term eta_k = 0.9 (|R_k| / |R_{k-1}|)^2, safeguarded by 0.9 eta_{k-1}^2 when that is
    // above 0.1, at most 0.1, and no tighter than half the tolerance the residual still has to gain
    double rtol = ctx->newton_rtol;
    if (rtol == 0.0) {
      if (r_prev > 0.0) {
        const double ratio = rn / r_prev, safe = 0.9 * eta * eta;
        eta = 0.9 * ratio * ratio;
        if (safe > 0.1) eta = std::max(eta, safe);
      }
      eta = std::min(eta, 0.1);
      eta = std::max(eta, 0.5 * tol * std::max(1.0, r0) / rn);
      eta = std::max(eta, 1e-13);
      rtol = eta;
    }
    r_prev = rn;
    int iters = 0;
    double fres = 0.0;
    rc = hdg::trace_solve(ctx, ctx->d_S, ctx->d_g, ctx->d_dVh, ctx->newton_solver, rtol, ctx->newton_max_it, &iters,
                          &fres, s);
    if (trace_iters) *trace_iters += iters;
    if (rc) return rc;
    rc = hdg::launch_recover(ctx, ctx->d_recov, ctx->d_dVh, ctx->d_dV, s);
    if (rc) return rc;
    rc = hdg::launch_axpy(len_V(ctx), 1.0, ctx->d_dV, V, s);
    if (rc) return rc;
    rc = hdg::launch_axpy(ctx->ntrace, 1.0, ctx->d_dVh, Vhat, s);
    if (rc) return rc;
    *newton_iters = it + 1;
  }
}

int hdg_newton_step(hdg_ctx_t ctx, double* V, double* Vhat, const double* V_n, const double* V_nm1, double dt,
                    int bdf_order, int precision, double tol, int max_newton, const hdg_warmstart* warmstart,
                    int* newton_iters, double* res_norm, double* res_history, int* trace_iters, void* stream) {
  HDG_REQUIRE(ctx && V && Vhat && newton_iters && res_norm && tol > 0.0 && max_newton >= 0,
              "hdg_newton_step: invalid argument");
  HDG_REQUIRE(bdf_order >= 0 && bdf_order <= 2, "hdg_newton_step: bdf_order must be 0, 1 or 2");
  HDG_REQUIRE(bdf_order == 0 || (dt > 0.0 && V_n), "hdg_newton_step: BDF needs dt > 0 and V_n");
  HDG_REQUIRE(bdf_order < 2 || V_nm1, "hdg_newton_step: BDF2 needs V_nm1");
  HDG_REQUIRE(!warmstart || (warmstart->vhat_n && warmstart->dvhat1 && warmstart->dvhat2),
              "hdg_newton_step: warm start needs vhat_n, dvhat1 and dvhat2");
  HDG_REQUIRE(precision == HDG_PREC_FP64 || precision == HDG_PREC_MIXED, "hdg_newton_step: precision");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nV = len_V(ctx);
  // BDF coefficients: mass_coef (u(v), w) - hist, hist = c0 (u(v^n), w) + c1 (u(v^{n-1}), w)
  double mass = 0.0;
  const double* hist = nullptr;
  if (bdf_order > 0) {
    if (!ctx->d_hist) HDG_CK(cudaMalloc(&ctx->d_hist, sizeof(double) * nV));
    const double c0 = bdf_order == 1 ? 1.0 / dt : 2.0 / dt, c1 = bdf_order == 1 ? 0.0 : -0.5 / dt;
    mass = bdf_order == 1 ? 1.0 / dt : 1.5 / dt;
    int rc = hdg::launch_history(ctx, V_n, bdf_order == 2 ? V_nm1 : nullptr, c0, c1, ctx->d_hist, s);
    if (rc) return rc;
    hist = ctx->d_hist;
  }
  if (!warmstart)
    return hdg_newton_solve(ctx, V, Vhat, hist, mass, precision, tol, max_newton, newton_iters, res_norm,
                            res_history, trace_iters, stream);
  // Learned (or element-local) start: the caller's guess (V0, Vhat0) is linearised once;
  // the network's trace (or Vhat0 itself) takes the place of the first global trace solve and
  // the interior follows from the element-local recovery dV = -y - X P (vhat_m - Vhat0).
  if (ctx->scheme || ctx->pm) {
    set_error("hdg_newton_step: the learned warm start works on face traces (HDG) of one degree only");
    return HDG_ERR_UNSUPPORTED;
  }
  const hdg_warmstart& w = *warmstart;
  if (!ctx->d_S) {
    HDG_CK(cudaMalloc(&ctx->d_S, sizeof(double) * ctx->E * ctx->NT * ctx->NT));
    if (!ctx->d_g) HDG_CK(cudaMalloc(&ctx->d_g, sizeof(double) * ctx->E * ctx->NT));
    HDG_CK(cudaMalloc(&ctx->d_recov, sizeof(double) * ctx->E * (ctx->NV * ctx->NT + ctx->NV)));
    HDG_CK(cudaMalloc(&ctx->d_R, sizeof(double) * ctx->E * (ctx->NV + ctx->NT)));
    HDG_CK(cudaMalloc(&ctx->d_dV, sizeof(double) * nV));
    HDG_CK(cudaMalloc(&ctx->d_dVh, sizeof(double) * ctx->ntrace));
  }
  if (!ctx->d_status) HDG_CK(cudaMalloc(&ctx->d_status, sizeof(int32_t) * ctx->E));
  if (!ctx->d_V0) {
    HDG_CK(cudaMalloc(&ctx->d_V0, sizeof(double) * nV));
    HDG_CK(cudaMalloc(&ctx->d_Vh0, sizeof(double) * ctx->ntrace));
  }
  HDG_CK(cudaMemcpyAsync(ctx->d_V0, V, sizeof(double) * nV, cudaMemcpyDeviceToDevice, s));
  HDG_CK(cudaMemcpyAsync(ctx->d_Vh0, Vhat, sizeof(double) * ctx->ntrace, cudaMemcpyDeviceToDevice, s));
  int rc = HDG_OK;
  if (w.params) {
    HDG_REQUIRE(w.feat_mean && w.feat_std && w.tmean && w.tscale, "hdg_newton_step: incomplete network");
    HDG_REQUIRE(w.nin == 4 * ctx->NFN * ctx->M && w.nout == ctx->NFN * ctx->M,
                "hdg_newton_step: network sizes do not match the mesh (nin = 4 Nf m, nout = Nf m)");
    const int64_t need = ctx->F * (int64_t)std::max(w.nin, w.nout);
    if (ctx->feat_cap < need) {
      if (ctx->d_feat) cudaFree(ctx->d_feat);
      if (ctx->d_pred) cudaFree(ctx->d_pred);
      ctx->d_feat = ctx->d_pred = nullptr;
      ctx->feat_cap = 0;
      HDG_CK(cudaMalloc(&ctx->d_feat, sizeof(float) * need));
      HDG_CK(cudaMalloc(&ctx->d_pred, sizeof(float) * need));
      ctx->feat_cap = need;
    }
    if ((rc = hdg_mlp_features(ctx, V_n ? V_n : V, w.vhat_n, w.dvhat1, w.dvhat2, w.feat_mean, w.feat_std,
                               ctx->d_feat, stream)) ||
        (rc = hdg_mlp_forward(w.params, w.nin, w.nh, w.nout, ctx->d_feat, ctx->F, ctx->d_pred, stream)) ||
        (rc = hdg_mlp_apply_trace(ctx, w.vhat_n, w.dvhat1, ctx->d_pred, w.tmean, w.tscale, ctx->d_dVh, stream)))
      return rc;
    if ((rc = hdg::launch_axpby(ctx->ntrace, 1.0, ctx->d_dVh, -1.0, Vhat, ctx->d_dVh, s))) return rc;
  } else {
    HDG_CK(cudaMemsetAsync(ctx->d_dVh, 0, sizeof(double) * ctx->ntrace, s));
  }
  HDG_CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t) * ctx->E, s));
  if ((rc = hdg_assemble_condense(ctx, V, Vhat, hist, mass, precision, ctx->d_S, ctx->d_g, ctx->d_recov, ctx->d_R,
                                  ctx->d_status, stream)) ||
      (rc = hdg::launch_recover(ctx, ctx->d_recov, ctx->d_dVh, ctx->d_dV, s)) ||
      (rc = hdg::launch_axpy(nV, 1.0, ctx->d_dV, V, s)) || (rc = hdg::launch_axpy(ctx->ntrace, 1.0, ctx->d_dVh, Vhat, s)))
    return rc;
  rc = hdg_newton_solve(ctx, V, Vhat, hist, mass, precision, tol, max_newton, newton_iters, res_norm, res_history,
                        trace_iters, stream);
  if (rc == HDG_OK || rc == HDG_ERR_CUDA || rc == HDG_ERR_INVALID_ARG) return rc;
  // the plain solve from the caller's guess decides when the warm start fails
  HDG_CK(cudaMemcpyAsync(V, ctx->d_V0, sizeof(double) * nV, cudaMemcpyDeviceToDevice, s));
  HDG_CK(cudaMemcpyAsync(Vhat, ctx->d_Vh0, sizeof(double) * ctx->ntrace, cudaMemcpyDeviceToDevice, s));
  return hdg_newton_solve(ctx, V, Vhat, hist, mass, precision, tol, max_newton, newton_iters, res_norm, res_history,
                          trace_iters, stream);
}

namespace {

// Butcher tableau of Alexander's three-stage, third-order, L-stable DIRK(3,3): the diagonal g
// is the root in (1/6, 1/2) of g^3 - 3g^2 + 3g/2 - 1/6 = 0, c_2 = (1 + g)/2, the last row is
// b = (-(6g^2 - 16g + 1)/4, (6g^2 - 20g + 5)/4, g).
struct Dirk3 {
  double g, a21, a31, a32;
  Dirk3() {
    double lo = 1.0 / 6.0, hi = 0.5;  // f(lo) > 0 > f(hi)
    for (int i = 0; i < 200; ++i) {
      const double m = 0.5 * (lo + hi);
      const double f = ((m - 3.0) * m + 1.5) * m - 1.0 / 6.0;
      (f > 0.0 ? lo : hi) = m;
    }
    g = 0.5 * (lo + hi);
    a21 = 0.5 * (1.0 + g) - g;
    a31 = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0;
    a32 = (6.0 * g * g - 20.0 * g + 5.0) / 4.0;
  }
};

}  // namespace

extern "C" int hdg_dirk3_step(hdg_ctx_t ctx, double* V, double* Vhat, const double* V_n, double dt, int precision,
                              double tol, int max_newton, int* stage_iters, double* res_norm, int* trace_iters,
                              void* stream) {
  HDG_REQUIRE(ctx && V && Vhat && V_n && stage_iters && res_norm && dt > 0.0 && tol > 0.0 && max_newton >= 0,
              "hdg_dirk3_step: invalid argument");
  HDG_REQUIRE(precision == HDG_PREC_FP64 || precision == HDG_PREC_MIXED, "hdg_dirk3_step: precision");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = len_V(ctx);
  if (!ctx->d_hist) HDG_CK(cudaMalloc(&ctx->d_hist, sizeof(double) * n));
  if (!ctx->d_dirk) HDG_CK(cudaMalloc(&ctx->d_dirk, sizeof(double) * 4 * n));
  double *Un = ctx->d_dirk, *Ui = Un + n, *K1 = Ui + n, *K2 = K1 + n, *hist = ctx->d_hist;
  static const Dirk3 T;
  const double w = 1.0 / (dt * T.g);  // mass coefficient of every stage
  const double c[3][2] = {{0.0, 0.0}, {T.a21 / T.g, 0.0}, {T.a31 / T.g, T.a32 / T.g}};
  int rc = hdg::launch_history(ctx, V_n, nullptr, 1.0, 0.0, Un, s);  // (u_n, w)
  if (rc) return rc;
  if (trace_iters) *trace_iters = 0;
  for (int i = 0; i < 3; ++i) {
    // hist_i = (u_n, w)/(dt a_ii) + sum_{j<i} (a_ij / a_ii) (k_j, w)
    if ((rc = i == 0 ? hdg::launch_axpby(n, w, Un, 0.0, Un, hist, s)  // K1 is not yet written
                     : hdg::launch_axpby(n, w, Un, c[i][0], K1, hist, s)))
      return rc;
    if (i == 2 && (rc = hdg::launch_axpby(n, 1.0, hist, c[i][1], K2, hist, s))) return rc;
    int it = 0, tr = 0;
    rc = hdg_newton_solve(ctx, V, Vhat, hist, w, precision, tol, max_newton, &it, res_norm, nullptr, &tr, stream);
    stage_iters[i] = it;
    if (trace_iters) *trace_iters += tr;
    if (rc) return rc;
    if (i == 2) break;
    // (k_i, w) = (u_i - u_n, w)/(dt a_ii) - sum_{j<i} (a_ij / a_ii) (k_j, w)
    double* K = i == 0 ? K1 : K2;
    if ((rc = hdg::launch_history(ctx, V, nullptr, 1.0, 0.0, Ui, s)) ||
        (rc = hdg::launch_axpby(n, w, Ui, -w, Un, K, s)))
      return rc;
    if (i == 1 && (rc = hdg::launch_axpby(n, 1.0, K2, -c[1][0], K1, K2, s))) return rc;
  }
  return HDG_OK;
}

}  // extern "C"
