// Internal context shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hdg.h"
#include "hdg_device.cuh"
#include "mesh.hpp"
#include "pclass.hpp"

struct hdg_mesh {
  hdg::Mesh m;
};

struct hdg_ctx {
  hdg_mesh* mesh = nullptr;
  int device = 0;
  hdg::PhysParams ph{};
  bool visc = false;
  int dim = 0, p = 0, K = 0, M = 0, NP = 0, NFN = 0, NF = 0, NG = 0, NGF = 0, NV = 0, NT = 0, GEO = 0;
  int64_t E = 0, F = 0, ntrace = 0;
  int scheme = 0;            // 0: HDG (trace per face), 1: EDG (continuous trace, Sec. 3.4)
  int64_t n_tnodes = 0;      // trace nodes: F NFN (HDG) or skeleton nodes (EDG)
  int* d_tr_ptr = nullptr;   // [n_tnodes + 1] CSR of the local occurrences of each trace node
  int* d_tr_occ = nullptr;   // [E NF NFN] local occurrence e NF NFN + f NFN + c
  double* d_pcn = nullptr;   // EDG preconditioner: inverse node blocks [n_tnodes][M][M]
  // boundary faces (bounded meshes): (e NF + f, type) in ascending e, host and device copies;
  // the boundary state of the HDG_BC_STATE faces in the trace layout
  std::vector<int> h_bface;
  int* d_bface = nullptr;    // [nb] e NF + f
  int* d_bkind = nullptr;    // [nb] HDG_BC_*
  // EDG on a bounded mesh: every occurrence (e NF + f) NFN + c, ascending, of a trace node on a
  // BC_STATE face (the state is imposed strongly there), and which occurrence carries the node's
  // equation (the first)
  std::vector<int> h_dir;
  int* d_dir = nullptr;
  int* d_dir_first = nullptr;
  bool has_state_bc = false;
  double* d_vb = nullptr;    // [ntrace] (allocated when the state is first set)
  bool vb_set = false;
  // device tables
  double* d_tab = nullptr;
  size_t tab_size = 0;       // doubles in d_tab
  float* d_tab_df = nullptr; // the same tables as double-float pairs (mixed form)
  int* d_itab = nullptr;
  hdg::DevTables T{};
  int* d_tgidx = nullptr;    // [E][NF][NFN] canonical global face node of each local face node
  double* d_geo = nullptr;   // [E][GEO]
  int* d_fs_elem = nullptr;  // [F][2] element of each side (owner first; -1: boundary face)
  int* d_fs_loc = nullptr;   // [F][2][NFN] local face-node row (f*NFN + c) for canonical node
  // assembly scratch (chunked over elements)
  int64_t chunk = 0;
  double* d_scr = nullptr;
  size_t scr_bytes = 0;
  // autotuned tile shape of the mixed assembly (-1: not chosen yet)
  int asm_variant = -1, asm_variant_threads = 0, asm_variant_gt = 0;  // volume products
  int face_variant = -1;                                              // face products
  int cond_variant = -1, cond_variant_threads = 0;  // mixed condensation shape
  // solver scratch
  double* d_sw = nullptr;    // GMRES / matvec workspace
  size_t sw_bytes = 0;
  double* d_pc = nullptr;    // face-block Jacobi: inverse face blocks, transposed [F][B][B]
  double* d_dense = nullptr; // dense trace matrix for the direct solver
  int* d_dpiv = nullptr;
  size_t dense_n = 0;
  cudaGraphExec_t lu_graph_exec = nullptr;  // recorded pivot/scale/update sequence
  double* d_red = nullptr;   // reduction buffer (device)
  double* h_red = nullptr;   // pinned host mirror
  // streaming of S to host memory (hdg_assemble_condense_host): while `sink_host` is set, the
  // element chunks write S into a ring of device buffers in turn and each chunk's S is copied to
  // the host on `copy_stream` while the next chunks compute
  double* sink_host = nullptr;
  int sink_idx = 0;
  static constexpr int kSinkMax = 8;
  int sink_bufs = 4;       // device buffers in the ring (environment HDG_SINK_BUFFERS, 2..8)
  double* d_Sbuf[kSinkMax] = {};
  int64_t Sbuf_chunk = 0;  // elements per buffer
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_done[kSinkMax] = {}, ev_copied[kSinkMax] = {};
  // CUDA graph of one assemble + condense (hdg_assemble_condense_graph): the arguments and
  // library state it was captured with, and the launches it adds per replay
  struct GraphKey {
    const void* p[9] = {};
    double mass_coef = 0.0;
    int precision = -1;
    const void* scratch = nullptr;
    int64_t chunk = 0;
    bool operator==(const GraphKey& o) const {
      for (int i = 0; i < 9; ++i)
        if (p[i] != o.p[i]) return false;
      return mass_coef == o.mass_coef && precision == o.precision && scratch == o.scratch && chunk == o.chunk;
    }
  };
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t ac_graph = nullptr;
  GraphKey ac_key;
  int64_t ac_launches[HDG_KERNEL_CLASSES] = {0};
  bool ac_graph_failed = false;
  int64_t ac_replays = 0;  // graph launches so far (hdg_ctx_graph_replays)
  // Newton workspace
  double *d_S = nullptr, *d_g = nullptr, *d_recov = nullptr, *d_R = nullptr, *d_dV = nullptr, *d_dVh = nullptr;
  int32_t* d_status = nullptr;
  // time step (hdg_newton_step): BDF history, the entry state (plain start, kept for the
  // fallback of a failed warm start), MLP features and prediction
  double *d_hist = nullptr, *d_V0 = nullptr, *d_Vh0 = nullptr;
  double* d_dirk = nullptr;  // DIRK(3,3): (u_n, w), stage (u_i, w), weak stage derivatives k_1, k_2
  double* d_ent = nullptr;   // the two integrals of hdg_entropy_production
  float *d_feat = nullptr, *d_pred = nullptr;
  int64_t feat_cap = 0;
  // mixed form: refinement tolerance of the condensation's status bit and the FP64
  // recomputation of the blocks it flags (hdg_ctx_set_refinement)
  double refine_tol = 1e-10;
  bool refine_fallback = true;
  // test hook (environment HDG_T5_STALL_FIRST_COPY): k_condense_t5 never issues its first operand
  // copy, so its bounded waits run out and it reports HDG_ELEM_TIMEOUT
  bool t5_stall = false;
  // trace solver of the Newton iterations (hdg_ctx_set_trace_solver)
  int newton_solver = HDG_SOLVER_AUTO;
  double newton_rtol = 1e-12;
  int newton_max_it = 600;
  // dynamic shared-memory limits raised on this context's device (cudaFuncSetAttribute
  // applies per device; a context belongs to one device)
  bool attr_fp64 = false, attr_mixed = false, attr_noalloc = false, attr_matvec = false;
  int num_sms = 0;               // SMs of the device (persistent grids)
  hdg::PMix* pm = nullptr;       // mixed-degree mesh: class tables, packed layout, work queue
  int* d_mv_err = nullptr;       // set by the staged trace matvec when a copy wait gave up
  void* d_Sdf = nullptr;         // double-float copy of S for the GMRES products [E][NT][NT]
  // device-resident GMRES: the restart cycle's state (device and pinned host copies) and the CUDA
  // graph of one cycle's Arnoldi steps, with the pointers it was captured for
  void* d_gm = nullptr;
  void* h_gm = nullptr;
  cudaStream_t gm_stream = nullptr;
  cudaGraphExec_t gm_graph = nullptr;
  const void* gm_key[6] = {};
  bool gm_graph_failed = false;
  int64_t gm_cycles = 0, gm_replays = 0;  // cycles run, of them by graph replay
  size_t sdf_bytes = 0;
  bool sdf_unavailable = false;  // no device memory for it: FP64 products throughout
  // measurement: launch counts per kernel class and (when enabled) event pairs
  bool prof = false;
  int64_t launches[HDG_KERNEL_CLASSES] = {0};
  struct EvRec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<EvRec> pending;
  double prof_ms[HDG_KERNEL_CLASSES] = {0};
  int64_t prof_n[HDG_KERNEL_CLASSES] = {0};
};

namespace hdg {

void set_error(const std::string& msg);
int cuda_fail(cudaError_t err, const char* what);

#define HDG_CK(call)                                           \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return ::hdg::cuda_fail(_e, #call); \
  } while (0)

// Launch bracketing for the measurement hooks (see hdg_profile_read).
struct LaunchScope {
  hdg_ctx* c;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  LaunchScope(hdg_ctx* ctx, int k, cudaStream_t st) : c(ctx), cls(k), s(st) {
    c->launches[cls]++;
    if (c->prof) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, s);
    }
  }
  ~LaunchScope() {
    if (a) {
      cudaEventRecord(b, s);
      c->pending.push_back({cls, a, b});
    }
  }
};

// Chunk loops of assemble + condense: the S array a chunk [e0, e0 + ne) writes (indexed by the
// global element, as the kernels do), and the end of the chunk's launches (capi.cu).
double* chunk_S(hdg_ctx* ctx, double* S, int64_t e0, cudaStream_t s, int* rc);
int chunk_done(hdg_ctx* ctx, int64_t e0, int64_t ne, cudaStream_t s);

// assemble + condense (assemble_fp64.cu / assemble_mixed.cu)
int assemble_condense_fp64(hdg_ctx* ctx, const double* V, const double* Vhat, const double* hist, double mass_coef,
                           double* S, double* g, double* recov, double* R, int32_t* status, cudaStream_t s);
int assemble_condense_mixed(hdg_ctx* ctx, const double* V, const double* Vhat, const double* hist,
                            double mass_coef, double* S, double* g, double* recov, double* R, int32_t* status,
                            cudaStream_t s);
bool config_supported(int dim, int p, int K, bool visc);
struct AssembleArgs;  // assemble_fp64.cuh
// the boundary term of the chunk's boundary faces, written over the interior-face rows the
// element assembly left in R_t, C and D (boundary.cu); precision selects the output form
int boundary_patch(hdg_ctx* ctx, const AssembleArgs& a, int precision, cudaStream_t s);
// int rho s and the physical entropy production of Eq. PiS added into acc[0], acc[1]
int entropy_terms(hdg_ctx* ctx, const double* V, const double* Vhat, double* acc, cudaStream_t s);

// trace-space and element helpers (trace.cu)
int launch_prim_to_entropy(hdg_ctx* ctx, const double* prim, int64_t n, double* v, cudaStream_t s);
int launch_history(hdg_ctx* ctx, const double* V0, const double* V1, double c0, double c1, double* hist,
                   cudaStream_t s);
int launch_source_weak(hdg_ctx* ctx, const double* src, double c, double* hist, cudaStream_t s);
int launch_trace_matvec(hdg_ctx* ctx, const double* S, const double* x, double* y, double* work, cudaStream_t s,
                        const int* skip = nullptr);
int launch_trace_rhs(hdg_ctx* ctx, const double* g, double* rhs, cudaStream_t s);
int launch_recover(hdg_ctx* ctx, const double* recov, const double* dVhat, double* dV, cudaStream_t s);
int residual_norm(hdg_ctx* ctx, const double* R, double* norm, cudaStream_t s);
int trace_solve(hdg_ctx* ctx, const double* S, const double* g, double* dVhat, int method, double rtol, int max_it,
                int* iters, double* final_res, cudaStream_t s);
int launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s);
int launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s);

}  // namespace hdg
