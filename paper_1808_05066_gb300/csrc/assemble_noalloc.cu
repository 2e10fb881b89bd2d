// hdg_assemble_condense_noalloc: the FP64 assemble + condense with its scratch in a
// fixed, statically allocated device array instead of memory the library allocates.
//
// Who needs it: callers that may not allocate device memory at call time, for example
// runtimes that hand the library a fixed memory arena and forbid any further
// cudaMalloc/cudaFree (the arena owner accounts for every byte), or latency-critical loops
// where an allocation and the implicit device synchronisation of cudaFree are not
// acceptable. The ordinary entry point sizes its scratch lazily with cudaMalloc; this one
// never calls cudaMalloc, cudaFree or any allocating library routine.
//
// The scratch is one array of kNoAllocScratchBytes (64 MiB) in this translation unit's
// device memory, present on every GPU that loads the library until the process exits.
// Elements are processed in chunks sized to fit it; the per-element scratch of a
// configuration must fit at least once, otherwise the call is rejected with
// HDG_ERR_INVALID_ARG. Host code cannot use the array's name as a device address, so the
// first call on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it for the life of the process; a device reset
// (cudaDeviceReset) discards the module holding the array, so calls after one are invalid.
// All calls share the array: two calls whose kernels overlap on the GPU (different
// streams without ordering) race on it. Every byte a kernel reads from the array is
// written earlier in the same chunk, so nothing needs clearing between calls.
#include <algorithm>
#include <mutex>

#include "assemble_fp64.cuh"
#include "ctx.hpp"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Per-device set-up: resolve the array's device address (the device must be current).
int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) {
    hdg::set_error("hdg_assemble_condense_noalloc: device index out of range");
    return HDG_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return hdg::cuda_fail(err, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return HDG_OK;
}

template <class C>
int run_noalloc(hdg_ctx* ctx, double* scratch, const double* V, const double* Vhat, const double* hist,
                double mass_coef, double* S, double* g, double* recov, double* R, int32_t* status, cudaStream_t s) {
  using namespace hdg;
  const size_t per = (size_t)C::NG * C::PT_VOL + (size_t)C::NF * C::NGF * C::PT_FACE + (size_t)C::NV * C::NV +
                     (size_t)C::NT * C::NV;  // doubles per element
  const int64_t ch = std::min<int64_t>(ctx->E, (int64_t)(kNoAllocScratchBytes / sizeof(double) / per));
  if (ch < 1) {
    set_error("hdg_assemble_condense_noalloc: one element needs more scratch than the 64 MiB static array");
    return HDG_ERR_INVALID_ARG;
  }
  if (!ctx->attr_noalloc) {  // this file's instances of the kernels, once per context (one device)
    HDG_CK(cudaFuncSetAttribute(k_assemble<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AsmSmem<C>::bytes));
    HDG_CK(cudaFuncSetAttribute(k_condense<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CondSmem<C>::bytes));
    ctx->attr_noalloc = true;
  }
  AssembleArgs a{};
  a.V = V;
  a.Vhat = Vhat;
  a.tgidx = ctx->d_tgidx;
  a.geo = ctx->d_geo;
  a.hist = hist;
  a.mass_coef = mass_coef;
  a.S = S;
  a.g = g;
  a.recov = recov;
  a.R = R;
  a.status = status;
  a.ptv = scratch;
  a.ptf = a.ptv + ch * C::NG * C::PT_VOL;
  a.Ap = a.ptf + ch * C::NF * C::NGF * C::PT_FACE;
  a.Cp = a.Ap + ch * C::NV * C::NV;
  for (int64_t e0 = 0; e0 < ctx->E; e0 += ch) {
    a.e0 = e0;
    a.ne = std::min<int64_t>(ch, ctx->E - e0);
    launch_pointwise<C>(a, ctx->T, ctx->ph, s);
    k_assemble<C><<<(unsigned)a.ne, 256, AsmSmem<C>::bytes, s>>>(a, ctx->T);
    if (int rc_b = boundary_patch(ctx, a, HDG_PREC_FP64, s)) return rc_b;
    k_condense<C><<<(unsigned)a.ne, 256, CondSmem<C>::bytes, s>>>(a);
  }
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

}  // namespace

#define HDG_NOALLOC_CASE(D, P, VISC)                                                                  \
  if (ctx->dim == D && ctx->p == P && ctx->K == P + 1 && ctx->visc == VISC)                          \
    return run_noalloc<hdg::Cfg<D, P, P + 1, VISC>>(ctx, scratch, V, Vhat, hist, mass_coef, S, g, recov, R, \
                                                    elem_status, s);

extern "C" int hdg_assemble_condense_noalloc(hdg_ctx_t ctx, const double* V, const double* Vhat, const double* hist,
                                             double mass_coef, double* S, double* g, double* recov, double* R,
                                             int32_t* elem_status, void* stream) {
  if (!ctx || !V || !Vhat || !S || !g || !recov || !R || !elem_status) {
    hdg::set_error("hdg_assemble_condense_noalloc: null argument (elem_status is required)");
    return HDG_ERR_INVALID_ARG;
  }
  if (ctx->pm) {
    hdg::set_error("hdg_assemble_condense_noalloc: not built for meshes of mixed degree");
    return HDG_ERR_UNSUPPORTED;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) {
    hdg::set_error("hdg_assemble_condense_noalloc: cannot make the context's device current");
    return HDG_ERR_CUDA;
  }
  double* scratch = nullptr;
  int rc = noalloc_scratch(ctx->device, &scratch);
  cudaStream_t s = (cudaStream_t)stream;
  if (rc == HDG_OK) {
    rc = [&]() -> int {
      HDG_NOALLOC_CASE(2, 1, false)
      HDG_NOALLOC_CASE(2, 2, false)
      HDG_NOALLOC_CASE(2, 3, false)
      HDG_NOALLOC_CASE(2, 4, false)
      HDG_NOALLOC_CASE(2, 1, true)
      HDG_NOALLOC_CASE(2, 2, true)
      HDG_NOALLOC_CASE(2, 3, true)
      HDG_NOALLOC_CASE(2, 4, true)
      HDG_NOALLOC_CASE(3, 1, true)
      HDG_NOALLOC_CASE(3, 2, true)
      HDG_NOALLOC_CASE(3, 3, true)
      hdg::set_error("hdg_assemble_condense_noalloc: configuration not compiled in");
      return HDG_ERR_UNSUPPORTED;
    }();
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return rc;
}
