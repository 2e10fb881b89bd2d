// Dispatch of the plain FP64 assemble + condense kernels over the compiled element
// configurations, processing elements in chunks that share one scratch buffer.
#include <algorithm>

#include "assemble_fp64.cuh"
#include "ctx.hpp"

namespace hdg {

namespace {

template <class C>
size_t scratch_per_element() {
  return sizeof(double) * ((size_t)C::NG * C::PT_VOL + (size_t)C::NF * C::NGF * C::PT_FACE +
                           (size_t)C::NV * C::NV + (size_t)C::NT * C::NV);
}

template <class C>
int run_fp64(hdg_ctx* ctx, const double* V, const double* Vhat, const double* hist, double mass_coef, double* S,
             double* g, double* recov, double* R, int32_t* status, cudaStream_t s) {
  const size_t per = scratch_per_element<C>();
  if (ctx->chunk == 0) {
    int64_t ch = std::min<int64_t>(ctx->E, 8192);
    while (ch > 256 && per * ch > ((size_t)3 << 30)) ch /= 2;
    ctx->chunk = ch;
  }
  const size_t need = per * ctx->chunk;
  if (ctx->scr_bytes < need) {
    if (ctx->d_scr) cudaFree(ctx->d_scr);
    ctx->d_scr = nullptr;
    ctx->scr_bytes = 0;
    HDG_CK(cudaMalloc(&ctx->d_scr, need));
    ctx->scr_bytes = need;
  }
  if (!ctx->attr_fp64) {  // per context, hence per device
    HDG_CK(cudaFuncSetAttribute(k_assemble<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AsmSmem<C>::bytes));
    HDG_CK(cudaFuncSetAttribute(k_condense<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CondSmem<C>::bytes));
    ctx->attr_fp64 = true;
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
  const int64_t ch = ctx->chunk;
  a.ptv = ctx->d_scr;
  a.ptf = a.ptv + ch * C::NG * C::PT_VOL;
  a.Ap = a.ptf + ch * C::NF * C::NGF * C::PT_FACE;
  a.Cp = a.Ap + ch * C::NV * C::NV;
  for (int64_t e0 = 0; e0 < ctx->E; e0 += ch) {
    a.e0 = e0;
    a.ne = std::min<int64_t>(ch, ctx->E - e0);
    {
      int rc_s = HDG_OK;
      a.S = chunk_S(ctx, S, e0, s, &rc_s);
      if (rc_s) return rc_s;
    }
    {
      LaunchScope ls(ctx, HDG_KERNEL_POINTWISE, s);
      launch_pointwise<C>(a, ctx->T, ctx->ph, s);
    }
    {
      LaunchScope ls(ctx, HDG_KERNEL_ASSEMBLE, s);
      k_assemble<C><<<(unsigned)a.ne, 256, AsmSmem<C>::bytes, s>>>(a, ctx->T);
    }
    if (int rc_b = boundary_patch(ctx, a, HDG_PREC_FP64, s)) return rc_b;
    {
      LaunchScope ls(ctx, HDG_KERNEL_CONDENSE, s);
      k_condense<C><<<(unsigned)a.ne, 256, CondSmem<C>::bytes, s>>>(a);
    }
    if (int rc_d = chunk_done(ctx, e0, a.ne, s)) return rc_d;
  }
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

template <class C>
int run_entropy(hdg_ctx* ctx, const double* V, const double* Vhat, double* acc, cudaStream_t s) {
  AssembleArgs a{};
  a.V = V;
  a.Vhat = Vhat;
  a.tgidx = ctx->d_tgidx;
  a.geo = ctx->d_geo;
  a.e0 = 0;
  a.ne = ctx->E;
  LaunchScope ls(ctx, HDG_KERNEL_OTHER, s);
  k_entropy_terms<C><<<(unsigned)ctx->E, 128, 0, s>>>(a, ctx->T, ctx->ph, acc);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

}  // namespace

#define HDG_ENTROPY_CASE(D, P, VISC)                                          \
  if (ctx->dim == D && ctx->p == P && ctx->K == P + 1 && ctx->visc == VISC) \
    return run_entropy<Cfg<D, P, P + 1, VISC>>(ctx, V, Vhat, acc, s);

int entropy_terms(hdg_ctx* ctx, const double* V, const double* Vhat, double* acc, cudaStream_t s) {
  HDG_ENTROPY_CASE(2, 1, false)
  HDG_ENTROPY_CASE(2, 2, false)
  HDG_ENTROPY_CASE(2, 3, false)
  HDG_ENTROPY_CASE(2, 4, false)
  HDG_ENTROPY_CASE(2, 1, true)
  HDG_ENTROPY_CASE(2, 2, true)
  HDG_ENTROPY_CASE(2, 3, true)
  HDG_ENTROPY_CASE(2, 4, true)
  HDG_ENTROPY_CASE(3, 1, true)
  HDG_ENTROPY_CASE(3, 2, true)
  HDG_ENTROPY_CASE(3, 3, true)
  set_error("entropy_terms: configuration not compiled in");
  return HDG_ERR_UNSUPPORTED;
}

#define HDG_FP64_CASE(D, P, VISC)                                                                       \
  if (ctx->dim == D && ctx->p == P && ctx->K == P + 1 && ctx->visc == VISC)                            \
    return run_fp64<Cfg<D, P, P + 1, VISC>>(ctx, V, Vhat, hist, mass_coef, S, g, recov, R, status, s);

int assemble_condense_fp64(hdg_ctx* ctx, const double* V, const double* Vhat, const double* hist, double mass_coef,
                           double* S, double* g, double* recov, double* R, int32_t* status, cudaStream_t s) {
  HDG_FP64_CASE(2, 1, false)
  HDG_FP64_CASE(2, 2, false)
  HDG_FP64_CASE(2, 3, false)
  HDG_FP64_CASE(2, 4, false)
  HDG_FP64_CASE(2, 1, true)
  HDG_FP64_CASE(2, 2, true)
  HDG_FP64_CASE(2, 3, true)
  HDG_FP64_CASE(2, 4, true)
  HDG_FP64_CASE(3, 1, true)
  HDG_FP64_CASE(3, 2, true)
  HDG_FP64_CASE(3, 3, true)
  set_error("assemble_condense: configuration not compiled in");
  return HDG_ERR_UNSUPPORTED;
}

bool config_supported(int dim, int p, int K, bool visc) {
  if (K != p + 1) return false;
  if (dim == 2) return p >= 1 && p <= 4;
  if (dim == 3) return visc && p >= 1 && p <= 3;
  return false;
}

}  // namespace hdg
