// Dispatch of the mixed-precision assemble + condense (see assemble_mixed.cuh).
#include <algorithm>
#include <vector>

#include "assemble_mixed.cuh"
#include "ctx.hpp"

namespace hdg {

namespace {

constexpr int kThreads = 256;
constexpr int kRefine = 2;

int ensure_df_tables(hdg_ctx* ctx) {
  if (ctx->d_tab_df) return HDG_OK;
  // double-float copies of the reference tables, converted on the device-independent host
  const size_t n_total = ctx->tab_size;
  std::vector<double> h(n_total);
  HDG_CK(cudaMemcpy(h.data(), ctx->d_tab, sizeof(double) * n_total, cudaMemcpyDeviceToHost));
  std::vector<float> hd(2 * n_total);
  for (size_t i = 0; i < n_total; ++i) {
    float hi = (float)h[i];
    float lo = (float)(h[i] - (double)hi);
    hd[2 * i] = hi;
    hd[2 * i + 1] = lo;
  }
  HDG_CK(cudaMalloc(&ctx->d_tab_df, sizeof(float) * hd.size()));
  HDG_CK(cudaMemcpy(ctx->d_tab_df, hd.data(), sizeof(float) * hd.size(), cudaMemcpyHostToDevice));
  return HDG_OK;
}

// One compiled tile shape of the mixed assembly kernel.
struct AsmVariant {
  int threads, gt;
  size_t smem;
  void (*kernel)(AssembleArgs, DevTables, DevTablesDF);
};

template <class C, int NTH, int GTM>
AsmVariant make_variant() {
  return AsmVariant{NTH, GTM, MixCfg<C, NTH, GTM>::asm_bytes, &k_assemble_df<C, NTH, GTM>};
}

template <class C>
int run_mixed(hdg_ctx* ctx, const double* V, const double* Vhat, const double* hist, double mass_coef, double* S,
              double* g, double* recov, double* R, int32_t* status, cudaStream_t s) {
  int rc = ensure_df_tables(ctx);
  if (rc) return rc;
  const size_t per = sizeof(double) * ((size_t)C::NG * C::PT_VOL + (size_t)C::NF * C::NGF * C::PT_FACE +
                                       (size_t)C::NV * C::NV + (size_t)C::NT * C::NV);
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
  // compiled tile shapes of the assembly kernel (threads, volume points per tile)
  const AsmVariant variants[] = {make_variant<C, 256, 64>(), make_variant<C, 256, 32>(),
                                 make_variant<C, 512, 64>(), make_variant<C, 128, 16>()};
  constexpr int NVAR = 4;
  static bool attr_done = false;
  if (!attr_done) {
    for (const AsmVariant& v : variants)
      HDG_CK(cudaFuncSetAttribute(v.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem));
    HDG_CK(cudaFuncSetAttribute(k_condense_df<C, kThreads, kRefine>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)CondCfg<C, kThreads>::bytes));
    attr_done = true;
  }
  const df2* td = reinterpret_cast<const df2*>(ctx->d_tab_df);
  DevTablesDF TD;
  TD.Phi = td + (ctx->T.Phi - ctx->d_tab);
  TD.dPhi = td + (ctx->T.dPhi - ctx->d_tab);
  TD.PL = td + (ctx->T.PL - ctx->d_tab);
  TD.PhiF = td + (ctx->T.PhiF - ctx->d_tab);
  TD.dPhiF = td + (ctx->T.dPhiF - ctx->d_tab);
  TD.PLF = td + (ctx->T.PLF - ctx->d_tab);
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
  const int pw_threads = ((C::NG + C::NF * C::NGF + 31) / 32) * 32;
  for (int64_t e0 = 0; e0 < ctx->E; e0 += ch) {
    a.e0 = e0;
    a.ne = std::min<int64_t>(ch, ctx->E - e0);
    {
      LaunchScope ls(ctx, HDG_KERNEL_POINTWISE, s);
      k_pointwise<C, df2><<<(unsigned)a.ne, pw_threads, 0, s>>>(a, ctx->T, ctx->ph);
    }
    if (ctx->asm_variant < 0 && a.ne >= 512) {
      // autotune on this chunk: time every compiled shape (each writes the same outputs)
      float best = 1e30f;
      int best_i = 0;
      cudaEvent_t t0, t1;
      HDG_CK(cudaEventCreate(&t0));
      HDG_CK(cudaEventCreate(&t1));
      for (int i = 0; i < NVAR; ++i) {
        HDG_CK(cudaEventRecord(t0, s));
        variants[i].kernel<<<(unsigned)a.ne, variants[i].threads, variants[i].smem, s>>>(a, ctx->T, TD);
        HDG_CK(cudaEventRecord(t1, s));
        HDG_CK(cudaEventSynchronize(t1));
        HDG_CK(cudaGetLastError());
        float ms = 0.f;
        HDG_CK(cudaEventElapsedTime(&ms, t0, t1));
        if (ms < best) {
          best = ms;
          best_i = i;
        }
      }
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      ctx->asm_variant = best_i;
      ctx->asm_variant_threads = variants[best_i].threads;
      ctx->asm_variant_gt = variants[best_i].gt;
    }
    const AsmVariant& v = variants[ctx->asm_variant < 0 ? 0 : ctx->asm_variant];
    {
      LaunchScope ls(ctx, HDG_KERNEL_MIXED_ASSEMBLE, s);
      v.kernel<<<(unsigned)a.ne, v.threads, v.smem, s>>>(a, ctx->T, TD);
    }
    {
      LaunchScope ls(ctx, HDG_KERNEL_MIXED_CONDENSE, s);
      k_condense_df<C, kThreads, kRefine><<<(unsigned)a.ne, kThreads, CondCfg<C, kThreads>::bytes, s>>>(a);
    }
  }
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

}  // namespace

#define HDG_MIX_CASE(D, P, VISC)                                                                    \
  if (ctx->dim == D && ctx->p == P && ctx->K == P + 1 && ctx->visc == VISC)                        \
    return run_mixed<Cfg<D, P, P + 1, VISC>>(ctx, V, Vhat, hist, mass_coef, S, g, recov, R, status, s);

int assemble_condense_mixed(hdg_ctx* ctx, const double* V, const double* Vhat, const double* hist,
                            double mass_coef, double* S, double* g, double* recov, double* R, int32_t* status,
                            cudaStream_t s) {
  HDG_MIX_CASE(2, 2, false)
  HDG_MIX_CASE(2, 3, true)
  HDG_MIX_CASE(2, 4, true)
  HDG_MIX_CASE(3, 1, true)
  HDG_MIX_CASE(3, 2, true)
  HDG_MIX_CASE(3, 3, true)
  set_error("assemble_condense: mixed form not compiled for this configuration");
  return HDG_ERR_UNSUPPORTED;
}

}  // namespace hdg
