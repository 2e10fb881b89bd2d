// Dispatch of the mixed-precision assemble + condense (asm_tc.cuh, condense_tc.cuh).
#include <algorithm>
#include <vector>

#include "asm_tc.cuh"
#include "condense_t5.cuh"
#include "condense_tc.cuh"
#include "ctx.hpp"

namespace hdg {

namespace {

constexpr int kSlices = 6;  // exact bf16 slices per operand in every tensor-core product

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

// One compiled shape of the assembly products: MTC row tiles (16 MTC rows) per CTA, NJW
// column tiles per warp.
struct AsmVariant {
  int mtc, njw, threads;
  void (*run_vol)(const AssembleArgs&, const DevTablesDF&, cudaStream_t);
  void (*run_face)(const AssembleArgs&, const DevTables&, const DevTablesDF&, cudaStream_t);
  int (*set_attr)();
  void run(const AssembleArgs& a, const DevTables& T, const DevTablesDF& TD, cudaStream_t s) const {
    run_vol(a, TD, s);
    run_face(a, T, TD, s);
  }
};

template <class C, int MTC, int NJW>
void run_vol(const AssembleArgs& a, const DevTablesDF& TD, cudaStream_t s) {
  using Q = AsmTC<C, kSlices, MTC, NJW>;
  k_asm_vol_tc<C, kSlices, MTC, NJW><<<dim3(Q::NPASS, (unsigned)a.ne), Q::NTH, Q::vol_bytes, s>>>(a, TD);
}

template <class C, int MTC, int NJW>
void run_face(const AssembleArgs& a, const DevTables& T, const DevTablesDF& TD, cudaStream_t s) {
  using Q = AsmTC<C, kSlices, MTC, NJW>;
  k_asm_face_tc<C, kSlices, MTC, NJW><<<dim3(Q::NFCTA, (unsigned)a.ne), Q::NTH, Q::face_bytes, s>>>(a, T, TD);
}

template <class C, int MTC, int NJW>
int set_products_attr() {
  using Q = AsmTC<C, kSlices, MTC, NJW>;
  HDG_CK(cudaFuncSetAttribute(k_asm_vol_tc<C, kSlices, MTC, NJW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Q::vol_bytes));
  HDG_CK(cudaFuncSetAttribute(k_asm_face_tc<C, kSlices, MTC, NJW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Q::face_bytes));
  return HDG_OK;
}

template <class C, int MTC, int NJW>
AsmVariant make_variant() {
  return AsmVariant{MTC, NJW, AsmTC<C, kSlices, MTC, NJW>::NTH, &run_vol<C, MTC, NJW>, &run_face<C, MTC, NJW>,
                    &set_products_attr<C, MTC, NJW>};
}

// One compiled shape of the condensation kernel, with the prep kernel that lays out its operands.
struct CondVariant {
  int threads;
  size_t smem;
  void (*kernel)(AssembleArgs);
  int ctas_per_element;
  void (*prep)(AssembleArgs);
  unsigned grid(int64_t ne) const { return (unsigned)(ne * ctas_per_element); }
};

template <class C, int NTH>
CondVariant make_cond_variant() {
  return CondVariant{NTH, CondTC<C, NTH, kSlices>::bytes, &k_condense_tc<C, NTH, kSlices>, 1,
                     &k_condense_prep<C, kSlices, false>};
}

// 16-column blocks, two CTAs per SM
template <class C>
CondVariant make_cond_variant2() {
  return CondVariant{256, CondTC2<C, 256, kSlices>::bytes, &k_condense_tc2<C, 256, kSlices>, 2,
                     &k_condense_prep<C, kSlices, false>};
}

// tcgen05 products with TMEM accumulators, 32-column blocks, one CTA per SM
template <class C>
CondVariant make_cond_variant_t5() {
  using Q = CondT5<C, kSlices>;
  return CondVariant{Q::NTH, Q::bytes, &k_condense_t5<C, kSlices>, 1, &k_condense_prep<C, kSlices, true>};
}

// Times `launch` once on the stream (the chunk's outputs are rewritten each time).
template <class F>
int time_launch(cudaStream_t s, F launch, float* ms) {
  cudaEvent_t t0, t1;
  HDG_CK(cudaEventCreate(&t0));
  HDG_CK(cudaEventCreate(&t1));
  HDG_CK(cudaEventRecord(t0, s));
  launch();
  HDG_CK(cudaEventRecord(t1, s));
  HDG_CK(cudaEventSynchronize(t1));
  HDG_CK(cudaGetLastError());
  HDG_CK(cudaEventElapsedTime(ms, t0, t1));
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return HDG_OK;
}

template <class C>
int run_mixed(hdg_ctx* ctx, const double* V, const double* Vhat, const double* hist, double mass_coef, double* S,
              double* g, double* recov, double* R, int32_t* status, cudaStream_t s) {
  int rc = ensure_df_tables(ctx);
  if (rc) return rc;
  using TC = CondTC<C, 256, kSlices>;
  using AQ = AsmTC<C, kSlices, 2>;  // the operator slices do not depend on the row tiling
  const size_t per_pt = sizeof(double) * ((size_t)C::NG * C::PT_VOL + (size_t)C::NF * C::NGF * C::PT_FACE +
                                          (size_t)C::NV * C::NV + (size_t)C::NT * C::NV);
  const size_t slice_bytes = std::max(sizeof(uint4) * TC::slice_uint4, CondT5<C, kSlices>::slice_bytes);
  const size_t per = per_pt + slice_bytes + sizeof(float) * TC::prep_floats + sizeof(uint2) * AQ::rb_u2;
  if (ctx->chunk == 0) {
    int64_t ch = std::min<int64_t>(ctx->E, 8192);
    while (ch > 256 && per * ch > ((size_t)16 << 30)) ch /= 2;
    ctx->chunk = ch;
  }
  const size_t need = per * ctx->chunk + 1024;  // + room to align the slice, prep and operator scratch
  if (ctx->scr_bytes < need) {
    if (ctx->d_scr) cudaFree(ctx->d_scr);
    ctx->d_scr = nullptr;
    ctx->scr_bytes = 0;
    HDG_CK(cudaMalloc(&ctx->d_scr, need));
    ctx->scr_bytes = need;
  }
  // compiled tile shapes of the assembly kernel (threads, volume points per tile)
  const AsmVariant variants[] = {make_variant<C, 2, 4>(), make_variant<C, 4, 4>(), make_variant<C, 2, 2>(),
                                 make_variant<C, 4, 2>()};
  constexpr int NVAR = 4;
  const CondVariant cvariants[] = {make_cond_variant<C, 256>(), make_cond_variant<C, 512>(), make_cond_variant2<C>(),
                                   make_cond_variant_t5<C>()};
  constexpr int NCVAR = 4;
  if (!ctx->attr_mixed) {  // per context, hence per device
    for (const AsmVariant& v : variants)
      if (int rc2 = v.set_attr()) return rc2;
    for (const CondVariant& v : cvariants) {
      HDG_CK(cudaFuncSetAttribute(v.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem));
      HDG_CK(cudaFuncSetAttribute(v.kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    }
    HDG_CK(cudaFuncSetAttribute(k_condense_prep<C, kSlices, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TC::prep_bytes));
    HDG_CK(cudaFuncSetAttribute(k_condense_prep<C, kSlices, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TC::prep_bytes));
    // the FP64 kernels of the flagged-only recomputation
    HDG_CK(cudaFuncSetAttribute(k_assemble<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AsmSmem<C>::bytes));
    HDG_CK(cudaFuncSetAttribute(k_condense<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CondSmem<C>::bytes));
    ctx->attr_mixed = true;
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
  a.refine_tol = (float)ctx->refine_tol;
  a.stall_first_copy = ctx->t5_stall ? 1 : 0;
  const int64_t ch = ctx->chunk;
  a.ptv = ctx->d_scr;
  a.ptf = a.ptv + ch * C::NG * C::PT_VOL;
  a.Ap = a.ptf + ch * C::NF * C::NGF * C::PT_FACE;
  a.Cp = a.Ap + ch * C::NV * C::NV;
  {  // 256-byte aligned start of the slice scratch (chunk sizes may be odd)
    const uintptr_t p = reinterpret_cast<uintptr_t>(a.Cp + ch * C::NT * C::NV);
    a.oz = reinterpret_cast<uint4*>((p + 255) & ~(uintptr_t)255);
    const uintptr_t q = reinterpret_cast<uintptr_t>(a.oz) + ch * slice_bytes;
    a.prep = reinterpret_cast<float*>((q + 255) & ~(uintptr_t)255);
    const uintptr_t r = reinterpret_cast<uintptr_t>(a.prep + ch * TC::prep_floats);
    a.rb = reinterpret_cast<uint2*>((r + 255) & ~(uintptr_t)255);
  }
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
      launch_pointwise<C, df2>(a, ctx->T, ctx->ph, s);
    }
    {
      LaunchScope ls(ctx, HDG_KERNEL_MIXED_OPERATORS, s);
      k_asm_rb<C, kSlices, 2><<<(unsigned)a.ne, 256, 0, s>>>(a, ctx->T, TD);
    }
    {
      LaunchScope ls(ctx, HDG_KERNEL_MIXED_OPERATORS, s);
      k_asm_residual<C><<<(unsigned)a.ne, 128, 0, s>>>(a, ctx->T);
    }
    if ((ctx->asm_variant < 0 || ctx->face_variant < 0 || ctx->cond_variant < 0) && a.ne >= 512) {
      // autotune on this chunk: time every compiled shape (each rewrites the same outputs);
      // the volume and face products are tuned separately (the faces add to the volume's
      // output, so the volume runs again before each face trial)
      if (ctx->asm_variant < 0) {
        float best = 1e30f;
        int best_i = 0;
        for (int i = 0; i < NVAR; ++i) {
          float ms = 0.f;
          const AsmVariant& v = variants[i];
          int rc = time_launch(s, [&] { v.run_vol(a, TD, s); }, &ms);
          if (rc) return rc;
          if (ms < best) {
            best = ms;
            best_i = i;
          }
        }
        ctx->asm_variant = best_i;
        ctx->asm_variant_threads = variants[best_i].threads;
        ctx->asm_variant_gt = 16 * variants[best_i].mtc;
      }
      if (ctx->face_variant < 0) {
        float best = 1e30f;
        int best_i = 0;
        for (int i = 0; i < NVAR; ++i) {
          variants[ctx->asm_variant].run_vol(a, TD, s);
          float ms = 0.f;
          const AsmVariant& v = variants[i];
          int rc = time_launch(s, [&] { v.run_face(a, ctx->T, TD, s); }, &ms);
          if (rc) return rc;
          if (ms < best) {
            best = ms;
            best_i = i;
          }
        }
        ctx->face_variant = best_i;
      }
      if (ctx->cond_variant < 0) {
        const AsmVariant& vv = variants[ctx->asm_variant];
        const AsmVariant& vf = variants[ctx->face_variant];
        float best = 1e30f;
        int best_i = 0;
        for (int i = 0; i < NCVAR; ++i) {
          // the condensation overwrites its inputs: assemble again before each trial
          vv.run_vol(a, TD, s);
          vf.run_face(a, ctx->T, TD, s);
          const CondVariant& cv = cvariants[i];
          cv.prep<<<(unsigned)a.ne, TC::PTH, TC::prep_bytes, s>>>(a);
          float ms = 0.f;
          int rc = time_launch(s, [&] { cv.kernel<<<cv.grid(a.ne), cv.threads, cv.smem, s>>>(a); }, &ms);
          if (rc) return rc;
          if (ms < best) {
            best = ms;
            best_i = i;
          }
        }
        ctx->cond_variant = best_i;
        ctx->cond_variant_threads = cvariants[best_i].threads;
      }
    }
    {
      LaunchScope ls(ctx, HDG_KERNEL_MIXED_ASSEMBLE, s);
      variants[ctx->asm_variant < 0 ? 0 : ctx->asm_variant].run_vol(a, TD, s);
    }
    {
      LaunchScope ls(ctx, HDG_KERNEL_MIXED_FACE, s);
      variants[ctx->face_variant < 0 ? 0 : ctx->face_variant].run_face(a, ctx->T, TD, s);
    }
    if (int rc_b = boundary_patch(ctx, a, HDG_PREC_MIXED, s)) return rc_b;
    const CondVariant& cv = cvariants[ctx->cond_variant < 0 ? 0 : ctx->cond_variant];
    {
      LaunchScope ls(ctx, HDG_KERNEL_MIXED_PREP, s);
      cv.prep<<<(unsigned)a.ne, TC::PTH, TC::prep_bytes, s>>>(a);
    }
    {
      LaunchScope ls(ctx, HDG_KERNEL_MIXED_CONDENSE, s);
      cv.kernel<<<cv.grid(a.ne), cv.threads, cv.smem, s>>>(a);
    }
    if (ctx->refine_fallback) {
      // blocks whose refinement missed its tolerance (or whose condensation gave up a wait) are
      // recomputed by the FP64 kernels (the chunk's scratch is free again); every other CTA
      // returns at once
      AssembleArgs f = a;
      f.only_flag = HDG_STATUS_REFINE | HDG_STATUS_TIMEOUT;
      {
        LaunchScope ls(ctx, HDG_KERNEL_POINTWISE, s);
        launch_pointwise<C>(f, ctx->T, ctx->ph, s);
      }
      {
        LaunchScope ls(ctx, HDG_KERNEL_ASSEMBLE, s);
        k_assemble<C><<<(unsigned)a.ne, 256, AsmSmem<C>::bytes, s>>>(f, ctx->T);
      }
      if (int rc_b = boundary_patch(ctx, f, HDG_PREC_FP64, s)) return rc_b;
      {
        LaunchScope ls(ctx, HDG_KERNEL_CONDENSE, s);
        k_condense<C><<<(unsigned)a.ne, 256, CondSmem<C>::bytes, s>>>(f);
      }
    }
    if (int rc_d = chunk_done(ctx, e0, a.ne, s)) return rc_d;
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
