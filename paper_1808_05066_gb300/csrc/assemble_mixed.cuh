// Mixed-precision assemble + condense.
//
// Same mathematics as the FP64 form (assemble_fp64.cuh), arranged for GB300's pipes:
//   * pointwise fluxes and Jacobians: FP64 (k_pointwise), stored as double-floats;
//   * quadrature contractions for A', B', C', D': double-float multiply-accumulate on
//     the FP32 pipe, each thread accumulating a strip of JW outputs in registers;
//   * LU with partial pivoting in FP32 (shared memory) of the equilibrated matrix
//     D^{-1/2} A' D^{-1/2}, D = |diag A'|: at low Mach the state components differ by
//     orders of magnitude and A' has condition numbers ~1e6 (3D, M = 0.1), which the
//     symmetric diagonal scaling brings to ~1e2, within reach of FP32 refinement;
//   * X = A'^{-1} [B' | R_v]: FP32 triangular solves, then NREF sweeps of iterative
//     refinement  r = B' - A' X (double-float), X += D^{-1/2} LU^{-1} D^{-1/2} r (FP32);
//   * S = D' - C' X and g = R_t - C' y: double-float.
// The result agrees with the FP64 oracle to ~1e-12 relative (double-float carries
// ~48 bits; refinement removes the FP32 factorisation error).
#pragma once
#include "assemble_fp64.cuh"
#include "dfloat.cuh"

namespace hdg {

struct DevTablesDF {
  const df2* Phi;    // [NG][NP]
  const df2* dPhi;   // [D][NG][NP]
  const df2* PL;     // [NF][NG][NFN]
  const df2* PhiF;   // [NF][NGF][NP]
  const df2* dPhiF;  // [NF][D][NGF][NP]
  const df2* PLF;    // [NF][NF][NGF][NFN]
};

template <class C, int NTHREADS>
struct MixCfg {
  static constexpr int GT = C::NG < 64 ? C::NG : 64;
  static constexpr int JW = (C::NP * C::NZ + NTHREADS - 1) / NTHREADS;    // outputs per thread (volume)
  static constexpr int NSV = (C::NZ + JW - 1) / JW;                       // strips per row
  static constexpr int JWF = (C::NFN * C::NZ + NTHREADS - 1) / NTHREADS;  // faces
  static constexpr int NSF = (C::NZ + JWF - 1) / JWF;
  static constexpr int RB = C::NR * GT * C::NZ;
  static constexpr int RBF = C::NRF * C::NGF * C::NZ;
  static constexpr int RBMAX = RB > RBF ? RB : RBF;
  static constexpr int ZS = C::NP * GT * C::NR;
  static constexpr int ZSF = C::NFN * C::NGF * C::NRF;
  static constexpr int ZSMAX = ZS > ZSF ? ZS : ZSF;
  static constexpr size_t asm_bytes =
      sizeof(df2) * (RBMAX + ZSMAX + C::D * C::D + C::NF * C::D) + sizeof(double) * (C::NZ * C::M + C::GEO + C::NV + C::NT);
  // condense
  static constexpr int CB = 32;
  static constexpr size_t cond_bytes = sizeof(df2) * (C::NV * C::NV + 2 * C::NV * CB) +
                                       sizeof(float) * (C::NV * C::NV + C::NV * CB + C::NV) + sizeof(int) * C::NV + 64;
};

// ------------------------------------------------------------------------------------
// k_assemble_df: one CTA per element
// ------------------------------------------------------------------------------------
template <class C, int NTHREADS>
__global__ void __launch_bounds__(NTHREADS) k_assemble_df(AssembleArgs a, DevTables T, DevTablesDF TD) {
  constexpr int D = C::D, M = C::M, NP = C::NP, NFN = C::NFN, NF = C::NF, NG = C::NG, NGF = C::NGF;
  constexpr int NZ = C::NZ, NV = C::NV, NT = C::NT, NR = C::NR, NRF = C::NRF;
  using X = MixCfg<C, NTHREADS>;
  constexpr int GT = X::GT, JW = X::JW, NSV = X::NSV, JWF = X::JWF, NSF = X::NSF;
  extern __shared__ double smem_d[];
  df2* Rb = reinterpret_cast<df2*>(smem_d);
  df2* Zs = Rb + X::RBMAX;
  df2* JiD = Zs + X::ZSMAX;          // [D][D] Jinv as double-float
  df2* NsD = JiD + D * D;            // [NF][D] n_f s_f
  double(*z)[M] = reinterpret_cast<double(*)[M]>(NsD + NF * D);
  double* G = reinterpret_cast<double*>(z) + NZ * M;
  double* Rv = G + C::GEO;
  double* Rt = Rv + NV;
  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x;
  load_element<C>(a, e, z, G);
  __syncthreads();
  const double detJ = G[D * D];
  if (tid < D * D) JiD[tid] = df_from(G[tid]);
  if (tid < NF * D) {
    int f = tid / D, k = tid % D;
    const double* Gf = G + D * D + 1 + f * (D + 1);
    NsD[tid] = df_from(Gf[k] * (Gf[D] / detJ));
  }
  double* Ap = a.Ap + le * NV * NV;
  df2* Cp = reinterpret_cast<df2*>(a.Cp) + le * NT * NV;
  double* Bp = a.recov + e * (int64_t)(NV * NT + NV);
  double* Dp = a.S + e * (int64_t)NT * NT;
  const df2* ptv = reinterpret_cast<const df2*>(a.ptv) + le * NG * C::PT_VOL;
  const df2* ptf = reinterpret_cast<const df2*>(a.ptf) + le * NF * NGF * C::PT_FACE;

  // residual R_v, volume part (FP64 from double-float point data)
  for (int t = tid; t < NV; t += NTHREADS) {
    int an = t / M, i = t % M;
    double s = a.hist ? -a.hist[e * NV + t] : 0.0;
    for (int g = 0; g < NG; ++g) {
      const df2* P = ptv + g * C::PT_VOL;
      s += T.Phi[g * NP + an] * df_val(P[i]);
      for (int r = 0; r < D; ++r) s += T.dPhi[(r * NG + g) * NP + an] * df_val(P[M + r * M + i]);
    }
    Rv[t] = s;
  }
  __syncthreads();

  // ---------------- volume contractions ----------------
  for (int g0 = 0; g0 < NG; g0 += GT) {
    const int ng = (NG - g0) < GT ? (NG - g0) : GT;
    __syncthreads();
    for (int t = tid; t < NR * GT * NZ; t += NTHREADS) {
      int beta = t / (GT * NZ), gg = (t / NZ) % GT, j = t % NZ;
      df2 val = {0.f, 0.f};
      if (gg < ng) {
        int g = g0 + gg;
        if (beta == 0) {
          if (j < NP) val = TD.Phi[g * NP + j];
        } else {
          int k = beta - 1;
          dfacc acc;
          if (j < NP) {
            for (int r = 0; r < D; ++r) acc.mac(JiD[r * D + k], TD.dPhi[(r * NG + g) * NP + j]);
            for (int f = 0; f < NF; ++f) {
              int c = T.nodepos[f * NP + j];
              if (c >= 0) {
                df2 ns = NsD[f * D + k];
                ns.hi = -ns.hi;
                ns.lo = -ns.lo;
                acc.mac(ns, TD.PL[(f * NG + g) * NFN + c]);
              }
            }
          } else {
            int f = (j - NP) / NFN, c = (j - NP) % NFN;
            acc.mac(NsD[f * D + k], TD.PL[(f * NG + g) * NFN + c]);
          }
          val = acc.norm();
        }
      }
      Rb[t] = val;
    }
    for (int il = 0; il < M * M; ++il) {
      const int i = il / M, l = il % M;
      __syncthreads();
      for (int t = tid; t < NP * GT * NR; t += NTHREADS) {
        int an = t / (GT * NR), gg = (t / NR) % GT, beta = t % NR;
        df2 val = {0.f, 0.f};
        if (gg < ng) {
          int g = g0 + gg;
          const df2* P = ptv + g * C::PT_VOL;
          const df2* T0 = P + M + D * M;
          const df2* T1 = T0 + M * M;
          const df2* T2 = T1 + D * M * M;
          dfacc acc;
          if (beta == 0) {
            acc.mac(TD.Phi[g * NP + an], T0[i * M + l]);
            for (int r = 0; r < D; ++r) acc.mac(TD.dPhi[(r * NG + g) * NP + an], T1[(r * M + i) * M + l]);
          } else {
            int k = beta - 1;
            for (int r = 0; r < D; ++r) acc.mac(TD.dPhi[(r * NG + g) * NP + an], T2[((r * M + i) * M + l) * D + k]);
          }
          val = acc.norm();
        }
        Zs[t] = val;
      }
      __syncthreads();
      if (tid < NP * NSV) {
        const int an = tid / NSV, j0 = (tid % NSV) * JW;
        const int b0 = j0 >= NP ? 1 : 0;
        dfacc acc[JW];
        for (int gg = 0; gg < ng; ++gg)
          for (int beta = b0; beta < NR; ++beta) {
            const df2 zv = Zs[(an * GT + gg) * NR + beta];
            const df2* rb = Rb + (beta * GT + gg) * NZ + j0;
#pragma unroll
            for (int jj = 0; jj < JW; ++jj)
              if (j0 + jj < NZ) acc[jj].mac(zv, rb[jj]);
          }
        const int row = an * M + i;
#pragma unroll
        for (int jj = 0; jj < JW; ++jj) {
          const int j = j0 + jj;
          if (j >= NZ) continue;
          const double v = acc[jj].value();
          double* dst = j < NP ? Ap + row * NV + j * M + l : Bp + row * NT + (j - NP) * M + l;
          *dst = (g0 == 0) ? v : *dst + v;
        }
      }
    }
  }

  // ---------------- face contractions ----------------
  for (int f = 0; f < NF; ++f) {
    __syncthreads();
    for (int t = tid; t < NRF * NGF * NZ; t += NTHREADS) {
      int beta = t / (NGF * NZ), gf = (t / NZ) % NGF, j = t % NZ;
      const df2* phif = TD.PhiF + (f * NGF + gf) * NP;
      df2 val = {0.f, 0.f};
      if (beta == 0) {
        if (j < NP) val = phif[j];
      } else if (beta == 1) {
        if (j >= NP && (j - NP) / NFN == f) val = phif[T.fnodes[f * NFN + (j - NP) % NFN]];
      } else {
        int k = beta - 2;
        dfacc acc;
        if (j < NP) {
          for (int r = 0; r < D; ++r) acc.mac(JiD[r * D + k], TD.dPhiF[((f * D + r) * NGF + gf) * NP + j]);
          for (int fl = 0; fl < NF; ++fl) {
            int c = T.nodepos[fl * NP + j];
            if (c >= 0) {
              df2 ns = NsD[fl * D + k];
              ns.hi = -ns.hi;
              ns.lo = -ns.lo;
              acc.mac(ns, TD.PLF[((f * NF + fl) * NGF + gf) * NFN + c]);
            }
          }
        } else {
          int fl = (j - NP) / NFN, c = (j - NP) % NFN;
          acc.mac(NsD[fl * D + k], TD.PLF[((f * NF + fl) * NGF + gf) * NFN + c]);
        }
        val = acc.norm();
      }
      Rb[t] = val;
    }
    __syncthreads();
    for (int t = tid; t < NFN * M; t += NTHREADS) {
      int c = t / M, i = t % M;
      double s = 0.0;
      for (int gf = 0; gf < NGF; ++gf) {
        double psi = T.PhiF[(f * NGF + gf) * NP + T.fnodes[f * NFN + c]];
        s += psi * df_val(ptf[(f * NGF + gf) * C::PT_FACE + i]);
      }
      Rv[T.fnodes[f * NFN + c] * M + i] += s;
      Rt[(f * NFN + c) * M + i] = s;
    }
    for (int il = 0; il < M * M; ++il) {
      const int i = il / M, l = il % M;
      __syncthreads();
      for (int t = tid; t < NFN * NGF * NRF; t += NTHREADS) {
        int c = t / (NGF * NRF), gf = (t / NRF) % NGF, beta = t % NRF;
        const df2* P = ptf + (f * NGF + gf) * C::PT_FACE;
        const df2* U0 = P + M;
        const df2* U1 = U0 + M * M;
        const df2* U2 = U1 + M * M;
        df2 psi = TD.PhiF[(f * NGF + gf) * NP + T.fnodes[f * NFN + c]];
        df2 u = beta == 0 ? U0[i * M + l] : (beta == 1 ? U1[i * M + l] : U2[(i * M + l) * D + (beta - 2)]);
        dfacc acc;
        acc.mac(psi, u);
        Zs[t] = acc.norm();
      }
      __syncthreads();
      if (tid < NFN * NSF) {
        const int c = tid / NSF, j0 = (tid % NSF) * JWF;
        dfacc acc[JWF];
        for (int gf = 0; gf < NGF; ++gf)
          for (int beta = 0; beta < NRF; ++beta) {
            const df2 zv = Zs[(c * NGF + gf) * NRF + beta];
            const df2* rb = Rb + (beta * NGF + gf) * NZ + j0;
#pragma unroll
            for (int jj = 0; jj < JWF; ++jj)
              if (j0 + jj < NZ) acc[jj].mac(zv, rb[jj]);
          }
        const int rowv = T.fnodes[f * NFN + c] * M + i;
        const int rowt = (f * NFN + c) * M + i;
#pragma unroll
        for (int jj = 0; jj < JWF; ++jj) {
          const int j = j0 + jj;
          if (j >= NZ) continue;
          const double v = acc[jj].value();
          if (j < NP) {
            Ap[rowv * NV + j * M + l] += v;
            Cp[rowt * NV + j * M + l] = df_from(v);
          } else {
            const int tcol = (j - NP) * M + l;
            Bp[rowv * NT + tcol] += v;
            Dp[rowt * NT + tcol] = v;
          }
        }
      }
    }
  }
  __syncthreads();
  double* Rout = a.R + e * (int64_t)(NV + NT);
  for (int t = tid; t < NV; t += NTHREADS) Rout[t] = Rv[t];
  for (int t = tid; t < NT; t += NTHREADS) Rout[NV + t] = Rt[t];
}

// ------------------------------------------------------------------------------------
// k_condense_df: one CTA per element
// ------------------------------------------------------------------------------------
template <int NV, int CB, int NTHREADS>
HDG_DEVI void lu_solve_f32(const float* LU, const int* piv, float* W) {
  // W [NV][CB] <- LU^{-1} W (row interchanges, unit lower, upper)
  for (int c = threadIdx.x; c < CB; c += NTHREADS)
    for (int k = 0; k < NV; ++k) {
      int p = piv[k];
      if (p != k) {
        float t = W[k * CB + c];
        W[k * CB + c] = W[p * CB + c];
        W[p * CB + c] = t;
      }
    }
  __syncthreads();
  for (int k = 0; k < NV; ++k) {
    for (int t = threadIdx.x; t < (NV - k - 1) * CB; t += NTHREADS) {
      int r = k + 1 + t / CB, c = t % CB;
      W[r * CB + c] = fmaf(-LU[r * NV + k], W[k * CB + c], W[r * CB + c]);
    }
    __syncthreads();
  }
  for (int k = NV - 1; k >= 0; --k) {
    for (int c = threadIdx.x; c < CB; c += NTHREADS) W[k * CB + c] /= LU[k * NV + k];
    __syncthreads();
    for (int t = threadIdx.x; t < k * CB; t += NTHREADS) {
      int r = t / CB, c = t % CB;
      W[r * CB + c] = fmaf(-LU[r * NV + k], W[k * CB + c], W[r * CB + c]);
    }
    __syncthreads();
  }
}

template <class C, int NTHREADS, int NREF>
__global__ void __launch_bounds__(NTHREADS) k_condense_df(AssembleArgs a) {
  constexpr int NV = C::NV, NT = C::NT;
  using X = MixCfg<C, NTHREADS>;
  constexpr int CB = X::CB;
  extern __shared__ double smem_d[];
  df2* Ad = reinterpret_cast<df2*>(smem_d);  // [NV][NV]
  df2* Bb = Ad + NV * NV;                    // [NV][CB]
  df2* Xb = Bb + NV * CB;                    // [NV][CB]
  float* LU = reinterpret_cast<float*>(Xb + NV * CB);  // [NV][NV]
  float* W = LU + NV * NV;                   // [NV][CB]
  float* sc = W + NV * CB;                  // [NV] equilibration D^{-1/2}
  int* piv = reinterpret_cast<int*>(sc + NV);
  __shared__ int s_piv, s_bad;
  __shared__ float s_corr, s_xmax;
  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x;
  const double* Ap = a.Ap + le * NV * NV;
  const df2* Cp = reinterpret_cast<const df2*>(a.Cp) + le * NT * NV;
  double* Xg = a.recov + e * (int64_t)(NV * NT + NV);
  double* yg = Xg + NV * NT;
  double* S = a.S + e * (int64_t)NT * NT;
  const double* R = a.R + e * (int64_t)(NV + NT);
  for (int r = tid; r < NV; r += NTHREADS) {
    double d = fabs(Ap[r * NV + r]);
    sc[r] = d > 0.0 ? (float)(1.0 / ::sqrt(d)) : 1.f;
  }
  __syncthreads();
  for (int t = tid; t < NV * NV; t += NTHREADS) {
    double v = Ap[t];
    Ad[t] = df_from(v);
    LU[t] = (float)(v * (double)sc[t / NV] * (double)sc[t % NV]);
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int k = 0; k < NV; ++k) {
    if (tid < 32) {
      float best = -1.f;
      int bi = k;
      for (int r = k + tid; r < NV; r += 32) {
        float v = fabsf(LU[r * NV + k]);
        if (v > best) {
          best = v;
          bi = r;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        float ob = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        s_piv = bi;
        piv[k] = bi;
        if (!(best > 0.f)) s_bad |= HDG_STATUS_SINGULAR;
      }
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != k)
      for (int j = tid; j < NV; j += NTHREADS) {
        float t = LU[k * NV + j];
        LU[k * NV + j] = LU[pr * NV + j];
        LU[pr * NV + j] = t;
      }
    __syncthreads();
    const float d = LU[k * NV + k];
    const float inv = d != 0.f ? 1.f / d : 0.f;
    for (int r = k + 1 + tid; r < NV; r += NTHREADS) LU[r * NV + k] *= inv;
    __syncthreads();
    const int rem = NV - k - 1;
    for (int t = tid; t < rem * rem; t += NTHREADS) {
      int r = k + 1 + t / rem, c = k + 1 + t % rem;
      LU[r * NV + c] = fmaf(-LU[r * NV + k], LU[k * NV + c], LU[r * NV + c]);
    }
    __syncthreads();
  }
  for (int c0 = 0; c0 < NT + 1; c0 += CB) {
    const int nc = (NT + 1 - c0) < CB ? (NT + 1 - c0) : CB;
    __syncthreads();
    for (int t = tid; t < NV * CB; t += NTHREADS) {
      int r = t / CB, c = t % CB, col = c0 + c;
      double v = 0.0;
      if (c < nc) v = col < NT ? Xg[r * NT + col] : R[r];
      Bb[t] = df_from(v);
      W[t] = (float)(v * (double)sc[r]);
    }
    __syncthreads();
    lu_solve_f32<NV, CB, NTHREADS>(LU, piv, W);
    for (int t = tid; t < NV * CB; t += NTHREADS) Xb[t] = df_from((double)W[t] * (double)sc[t / CB]);
    for (int it = 0; it < NREF; ++it) {
      if (tid == 0) {
        s_corr = 0.f;
        s_xmax = 0.f;
      }
      __syncthreads();
      // residual r = B - A X in double-float
      for (int t = tid; t < NV * CB; t += NTHREADS) {
        int r = t / CB, c = t % CB;
        dfacc acc;
        acc.add(Bb[t]);
        for (int k = 0; k < NV; ++k) {
          df2 av = Ad[r * NV + k];
          av.hi = -av.hi;
          av.lo = -av.lo;
          acc.mac(av, Xb[k * CB + c]);
        }
        W[t] = (acc.hi + acc.lo) * sc[r];
      }
      __syncthreads();
      lu_solve_f32<NV, CB, NTHREADS>(LU, piv, W);
      for (int t = tid; t < NV * CB; t += NTHREADS) {
        W[t] *= sc[t / CB];
        dfacc acc;
        acc.add(Xb[t]);
        acc.add(df2{W[t], 0.f});
        Xb[t] = acc.norm();
        if (it == NREF - 1) {
          atomicMax(reinterpret_cast<int*>(&s_corr), __float_as_int(fabsf(W[t])));
          atomicMax(reinterpret_cast<int*>(&s_xmax), __float_as_int(fabsf(Xb[t].hi)));
        }
      }
      __syncthreads();
    }
    if (tid == 0 && !(s_corr <= 1e-10f * s_xmax)) s_bad |= 4;  // refinement did not reach 1e-10
    for (int t = tid; t < NV * CB; t += NTHREADS) {
      int r = t / CB, c = t % CB, col = c0 + c;
      if (c < nc) {
        if (col < NT)
          Xg[r * NT + col] = df_val(Xb[t]);
        else
          yg[r] = df_val(Xb[t]);
      }
    }
    // Schur products for this block: S[:, cols] = D' - C' X ; g = R_t - C' y
    for (int t = tid; t < NT * nc; t += NTHREADS) {
      int r = t / nc, c = t % nc, col = c0 + c;
      dfacc acc;
      const df2* Cr = Cp + r * NV;
      for (int k = 0; k < NV; ++k) acc.mac(Cr[k], Xb[k * CB + c]);
      if (col < NT)
        S[r * NT + col] -= acc.value();
      else
        a.g[e * NT + r] = R[NV + r] - acc.value();
    }
  }
  if (tid == 0 && s_bad) atomicOr(a.status + e, s_bad);
}

}  // namespace hdg
