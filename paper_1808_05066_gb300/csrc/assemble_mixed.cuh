// Mixed-precision assembly (the condensation that follows it is in condense_tc.cuh).
//
// Same mathematics as the FP64 form (assemble_fp64.cuh), arranged for GB300's pipes:
//   * pointwise fluxes and Jacobians: FP64 (k_pointwise), stored as double-floats;
//   * quadrature contractions for A', B', C', D': double-float multiply-accumulate on
//     the FP32 pipe, each thread accumulating a strip of JW outputs in registers;
//   * the four blocks leave as double-float pairs (hi, lo) in the 8-byte slots of the
//     arrays the FP64 form uses, ready for the mixed condensation;
//   * residuals R_v, R_t: FP64 from the double-float point data.
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

// Tile shape of the mixed assembly: NTHREADS threads per element CTA and GTMAX volume
// quadrature points per shared-memory tile (smaller tiles: less shared memory, more CTAs
// per SM). The library times the compiled shapes on the first chunk and keeps the fastest.
template <class C, int NTHREADS, int GTMAX = 64>
struct MixCfg {
  static constexpr int GT = C::NG < GTMAX ? C::NG : GTMAX;
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
  static constexpr int NTS = 1 + C::D + (C::VISC ? C::D * C::D : 0);  // point values one (i, l) needs
  static constexpr int TSV = GT * NTS;
  static constexpr int TSF = C::NGF * C::NRF;
  static constexpr int TSMAX = TSV > TSF ? TSV : TSF;
  static constexpr size_t asm_bytes = sizeof(df2) * (RBMAX + ZSMAX + TSMAX + C::D * C::D + C::NF * C::D) +
                                      sizeof(double) * (C::NZ * C::M + C::GEO + C::NV + C::NT);
};

HDG_DEVI df2 df_add(df2 x, const dfacc& y) {
  dfacc t = y;
  t.add(x);
  return t.norm();
}

// ------------------------------------------------------------------------------------
// k_assemble_df: one CTA per element
// ------------------------------------------------------------------------------------
template <class C, int NTHREADS, int GTMAX>
__global__ void __launch_bounds__(NTHREADS) k_assemble_df(AssembleArgs a, DevTables T, DevTablesDF TD) {
  constexpr int D = C::D, M = C::M, NP = C::NP, NFN = C::NFN, NF = C::NF, NG = C::NG, NGF = C::NGF;
  constexpr int NZ = C::NZ, NV = C::NV, NT = C::NT, NR = C::NR, NRF = C::NRF;
  using X = MixCfg<C, NTHREADS, GTMAX>;
  constexpr int GT = X::GT, JW = X::JW, NSV = X::NSV, JWF = X::JWF, NSF = X::NSF;
  extern __shared__ double smem_d[];
  df2* Rb = reinterpret_cast<df2*>(smem_d);
  df2* Zs = Rb + X::RBMAX;
  df2* Ts = Zs + X::ZSMAX;           // per-(i, l) point values staged from the point tensors
  df2* JiD = Ts + X::TSMAX;          // [D][D] Jinv as double-float
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
  // A', B', C', D' leave as double-float pairs (8 bytes, in the FP64 arrays' slots)
  df2* Ad = reinterpret_cast<df2*>(a.Ap) + le * NV * NV;
  df2* Cp = reinterpret_cast<df2*>(a.Cp) + le * NT * NV;
  df2* Bd = reinterpret_cast<df2*>(a.recov + e * (int64_t)(NV * NT + NV));
  df2* Dd = reinterpret_cast<df2*>(a.S + e * (int64_t)NT * NT);
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
    constexpr int NTS = X::NTS;
    for (int il = 0; il < M * M; ++il) {
      const int i = il / M, l = il % M;
      __syncthreads();
      // stage T0[i][l], T1[r][i][l], T2[r][i][l][k] of the tile's points
      for (int t = tid; t < GT * NTS; t += NTHREADS) {
        const int gg = t / NTS, q = t % NTS;
        df2 val = {0.f, 0.f};
        if (gg < ng) {
          const df2* P = ptv + (g0 + gg) * C::PT_VOL + M + D * M;  // T0
          if (q == 0)
            val = P[i * M + l];
          else if (q <= D)
            val = P[M * M + ((q - 1) * M + i) * M + l];
          else {
            const int r = (q - 1 - D) / D, k = (q - 1 - D) % D;
            val = P[M * M + D * M * M + ((r * M + i) * M + l) * D + k];
          }
        }
        Ts[t] = val;
      }
      __syncthreads();
      for (int t = tid; t < NP * GT * NR; t += NTHREADS) {
        int an = t / (GT * NR), gg = (t / NR) % GT, beta = t % NR;
        df2 val = {0.f, 0.f};
        if (gg < ng) {
          int g = g0 + gg;
          const df2* Tp = Ts + gg * NTS;
          dfacc acc;
          if (beta == 0) {
            acc.mac(TD.Phi[g * NP + an], Tp[0]);
            for (int r = 0; r < D; ++r) acc.mac(TD.dPhi[(r * NG + g) * NP + an], Tp[1 + r]);
          } else {
            int k = beta - 1;
            for (int r = 0; r < D; ++r) acc.mac(TD.dPhi[(r * NG + g) * NP + an], Tp[1 + D + r * D + k]);
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
          df2* dst = j < NP ? Ad + row * NV + j * M + l : Bd + row * NT + (j - NP) * M + l;
          *dst = (g0 == 0) ? acc[jj].norm() : df_add(*dst, acc[jj]);
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
      for (int t = tid; t < NGF * NRF; t += NTHREADS) {  // stage U0, U1, U2[k] of the face points
        const int gf = t / NRF, beta = t % NRF;
        const df2* U0 = ptf + (f * NGF + gf) * C::PT_FACE + M;
        Ts[t] = beta == 0 ? U0[i * M + l]
                          : (beta == 1 ? U0[M * M + i * M + l] : U0[2 * M * M + (i * M + l) * D + (beta - 2)]);
      }
      __syncthreads();
      for (int t = tid; t < NFN * NGF * NRF; t += NTHREADS) {
        int c = t / (NGF * NRF), gf = (t / NRF) % NGF, beta = t % NRF;
        df2 psi = TD.PhiF[(f * NGF + gf) * NP + T.fnodes[f * NFN + c]];
        dfacc acc;
        acc.mac(psi, Ts[gf * NRF + beta]);
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
          if (j < NP) {
            df2& dst = Ad[rowv * NV + j * M + l];
            dst = df_add(dst, acc[jj]);
            Cp[rowt * NV + j * M + l] = acc[jj].norm();
          } else {
            const int tcol = (j - NP) * M + l;
            df2& dst = Bd[rowv * NT + tcol];
            dst = df_add(dst, acc[jj]);
            Dd[rowt * NT + tcol] = acc[jj].norm();
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

}  // namespace hdg
