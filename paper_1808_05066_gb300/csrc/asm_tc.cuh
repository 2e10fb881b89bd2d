// Mixed-precision assembly on the bf16 tensor cores (exact slices, ozaki.cuh).
//
// The Jacobian blocks of Eqs. hDG_NS1-2 (after the exact elimination of q) are quadrature
// contractions. Written as products (rows il = (i, l) pairs of state components, an / c the
// test node, j the nodal column of the trial unknowns, beta the operator):
//   volume:  A'|B' [(an,i)][(j,l)] += sum_{beta,g} Z_il[an][beta,g] Rb[beta,g][j]
//            Z_il[an][0,g]   = Phi[g][an] T0[g][il] + sum_r dPhi_r[g][an] T1[g][r][il]
//            Z_il[an][1+k,g] = sum_r dPhi_r[g][an] T2[g][r][il][k]
//   face f:  F_f[(c,i)][(j,l)] = sum_{beta,gf} PhiF_f[gf][c] U[gf][beta][il] RbF_f[beta,gf][j]
//            C'|D' rows (f,c,i) = F_f;  A'|B' rows (fnode(f,c), i) += F_f
// T0, T1, T2, U are the pointwise flux Jacobians (double-float, k_pointwise); Rb, RbF are
// the element's value / lifted-gradient operators at the quadrature points (geometry x
// reference tables). Every product runs as exact bf16 slices: S slices per operand with a
// power-of-two scale per row (an FP32 bound of the row's largest entry) and per column,
// S(S+1)/2 mma.sync per tile, each slice diagonal accumulated exactly in FP32 over at most
// 128 k entries, combined in double-float.
//
// Kernels (per element chunk):
//   k_asm_rb      the operator slices Rb, RbF (fragment-native) and column exponents
//   k_asm_vol_tc  grid (element x row block): 16 MTC rows of (il, an) x all columns
//   k_asm_face_tc grid (element x il group): the faces, after the volume
//   k_asm_residual R_v, R_t in FP64 from the double-float point data
#pragma once
#include "assemble_mixed.cuh"
#include "ozaki.cuh"

namespace hdg {

template <class C, int S, int MTC, int NJW = 4>
struct AsmTC {
  static constexpr int D = C::D, M = C::M, NP = C::NP, NFN = C::NFN, NF = C::NF, NG = C::NG, NGF = C::NGF;
  static constexpr int NZ = C::NZ, NV = C::NV, NT = C::NT, NR = C::NR, NRF = C::NRF;
  static constexpr int NTN = (NZ + 7) / 8;    // n tiles over the nodal columns
  static constexpr int NGRP = (NTN + NJW - 1) / NJW;  // groups of NJW n tiles (one warp each)
  static constexpr int KTB = (NG + 15) / 16, KTV = NR * KTB;     // volume k tiles (beta-major)
  static constexpr int KTBF = (NGF + 15) / 16, KTF = NRF * KTBF;  // face k tiles
  static constexpr int KFLUSH = 8;            // k tiles per exact accumulation (128 entries)
  static constexpr int ROWS = 16 * MTC;       // product rows per CTA
  static constexpr int RV = M * M * NP;       // volume rows (il, an)
  static constexpr int NPASS = (RV + ROWS - 1) / ROWS;
  static constexpr int QIL = ROWS / NFN;      // il pairs per face CTA (whole pairs: no races)
  static constexpr int NFCTA = (M * M + QIL - 1) / QIL;
  static constexpr int NTH = 32 * MTC * NGRP;
  // NJW = 2 keeps a thread within 128 registers (two 256-thread CTAs or one 512-thread CTA per SM)
  static constexpr int MINB = NJW == 2 ? (512 / NTH > 0 ? 512 / NTH : 1) : 1;
  static constexpr int NILV = (ROWS + NP - 1) / NP + 1;  // il pairs one volume CTA touches
  static constexpr int NTS = 1 + D + (C::VISC ? D * D : 0);
  static_assert(QIL >= 1 && KTF <= KFLUSH, "face block");
  // operator slices per element (uint2 units): volume [KTV][NTN][S][32], faces [NF][KTF][NTN][S][32],
  // then the column exponents (int): volume [NTN*8], faces [NF][NTN*8]
  static constexpr size_t vol_u2 = (size_t)KTV * NTN * S * 32;
  static constexpr size_t face_u2 = (size_t)KTF * NTN * S * 32;
  static constexpr int NEXP = NTN * 8 * (1 + NF);
  static constexpr size_t rb_u2 = (vol_u2 + NF * face_u2 + (NEXP + 1) / 2 + 31) / 32 * 32;
  static constexpr size_t stripe_u2 = (size_t)NTN * S * 32;  // one k tile of operator slices
  // shared memory of the product kernels
  static constexpr size_t zs_u4 = (size_t)MTC * S * 32;       // one k tile of Z slices
  static constexpr int NPP = NP | 1;                // odd row stride of the staged basis (banks)
  static constexpr int NPSI = (1 + D) * NG * NPP;  // Phi and dPhi of all volume points
  // with one CTA per SM (64-row blocks) the first half-K result waits in shared memory for
  // the second instead of a global read-modify-write
  static constexpr bool FLUSH_SMEM = MTC >= 4 && KTV > KFLUSH;
  static constexpr size_t flush_df2 = FLUSH_SMEM ? (size_t)ROWS * NTN * 8 : 0;
  static constexpr size_t vol_bytes = sizeof(uint4) * 2 * zs_u4 + sizeof(uint2) * 2 * stripe_u2 +
                                      sizeof(df2) * (NG * NILV * NTS + NPSI + flush_df2) +
                                      sizeof(int) * (ROWS + NTN * 8) + 64;
  static constexpr size_t face_bytes =
      sizeof(uint4) * 2 * zs_u4 + sizeof(uint2) * 2 * stripe_u2 +
      sizeof(df2) * (NF * NGF * QIL * NRF + NF * NGF * NFN + QIL * NP * NZ) + sizeof(int) * NF * (ROWS + NTN * 8) + 64;
};

// Geometry as double-floats: Jinv [D][D] and n_f s_f / |J| [NF][D].
template <class C>
HDG_DEVI void load_geo_df(const AssembleArgs& a, int64_t e, df2* JiD, df2* NsD) {
  constexpr int D = C::D, NF = C::NF;
  const double* G = a.geo + e * C::GEO;
  const double detJ = G[D * D];
  for (int t = threadIdx.x; t < D * D; t += blockDim.x) JiD[t] = df_from(G[t]);
  for (int t = threadIdx.x; t < NF * D; t += blockDim.x) {
    const int f = t / D, k = t % D;
    const double* Gf = G + D * D + 1 + f * (D + 1);
    NsD[t] = df_from(Gf[k] * (Gf[D] / detJ));
  }
}

// Volume operator Rb[beta,g][j]: value (double-float) or an FP32 bound of |value|.
template <class C, bool BOUND>
HDG_DEVI auto rb_vol(int beta, int g, int j, const DevTables& T, const DevTablesDF& TD, const df2* JiD,
                     const df2* NsD) {
  constexpr int D = C::D, NP = C::NP, NG = C::NG, NFN = C::NFN, NF = C::NF;
  dfacc acc;
  float bnd = 0.f;
  auto term = [&](df2 x, df2 y, bool neg) {
    if constexpr (BOUND) {
      bnd = fmaf(fabsf(x.hi), fabsf(y.hi), bnd);
    } else {
      if (neg) x = df2{-x.hi, -x.lo};
      acc.mac(x, y);
    }
  };
  if (g < NG && j < C::NZ) {
    if (beta == 0) {
      if (j < NP) term(TD.Phi[g * NP + j], df2{1.f, 0.f}, false);
    } else {
      const int k = beta - 1;
      if (j < NP) {
        for (int r = 0; r < D; ++r) term(JiD[r * D + k], TD.dPhi[(r * NG + g) * NP + j], false);
        for (int f = 0; f < NF; ++f) {
          const int c = T.nodepos[f * NP + j];
          if (c >= 0) term(NsD[f * D + k], TD.PL[(f * NG + g) * NFN + c], true);
        }
      } else {
        const int f = (j - NP) / NFN, c = (j - NP) % NFN;
        term(NsD[f * D + k], TD.PL[(f * NG + g) * NFN + c], false);
      }
    }
  }
  if constexpr (BOUND)
    return bnd;
  else
    return acc.norm();
}

// Face operator RbF_f[beta,gf][j].
template <class C, bool BOUND>
HDG_DEVI auto rb_face(int f, int beta, int gf, int j, const DevTables& T, const DevTablesDF& TD, const df2* JiD,
                      const df2* NsD) {
  constexpr int D = C::D, NP = C::NP, NGF = C::NGF, NFN = C::NFN, NF = C::NF;
  dfacc acc;
  float bnd = 0.f;
  auto term = [&](df2 x, df2 y, bool neg) {
    if constexpr (BOUND) {
      bnd = fmaf(fabsf(x.hi), fabsf(y.hi), bnd);
    } else {
      if (neg) x = df2{-x.hi, -x.lo};
      acc.mac(x, y);
    }
  };
  if (gf < NGF && j < C::NZ) {
    const df2* phif = TD.PhiF + (f * NGF + gf) * NP;
    if (beta == 0) {
      if (j < NP) term(phif[j], df2{1.f, 0.f}, false);
    } else if (beta == 1) {
      if (j >= NP && (j - NP) / NFN == f) term(phif[T.fnodes[f * NFN + (j - NP) % NFN]], df2{1.f, 0.f}, false);
    } else {
      const int k = beta - 2;
      if (j < NP) {
        for (int r = 0; r < D; ++r) term(JiD[r * D + k], TD.dPhiF[((f * D + r) * NGF + gf) * NP + j], false);
        for (int fl = 0; fl < NF; ++fl) {
          const int c = T.nodepos[fl * NP + j];
          if (c >= 0) term(NsD[fl * D + k], TD.PLF[((f * NF + fl) * NGF + gf) * NFN + c], true);
        }
      } else {
        const int fl = (j - NP) / NFN, c = (j - NP) % NFN;
        term(NsD[fl * D + k], TD.PLF[((f * NF + fl) * NGF + gf) * NFN + c], false);
      }
    }
  }
  if constexpr (BOUND)
    return bnd;
  else
    return acc.norm();
}

// ------------------------------------------------------------------------------------
// k_asm_rb: operator slices and column exponents of one element
// ------------------------------------------------------------------------------------
template <class C, int S, int MTC>
__global__ void __launch_bounds__(256) k_asm_rb(AssembleArgs a, DevTables T, DevTablesDF TD) {
  using Q = AsmTC<C, S, MTC>;
  constexpr int D = C::D, NF = C::NF, NTN = Q::NTN, KTV = Q::KTV, KTF = Q::KTF, KTB = Q::KTB, KTBF = Q::KTBF;
  constexpr int NC = NTN * 8;
  __shared__ df2 JiD[D * D], NsD[NF * D];
  __shared__ int ex[Q::NEXP];
  __shared__ float bmax[Q::NEXP];
  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  load_geo_df<C>(a, e, JiD, NsD);
  for (int t = tid; t < Q::NEXP; t += blockDim.x) bmax[t] = 0.f;
  __syncthreads();
  // column bounds: volume (over beta, g) and per face (over beta, gf)
  for (int t = tid; t < NC * KTV * 16; t += blockDim.x) {
    const int j = t % NC, kk = t / NC, beta = kk / (KTB * 16), g = kk % (KTB * 16);
    const float b = rb_vol<C, true>(beta, g, j, T, TD, JiD, NsD);
    if (b > 0.f) atomicMax(reinterpret_cast<int*>(&bmax[j]), __float_as_int(b));
  }
  for (int t = tid; t < NF * NC * KTF * 16; t += blockDim.x) {
    const int j = t % NC, kk = (t / NC) % (KTF * 16), f = t / (NC * KTF * 16);
    const int beta = kk / (KTBF * 16), gf = kk % (KTBF * 16);
    const float b = rb_face<C, true>(f, beta, gf, j, T, TD, JiD, NsD);
    if (b > 0.f) atomicMax(reinterpret_cast<int*>(&bmax[NC * (1 + f) + j]), __float_as_int(b));
  }
  __syncthreads();
  uint2* out = reinterpret_cast<uint2*>(a.rb) + le * Q::rb_u2;
  int* exg = reinterpret_cast<int*>(out + Q::vol_u2 + NF * Q::face_u2);
  for (int t = tid; t < Q::NEXP; t += blockDim.x) {
    ex[t] = oz_exponent(bmax[t] * 1.0001f);  // margin for the bound's own rounding
    exg[t] = ex[t];
  }
  __syncthreads();
  // slices, one warp per 16 x 8 tile
  for (int u = warp; u < KTV * NTN; u += nw) {
    const int kt = u / NTN, nt = u % NTN;
    auto get = [&](int K, int j) { return rb_vol<C, false>(K / (KTB * 16), K % (KTB * 16), j, T, TD, JiD, NsD); };
    auto sc = [&](int j) { return oz_scale(ex[j]); };
    oz_slice_right_tile<S>(out + (size_t)u * S * 32, 32, kt * 16, nt * 8, lane, get, sc);
  }
  for (int u = warp; u < NF * KTF * NTN; u += nw) {
    const int f = u / (KTF * NTN), kt = (u / NTN) % KTF, nt = u % NTN;
    auto get = [&](int kk, int j) { return rb_face<C, false>(f, kk / (KTBF * 16), kk % (KTBF * 16), j, T, TD, JiD, NsD); };
    auto sc = [&](int j) { return oz_scale(ex[NC * (1 + f) + j]); };
    oz_slice_right_tile<S>(out + Q::vol_u2 + (size_t)u * S * 32, 32, kt * 16, nt * 8, lane, get, sc);
  }
}

// Shared pieces of the two product kernels.
// Word w of lane ln of a left-operand tile holds rows (ln/4) + 8 (w%2), k (2 (ln%4) + 8 (w/2)) + {0, 1}.
template <int S>
HDG_DEVI void put_left_word(uint4* zs, int lane, int w, const float (&v0)[S], const float (&v1)[S]) {
  unsigned* z32 = reinterpret_cast<unsigned*>(zs);
#pragma unroll
  for (int s = 0; s < S; ++s) z32[(s * 32 + lane) * 4 + w] = oz_pack2(v0[s], v1[s]);
}

// One warp's products for one k tile: m tile mt, n tiles [nt0, nt0 + NJW), tiles whose
// operator block is zero skipped (live(nt) false).
template <int S, int NTN, int NJW, class Live>
HDG_DEVI void tile_products(float (&acc)[NJW][S][4], const uint4* zs, const uint2* rbs, int mt, int nt0, int lane,
                            Live live) {
  uint4 a[S];
#pragma unroll
  for (int s = 0; s < S; ++s) a[s] = zs[(mt * S + s) * 32 + lane];
#pragma unroll
  for (int jj = 0; jj < NJW; ++jj) {
    const int nt = nt0 + jj;
    if (nt >= NTN || !live(nt)) continue;
    uint2 b[S];
#pragma unroll
    for (int s = 0; s < S; ++s) b[s] = rbs[(nt * S + s) * 32 + lane];
    oz_mma_tile<S>(acc[jj], a, b);
  }
}

// Warps 4..7, 12..15, ... of a CTA with at least 8 warps: one of every two warps a scheduler
// holds (warp w runs on scheduler w % 4).
HDG_DEVI bool stagger_late(int warp, int nthreads) { return nthreads >= 256 && ((warp >> 2) & 1); }

// ------------------------------------------------------------------------------------
// k_asm_vol_tc: rows [ROWS*blockIdx.y, +ROWS) of (il, an), all nodal columns
// ------------------------------------------------------------------------------------
template <class C, int S, int MTC, int NJW>
__global__ void __launch_bounds__(AsmTC<C, S, MTC, NJW>::NTH, AsmTC<C, S, MTC, NJW>::MINB)
    k_asm_vol_tc(AssembleArgs a, DevTablesDF TD) {
  using Q = AsmTC<C, S, MTC, NJW>;
  constexpr int D = C::D, M = C::M, NP = C::NP, NG = C::NG, NV = C::NV, NT = C::NT;
  constexpr int NTN = Q::NTN, NGRP = Q::NGRP, KTB = Q::KTB, KTV = Q::KTV, ROWS = Q::ROWS, NILV = Q::NILV,
                NTS = Q::NTS, NTH = Q::NTH, NC = NTN * 8;
  extern __shared__ double smem_d[];
  uint4* Zs = reinterpret_cast<uint4*>(smem_d);                       // [2][MTC][S][32]
  uint2* Rs = reinterpret_cast<uint2*>(Zs + 2 * Q::zs_u4);            // [2][NTN][S][32]
  df2* Ts = reinterpret_cast<df2*>(Rs + 2 * Q::stripe_u2);            // [NG][NILV][NTS]
  df2* Ps = Ts + NG * NILV * NTS;                                     // Phi [NG][NP], dPhi [D][NG][NP]
  df2* Fb = Ps + Q::NPSI;                                             // [ROWS][NTN*8] first half-K result
  int* eR = reinterpret_cast<int*>(Fb + Q::flush_df2);                // [ROWS]
  int* eC = eR + ROWS;                                                // [NC]
  const int64_t le = blockIdx.y;  // the element's row blocks are neighbours in launch order
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = blockIdx.x * ROWS;
  const int il_lo = row0 / NP;
  const df2* ptv = reinterpret_cast<const df2*>(a.ptv) + le * NG * C::PT_VOL;
  const uint2* rbg = reinterpret_cast<const uint2*>(a.rb) + le * Q::rb_u2;
  const int* exg = reinterpret_cast<const int*>(rbg + Q::vol_u2 + C::NF * Q::face_u2);

  // stage T0, T1, T2 of the il pairs this block touches and the basis tables (asynchronous
  // copies, all in flight together); row exponents from FP32 bounds
  for (int t = tid; t < NG * NILV * NTS; t += NTH) {
    const int q = t % NTS, ilr = (t / NTS) % NILV, g = t / (NTS * NILV);
    const int il = il_lo + ilr;
    if (il < M * M) {
      const int i = il / M, l = il % M;
      const df2* P = ptv + g * C::PT_VOL + M + D * M;
      int off;
      if (q == 0)
        off = i * M + l;
      else if (q <= D)
        off = M * M + ((q - 1) * M + i) * M + l;
      else {
        const int r = (q - 1 - D) / D, k = (q - 1 - D) % D;
        off = M * M + D * M * M + ((r * M + i) * M + l) * D + k;
      }
      cp_async8(Ts + t, P + off);
    } else {
      Ts[t] = df2{0.f, 0.f};
    }
  }
  for (int t = tid; t < (1 + D) * NG * NP; t += NTH) {
    const int gr = t / NP, an = t % NP;  // gr = r * NG + g over Phi, then dPhi_r
    cp_async8(Ps + gr * Q::NPP + an, gr < NG ? TD.Phi + t : TD.dPhi + (t - NG * NP));
  }
  cp_async_commit();
  for (int t = tid; t < NC; t += NTH) eC[t] = exg[t];
  cp_async_wait_all();
  __syncthreads();
  constexpr int NPP = Q::NPP;
  const df2* Phi = Ps;              // [NG][NPP]
  const df2* dPhi = Ps + NG * NPP;  // [D][NG][NPP]
  {
    // threads per row: the largest power of two in NTH / ROWS (consecutive lanes of one warp)
    constexpr int TPR = (NTH / ROWS) >= 8 ? 8 : ((NTH / ROWS) >= 4 ? 4 : ((NTH / ROWS) >= 2 ? 2 : 1));
    const int rl = tid / TPR, part = tid % TPR, row = row0 + rl;
    float b = 0.f;
    if (rl < ROWS && row < Q::RV) {
      const int an = row % NP, ilr = row / NP - il_lo;
      for (int g = part; g < NG; g += TPR) {
        const df2* Tp = Ts + (g * NILV + ilr) * NTS;
        float b0 = fabsf(Phi[g * NPP + an].hi) * fabsf(Tp[0].hi);
#pragma unroll
        for (int r = 0; r < D; ++r) b0 = fmaf(fabsf(dPhi[(r * NG + g) * NPP + an].hi), fabsf(Tp[1 + r].hi), b0);
        b = fmaxf(b, b0);
        if constexpr (C::VISC)
#pragma unroll
          for (int k = 0; k < D; ++k) {
            float bk = 0.f;
#pragma unroll
            for (int r = 0; r < D; ++r)
              bk = fmaf(fabsf(dPhi[(r * NG + g) * NPP + an].hi), fabsf(Tp[1 + D + r * D + k].hi), bk);
            b = fmaxf(b, bk);
          }
      }
    }
#pragma unroll
    for (int off = 1; off < TPR; off <<= 1) b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, off));
    if (part == 0 && rl < ROWS) eR[rl] = oz_exponent(b * 1.0001f);
    __syncthreads();
  }

  // Z slices of k tile kt into buffer b. Unit u = (m tile, lane, word) of the fragment-native
  // tile; each thread's units, rows and scales are fixed over the k loop.
  constexpr int NU = (MTC * 128 + NTH - 1) / NTH;
  int u_rl[NU], u_an[NU], u_tb[NU], u_kk[NU], u_dst[NU];
  float u_sc[NU];
  bool u_ok[NU];
#pragma unroll
  for (int x = 0; x < NU; ++x) {
    const int u = tid + x * NTH;
    const int mt = u >> 7, ln = (u >> 2) & 31, w = u & 3;
    const int rl = mt * 16 + (ln >> 2) + 8 * (w & 1), row = row0 + rl;
    u_ok[x] = u < MTC * 128 && row < Q::RV;
    u_rl[x] = rl;
    u_an[x] = row % NP;
    u_tb[x] = (row / NP - il_lo) * NTS;
    u_kk[x] = 2 * (ln & 3) + 8 * (w >> 1);
    u_dst[x] = (mt * S * 32 + ln) * 4 + w;  // word index within one buffer, slice 0
    u_sc[x] = u < MTC * 128 ? oz_scale(eR[rl]) : 1.f;
  }
  auto produce = [&](int kt, int b) {
    const int beta = kt / KTB, g0 = (kt % KTB) * 16;
    unsigned* z32 = reinterpret_cast<unsigned*>(Zs + (size_t)b * Q::zs_u4);
#pragma unroll
    for (int x = 0; x < NU; ++x) {
      if (tid + x * NTH >= MTC * 128) break;
      float v[2][S];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int g = g0 + u_kk[x] + q;
        df2 z{0.f, 0.f};
        if (u_ok[x] && g < NG) {
          const df2* Tp = Ts + g * (NILV * NTS) + u_tb[x];
          const int an = u_an[x];
          dfacc acc;
          if (beta == 0) {
            acc.mac(Phi[g * NPP + an], Tp[0]);
#pragma unroll
            for (int r = 0; r < D; ++r) acc.mac(dPhi[(r * NG + g) * NPP + an], Tp[1 + r]);
          } else {
            const int k = beta - 1;
#pragma unroll
            for (int r = 0; r < D; ++r) acc.mac(dPhi[(r * NG + g) * NPP + an], Tp[1 + D + r * D + k]);
          }
          z = acc.norm();
        }
        oz_split<S>(z, u_sc[x], v[q]);
      }
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) z32[u_dst[x] + s2 * 128] = oz_pack2(v[0][s2], v[1][s2]);
    }
  };

  // operator stripe kt into buffer b (asynchronous; completed before the next barrier)
  auto fetch = [&](int kt, int b) {
    const uint4* src = reinterpret_cast<const uint4*>(rbg + (size_t)kt * Q::stripe_u2);
    uint4* dst = reinterpret_cast<uint4*>(Rs + (size_t)b * Q::stripe_u2);
    for (int t = tid; t < (int)(Q::stripe_u2 / 2); t += NTH) cp_async16(dst + t, src + t);
    cp_async_commit();
  };

  const int mt = warp / NGRP, nt0 = NJW * (warp % NGRP);
  float acc[NJW][S][4];
  auto zero = [&]() {
#pragma unroll
    for (int jj = 0; jj < NJW; ++jj)
#pragma unroll
      for (int d = 0; d < S; ++d)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[jj][d][q] = 0.f;
  };
  // flush: the exact diagonals into the double-float output (store first, then add). A lane's
  // two output rows (an, i) and component l are fixed: computed once.
  df2* const Aout = reinterpret_cast<df2*>(a.Ap) + le * NV * NV;
  df2* const Bout = reinterpret_cast<df2*>(a.recov + e * (int64_t)(NV * NT + NV));
  int f_row[2], f_l[2], f_rl[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int rl = mt * 16 + (lane >> 2) + 8 * h, row = row0 + rl;
    const int an = row % NP, il = row / NP;
    f_rl[h] = rl;
    f_row[h] = row < Q::RV ? an * M + il / M : -1;
    f_l[h] = il % M;
  }
  auto flush = [&](bool first) {
#pragma unroll
    for (int jj = 0; jj < NJW; ++jj) {
      const int nt = nt0 + jj;
      if (nt >= NTN) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int h = q >> 1, rl = f_rl[h];
        const int j = nt * 8 + 2 * (lane & 3) + (q & 1);
        if (f_row[h] < 0 || j >= C::NZ) continue;
        const dfacc v = oz_combine<S>(acc[jj], q);
        const df2 p = oz_scaled(v, eR[rl] + eC[j]);
        df2* dst = j < NP ? Aout + f_row[h] * NV + j * M + f_l[h] : Bout + f_row[h] * NT + (j - NP) * M + f_l[h];
        if constexpr (Q::FLUSH_SMEM) {
          df2& fb = Fb[rl * (NTN * 8) + j];  // this lane's own entry in both flushes
          if (first) {
            fb = p;
          } else {
            dfacc t;
            t.add(fb);
            t.add(p);
            *dst = t.norm();
          }
        } else if (first) {
          *dst = p;
        } else {
          dfacc t;
          t.add(*dst);
          t.add(p);
          *dst = t.norm();
        }
      }
    }
  };
  // staggered roles: on every scheduler half the warps multiply before they produce the next
  // tile's slices, so that production and products overlap within each k tile
  const bool late = stagger_late(warp, NTH);
  zero();
  fetch(0, 0);
  produce(0, 0);
  cp_async_wait_all();
  __syncthreads();
  for (int kt = 0; kt < KTV; ++kt) {
    const bool more = kt + 1 < KTV;
    if (more) {
      fetch(kt + 1, (kt + 1) & 1);
      if (!late) produce(kt + 1, (kt + 1) & 1);
    }
    const bool beta0 = kt < KTB;
    tile_products<S, NTN, NJW>(acc, Zs + (size_t)(kt & 1) * Q::zs_u4, Rs + (size_t)(kt & 1) * Q::stripe_u2, mt, nt0, lane,
                          [&](int nt) { return !beta0 || nt * 8 < NP; });
    if (more && late) produce(kt + 1, (kt + 1) & 1);
    if ((kt + 1) % Q::KFLUSH == 0 || kt + 1 == KTV) {
      flush(kt + 1 <= Q::KFLUSH);
      zero();
    }
    cp_async_wait_all();
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// k_asm_face_tc: the face blocks of il pairs [QIL*blockIdx.x, +QIL). The four faces run as
// one pipeline of NF*KTF k tiles; each face's block goes to C', D' and is added, in shared
// memory, to the A', B' rows of its nodes, which are added to the volume part once at the end
// (this block owns these il pairs, so no other block touches those entries).
// ------------------------------------------------------------------------------------
template <class C, int S, int MTC, int NJW>
__global__ void __launch_bounds__(AsmTC<C, S, MTC, NJW>::NTH, AsmTC<C, S, MTC, NJW>::MINB)
    k_asm_face_tc(AssembleArgs a, DevTables T, DevTablesDF TD) {
  using Q = AsmTC<C, S, MTC, NJW>;
  constexpr int D = C::D, M = C::M, NP = C::NP, NFN = C::NFN, NF = C::NF, NGF = C::NGF, NV = C::NV, NT = C::NT;
  constexpr int NZ = C::NZ, NRF = C::NRF, NTN = Q::NTN, NGRP = Q::NGRP, KTBF = Q::KTBF, KTF = Q::KTF,
                ROWS = Q::ROWS, QIL = Q::QIL, NTH = Q::NTH, NC = NTN * 8, NK = NF * KTF;
  extern __shared__ double smem_d[];
  uint4* Zs = reinterpret_cast<uint4*>(smem_d);             // [2][MTC][S][32]
  uint2* Rs = reinterpret_cast<uint2*>(Zs + 2 * Q::zs_u4);  // [2][NTN][S][32]
  df2* Us = reinterpret_cast<df2*>(Rs + 2 * Q::stripe_u2);  // [NF][NGF][QIL][NRF]
  df2* Psi = Us + NF * NGF * QIL * NRF;                     // [NF][NGF][NFN] face basis at the face nodes
  df2* Acc = Psi + NF * NGF * NFN;                          // [QIL][NP][NZ] face part of A', B'
  int* eR = reinterpret_cast<int*>(Acc + QIL * NP * NZ);    // [NF][ROWS]
  int* eC = eR + NF * ROWS;                                 // [NF][NC]
  const int64_t le = blockIdx.y;
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int il0 = blockIdx.x * QIL;
  const df2* ptf = reinterpret_cast<const df2*>(a.ptf) + le * NF * NGF * C::PT_FACE;
  const uint2* rbg = reinterpret_cast<const uint2*>(a.rb) + le * Q::rb_u2;
  const int* exg = reinterpret_cast<const int*>(rbg + Q::vol_u2 + NF * Q::face_u2);
  df2* Ad = reinterpret_cast<df2*>(a.Ap) + le * NV * NV;
  df2* Cd = reinterpret_cast<df2*>(a.Cp) + le * NT * NV;
  df2* Bd = reinterpret_cast<df2*>(a.recov + e * (int64_t)(NV * NT + NV));
  df2* Dd = reinterpret_cast<df2*>(a.S + e * (int64_t)NT * NT);
  const int mt = warp / NGRP, nt0 = NJW * (warp % NGRP);
  auto rowinfo = [&](int rl, int& il, int& c) {  // false past the block's pairs
    il = il0 + rl / NFN;
    c = rl % NFN;
    return rl < QIL * NFN && il < M * M;
  };

  // U and the face basis of every face, the A', B' accumulator, row and column exponents
  for (int t = tid; t < NF * NGF * QIL * NRF; t += NTH) {  // asynchronous copies, all in flight
    const int beta = t % NRF, ilr = (t / NRF) % QIL, gf = (t / (NRF * QIL)) % NGF, f = t / (NRF * QIL * NGF);
    const int il = il0 + ilr;
    if (il < M * M) {
      const int i = il / M, l = il % M;
      const df2* U0 = ptf + (f * NGF + gf) * C::PT_FACE + M;
      cp_async8(Us + t, U0 + (beta == 0 ? i * M + l : (beta == 1 ? M * M + i * M + l : 2 * M * M + (i * M + l) * D + (beta - 2))));
    } else {
      Us[t] = df2{0.f, 0.f};
    }
  }
  for (int t = tid; t < NF * NGF * NFN; t += NTH) {
    const int c = t % NFN, gf = (t / NFN) % NGF, f = t / (NFN * NGF);
    cp_async8(Psi + t, TD.PhiF + (f * NGF + gf) * NP + T.fnodes[f * NFN + c]);
  }
  cp_async_commit();
  for (int t = tid; t < QIL * NP * NZ; t += NTH) Acc[t] = df2{0.f, 0.f};
  for (int t = tid; t < NF * ROWS; t += NTH) eR[t] = 0;
  for (int t = tid; t < NF * NC; t += NTH) eC[t] = exg[NC + t];
  cp_async_wait_all();
  __syncthreads();
  {
    float* bR = reinterpret_cast<float*>(eR);
    for (int t = tid; t < NF * ROWS * NGF; t += NTH) {
      const int rl = t % ROWS, gf = (t / ROWS) % NGF, f = t / (ROWS * NGF);
      int il, c;
      if (!rowinfo(rl, il, c)) continue;
      const float psi = fabsf(Psi[(f * NGF + gf) * NFN + c].hi);
      float um = 0.f;
      for (int beta = 0; beta < NRF; ++beta)
        um = fmaxf(um, fabsf(Us[((f * NGF + gf) * QIL + (il - il0)) * NRF + beta].hi));
      const float b = psi * um;
      if (b > 0.f) atomicMax(reinterpret_cast<int*>(&bR[f * ROWS + rl]), __float_as_int(b));
    }
    __syncthreads();
    for (int t = tid; t < NF * ROWS; t += NTH) eR[t] = oz_exponent(bR[t] * 1.0001f);
    __syncthreads();
  }
  // k tile kk of the chained sequence: face kk / KTF, tile kk % KTF
  auto produce = [&](int kk, int b) {
    const int f = kk / KTF, kt = kk % KTF;
    const int beta = kt / KTBF, g0 = (kt % KTBF) * 16;
    for (int u = tid; u < MTC * 128; u += NTH) {
      const int m = u >> 7, ln = (u >> 2) & 31, w = u & 3;
      const int rl = m * 16 + (ln >> 2) + 8 * (w & 1);
      const int kk0 = 2 * (ln & 3) + 8 * (w >> 1);
      const float sc = oz_scale(eR[f * ROWS + rl]);
      int il, c;
      const bool rv = rowinfo(rl, il, c);
      float v[2][S];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int gf = g0 + kk0 + q;
        df2 z{0.f, 0.f};
        if (rv && gf < NGF) {
          dfacc acc;
          acc.mac(Psi[(f * NGF + gf) * NFN + c], Us[((f * NGF + gf) * QIL + (il - il0)) * NRF + beta]);
          z = acc.norm();
        }
        oz_split<S>(z, sc, v[q]);
      }
      put_left_word<S>(Zs + (size_t)(b * MTC + m) * S * 32, ln, w, v[0], v[1]);
    }
  };
  auto fetch = [&](int kk, int b) {
    const uint4* src = reinterpret_cast<const uint4*>(rbg + Q::vol_u2 + (size_t)kk * Q::stripe_u2);
    uint4* dst = reinterpret_cast<uint4*>(Rs + (size_t)b * Q::stripe_u2);
    for (int t = tid; t < (int)(Q::stripe_u2 / 2); t += NTH) cp_async16(dst + t, src + t);
    cp_async_commit();
  };
  float acc[NJW][S][4];
  auto zero = [&]() {
#pragma unroll
    for (int jj = 0; jj < NJW; ++jj)
#pragma unroll
      for (int d = 0; d < S; ++d)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[jj][d][q] = 0.f;
  };
  // the face's block: C', D' rows (global) and the A', B' rows of its nodes (shared)
  auto emit = [&](int f) {
#pragma unroll
    for (int jj = 0; jj < NJW; ++jj) {
      const int nt = nt0 + jj;
      if (nt >= NTN) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int rl = mt * 16 + (lane >> 2) + 8 * (q >> 1);
        const int j = nt * 8 + 2 * (lane & 3) + (q & 1);
        int il, c;
        if (!rowinfo(rl, il, c) || j >= NZ) continue;
        const df2 p = oz_scaled(oz_combine<S>(acc[jj], q), eR[f * ROWS + rl] + eC[f * NC + j]);
        const int i = il / M, l = il % M, rowt = (f * NFN + c) * M + i;
        if (j < NP)
          Cd[rowt * NV + j * M + l] = p;
        else
          Dd[rowt * NT + (j - NP) * M + l] = p;
        df2& dst = Acc[((il - il0) * NP + T.fnodes[f * NFN + c]) * NZ + j];
        dst = df_add(dst, dfacc_of(p));
      }
    }
  };
  zero();
  fetch(0, 0);
  produce(0, 0);
  cp_async_wait_all();
  __syncthreads();
  for (int kk = 0; kk < NK; ++kk) {
    if (kk + 1 < NK) {
      fetch(kk + 1, (kk + 1) & 1);
      produce(kk + 1, (kk + 1) & 1);
    }
    const int f = kk / KTF, beta = (kk % KTF) / KTBF;
    const int jlo = NP + f * NFN, jhi = NP + (f + 1) * NFN;  // the face's own trace columns
    tile_products<S, NTN, NJW>(acc, Zs + (size_t)(kk & 1) * Q::zs_u4, Rs + (size_t)(kk & 1) * Q::stripe_u2, mt, nt0,
                               lane, [&](int nt) {
                                 if (beta == 0) return nt * 8 < NP;
                                 if (beta == 1) return nt * 8 < jhi && nt * 8 + 8 > jlo;
                                 return true;
                               });
    if (kk % KTF == KTF - 1) {
      emit(f);
      zero();
    }
    cp_async_wait_all();
    __syncthreads();
  }
  // add the faces' part to the A', B' rows of this block's il pairs (all of a thread's loads
  // in flight together)
  {
    constexpr int NADD = (QIL * NP * NZ + NTH - 1) / NTH;
    df2* dst[NADD];
    df2 old[NADD];
#pragma unroll
    for (int x = 0; x < NADD; ++x) {
      const int t = tid + x * NTH;
      const int j = t % NZ, an = (t / NZ) % NP, ilr = t / (NZ * NP), il = il0 + ilr;
      dst[x] = nullptr;
      if (t < QIL * NP * NZ && il < M * M) {
        const int i = il / M, l = il % M;
        dst[x] = j < NP ? Ad + (an * M + i) * NV + j * M + l : Bd + (an * M + i) * NT + (j - NP) * M + l;
        old[x] = *dst[x];
      }
    }
#pragma unroll
    for (int x = 0; x < NADD; ++x)
      if (dst[x]) *dst[x] = df_add(old[x], dfacc_of(Acc[tid + x * NTH]));
  }
}

// ------------------------------------------------------------------------------------
// k_asm_residual: R_v and R_t (FP64 from the double-float point data)
// ------------------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(128) k_asm_residual(AssembleArgs a, DevTables T) {
  constexpr int D = C::D, M = C::M, NP = C::NP, NFN = C::NFN, NF = C::NF, NG = C::NG, NGF = C::NGF;
  constexpr int NV = C::NV, NT = C::NT;
  constexpr int PV = M * (1 + D);  // the mass term and the flux rows of a volume point
  __shared__ double Rv[NV];
  __shared__ double Pv[NG * PV];        // the point values the residual reads, in FP64
  __shared__ double Pf[NF * NGF * M];   // (each converted once, not once per use)
  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x;
  const df2* ptv = reinterpret_cast<const df2*>(a.ptv) + le * NG * C::PT_VOL;
  const df2* ptf = reinterpret_cast<const df2*>(a.ptf) + le * NF * NGF * C::PT_FACE;
  double* Rout = a.R + e * (int64_t)(NV + NT);
  for (int t = tid; t < NG * PV; t += blockDim.x) {
    const df2 p = ptv[(t / PV) * C::PT_VOL + t % PV];
    Pv[t] = df_to_f64(p.hi, p.lo);
  }
  for (int t = tid; t < NF * NGF * M; t += blockDim.x) {
    const df2 p = ptf[(t / M) * C::PT_FACE + t % M];
    Pf[t] = df_to_f64(p.hi, p.lo);
  }
  __syncthreads();
  for (int t = tid; t < NV; t += blockDim.x) {
    const int an = t / M, i = t % M;
    double s = a.hist ? -a.hist[e * NV + t] : 0.0;
    for (int g = 0; g < NG; ++g) {
      const double* P = Pv + g * PV;
      s += T.Phi[g * NP + an] * P[i];
      for (int r = 0; r < D; ++r) s += T.dPhi[(r * NG + g) * NP + an] * P[M + r * M + i];
    }
    Rv[t] = s;
  }
  __syncthreads();
  for (int f = 0; f < NF; ++f) {
    for (int t = tid; t < NFN * M; t += blockDim.x) {
      const int c = t / M, i = t % M;
      double s = 0.0;
      for (int gf = 0; gf < NGF; ++gf)
        s += T.PhiF[(f * NGF + gf) * NP + T.fnodes[f * NFN + c]] * Pf[(f * NGF + gf) * M + i];
      Rv[T.fnodes[f * NFN + c] * M + i] += s;
      Rout[NV + (f * NFN + c) * M + i] = s;
    }
    __syncthreads();
  }
  for (int t = tid; t < NV; t += blockDim.x) Rout[t] = Rv[t];
}

}  // namespace hdg
