// Static condensation of one element on the FP32 pipe and the bf16 tensor cores
// (mixed form of Sec. 3.2's local elimination: S = D' - C' A'^{-1} B', g = R_t - C' A'^{-1} R_v).
//
// Inputs written by the mixed assembly, all double-float (hi, lo) pairs:
//   A' [NV][NV] and C' [NT][NV] in the chunk scratch, B' [NV][NT] in the recovery array,
//   D' [NT][NT] in the S array; R_v, R_t in FP64.
// Outputs (FP64): S over D', X = A'^{-1} B' over B' and y = A'^{-1} R_v, g.
//
// One CTA per element.
//   1. Jacobi equilibration sc = |diag A'|^{-1/2}; FP32 Gauss-Jordan inverse Ai of
//      sc A' sc with row pivoting (shared memory). A' and C' are cut into exact bf16
//      slices (ozaki.cuh), stored fragment-native in a per-element scratch (L2).
//   2. Per block of CB = 32 right-hand sides (columns of B' and R_v):
//        X0 = sc Ai sc B                            FP32
//        r0 = B - A' X0                             exact slices on the tensor cores
//        d0 = sc Ai sc r0,  r1 = r0 - A'_hi d0      FP32 (d0 ~ rho |X|, rho ~ 1e-5)
//        d1 = sc Ai sc r1,  X = X0 + d0 + d1        double-float
//        S[:, block] = D' - C' X,  g = R_t - C' y   exact slices on the tensor cores
//      A status bit flags a block whose last correction is not below 1e-10 relative.
#pragma once
#include "assemble_fp64.cuh"
#include "ozaki.cuh"

namespace hdg {

template <class C, int NTHREADS, int OZS>
struct CondTC {
  static constexpr int NV = C::NV, NT = C::NT;
  static constexpr int KT = (NV + 15) / 16;   // k tiles over the interior unknowns
  static constexpr int MTA = KT;              // row tiles of A'
  static constexpr int MTC = (NT + 15) / 16;  // row tiles of C'
  static constexpr int CB = 32, NTB = CB / 8;
  static constexpr int RT = NTHREADS >= 512 ? 2 : 4, CT = 4;  // FP32 register tile
  // fragment-native slices per element: [tile][slice][lane] uint4
  static constexpr size_t slice_uint4 = (size_t)(MTA + MTC) * KT * OZS * 32;
  static constexpr size_t xs_bytes = sizeof(uint2) * KT * NTB * OZS * 32;
  static_assert(xs_bytes >= sizeof(float) * 2 * NV * CB, "residual buffers alias the slice buffer");
  static constexpr size_t bytes = sizeof(float) * (2 * NV * NV + NV * CB + NV) + sizeof(df2) * NV * CB + xs_bytes +
                                  sizeof(int) * (NV + MTA * 16 + MTC * 16 + CB) + 64;
};

// out = Ai * W for an NV x CB block, RT x CT register tiles; epi(r0, c0, acc) stores.
template <int NV, int CB, int RT, int CT, int NTHREADS, class Epi>
HDG_DEVI void cond_gemm_f32(const float* __restrict__ A, const float* __restrict__ Wm, Epi epi) {
  constexpr int NRT = (NV + RT - 1) / RT, NCT = CB / CT;
  for (int tile = threadIdx.x; tile < NRT * NCT; tile += NTHREADS) {
    const int r0 = (tile / NCT) * RT, c0 = (tile % NCT) * CT;
    float acc[RT][CT] = {};
    for (int k = 0; k < NV; ++k) {
      const float4 w = *reinterpret_cast<const float4*>(Wm + k * CB + c0);
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        const float av = (r0 + i < NV) ? A[(r0 + i) * NV + k] : 0.f;
        acc[i][0] = fmaf(av, w.x, acc[i][0]);
        acc[i][1] = fmaf(av, w.y, acc[i][1]);
        acc[i][2] = fmaf(av, w.z, acc[i][2]);
        acc[i][3] = fmaf(av, w.w, acc[i][3]);
      }
    }
    epi(r0, c0, acc);
  }
}

// Exact-slice product of MT row tiles of a sliced left operand (global, fragment-native)
// with the sliced block Xs (shared memory), nnt column tiles; each warp owns one row tile
// and up to two column tiles at a time. epi(row, col, value_without_scales) per element.
template <int KT, int NTB, int OZS, int NWARP, class Epi>
HDG_DEVI void cond_oz_product(const uint4* __restrict__ Lsl, int MT, const uint2* Xs, int nnt, Epi epi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int NH = (nnt + 1) >> 1;
  for (int task = warp; task < MT * NH; task += NWARP) {
    const int mt = task / NH, nt0 = 2 * (task % NH);
    const bool two = nt0 + 1 < nnt;
    float acc[2][OZS][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int d = 0; d < OZS; ++d)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][d][q] = 0.f;
    const uint4* Lt = Lsl + (size_t)mt * KT * OZS * 32 + lane;
#pragma unroll 1
    for (int kt = 0; kt < KT; ++kt) {
      uint4 a[OZS];
#pragma unroll
      for (int s = 0; s < OZS; ++s) a[s] = Lt[(kt * OZS + s) * 32];
      {
        uint2 b[OZS];
#pragma unroll
        for (int s = 0; s < OZS; ++s) b[s] = Xs[((kt * NTB + nt0) * OZS + s) * 32 + lane];
        oz_mma_tile<OZS>(acc[0], a, b);
      }
      if (two) {
        uint2 b[OZS];
#pragma unroll
        for (int s = 0; s < OZS; ++s) b[s] = Xs[((kt * NTB + nt0 + 1) * OZS + s) * 32 + lane];
        oz_mma_tile<OZS>(acc[1], a, b);
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (j == 1 && !two) break;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = mt * 16 + (lane >> 2) + 8 * (q >> 1);
        const int col = (nt0 + j) * 8 + 2 * (lane & 3) + (q & 1);
        epi(row, col, oz_combine<OZS>(acc[j], q));
      }
    }
  }
}

HDG_DEVI df2 df_scaled(const dfacc& v, int e) {
  const float p = ldexpf(1.f, e);
  const df2 n = v.norm();
  return {n.hi * p, n.lo * p};
}

template <class C, int NTHREADS, int OZS>
__global__ void __launch_bounds__(NTHREADS) k_condense_tc(AssembleArgs a) {
  using Q = CondTC<C, NTHREADS, OZS>;
  constexpr int NV = C::NV, NT = C::NT, KT = Q::KT, MTA = Q::MTA, MTC = Q::MTC, CB = Q::CB, NTB = Q::NTB;
  constexpr int RT = Q::RT, CT = Q::CT, NWARP = NTHREADS / 32;
  extern __shared__ double smem_d[];
  df2* Xb = reinterpret_cast<df2*>(smem_d);                 // [NV][CB] current X block
  uint2* Xs = reinterpret_cast<uint2*>(Xb + NV * CB);       // [KT][NTB][OZS][32] X slices
  float* Rk = reinterpret_cast<float*>(Xs);                 // [NV][CB] residual (aliases Xs)
  float* Dk = Rk + NV * CB;                                 // [NV][CB] correction (aliases Xs)
  float* Ai = reinterpret_cast<float*>(reinterpret_cast<char*>(Xs) + Q::xs_bytes);  // [NV][NV]
  float* Ah = Ai + NV * NV;                                 // [NV][NV] A' (FP32)
  float* W = Ah + NV * NV;                                  // [NV][CB]
  float* sc = W + NV * CB;                                  // [NV]
  int* piv = reinterpret_cast<int*>(sc + NV);               // [NV]
  int* eA = piv + NV;                                       // [MTA*16] row exponents of A'
  int* eC = eA + MTA * 16;                                  // [MTC*16] row exponents of C'
  int* eX = eC + MTC * 16;                                  // [CB] column exponents of the X block
  __shared__ int s_piv, s_bad;
  __shared__ float s_corr[2], s_xmax;
  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const df2* Ap = reinterpret_cast<const df2*>(a.Ap) + le * NV * NV;
  const df2* Cp = reinterpret_cast<const df2*>(a.Cp) + le * NT * NV;
  uint4* slA = a.oz + le * Q::slice_uint4;
  uint4* slC = slA + (size_t)MTA * KT * OZS * 32;
  double* Xg = a.recov + e * (int64_t)(NV * NT + NV);  // B' (double-float) in, X out
  const df2* Bd = reinterpret_cast<const df2*>(Xg);
  double* yg = Xg + NV * NT;
  double* S = a.S + e * (int64_t)NT * NT;  // D' (double-float) in, S out
  const df2* Dd = reinterpret_cast<const df2*>(S);
  const double* R = a.R + e * (int64_t)(NV + NT);

  // ---- equilibration, FP32 copies of A', row exponents
  for (int r = tid; r < NV; r += NTHREADS) {
    const float d = fabsf(Ap[r * NV + r].hi);
    sc[r] = d > 0.f ? rsqrtf(d) : 1.f;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int r = warp; r < MTA * 16; r += NWARP) {
    float mx = 0.f;
    if (r < NV)
      for (int k = lane; k < NV; k += 32) {
        const float v = Ap[r * NV + k].hi;
        Ah[r * NV + k] = v;
        Ai[r * NV + k] = v * sc[r] * sc[k];
        mx = fmaxf(mx, fabsf(v));
      }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) eA[r] = oz_exponent(mx);
  }
  for (int r = warp; r < MTC * 16; r += NWARP) {
    float mx = 0.f;
    if (r < NT)
      for (int k = lane; k < NV; k += 32) mx = fmaxf(mx, fabsf(Cp[r * NV + k].hi));
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) eC[r] = oz_exponent(mx);
  }
  __syncthreads();
  // ---- slices of A' and C' (one warp per 16 x 16 tile)
  {
    auto getA = [&](int r, int k) { return (r < NV && k < NV) ? Ap[r * NV + k] : df2{0.f, 0.f}; };
    auto getC = [&](int r, int k) { return (r < NT && k < NV) ? Cp[r * NV + k] : df2{0.f, 0.f}; };
    auto sA = [&](int r) { return oz_scale(eA[r]); };
    auto sC = [&](int r) { return oz_scale(eC[r]); };
    for (int u = warp; u < (MTA + MTC) * KT; u += NWARP) {
      const int mt = u / KT, kt = u % KT;
      if (mt < MTA)
        oz_slice_left_tile<OZS>(slA + (size_t)u * OZS * 32, 32, mt * 16, kt * 16, lane, getA, sA);
      else
        oz_slice_left_tile<OZS>(slA + (size_t)u * OZS * 32, 32, (mt - MTA) * 16, kt * 16, lane, getC, sC);
    }
  }
  // ---- Gauss-Jordan inversion of sc A' sc in place with row pivoting
  for (int k = 0; k < NV; ++k) {
    if (tid < 32) {
      float best = -1.f;
      int bi = k;
      for (int r = k + tid; r < NV; r += 32) {
        const float v = fabsf(Ai[r * NV + k]);
        if (v > best) {
          best = v;
          bi = r;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
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
    const float pivv = Ai[pr * NV + k];
    const float ip = pivv != 0.f ? 1.f / pivv : 0.f;
    __syncthreads();
    for (int j = tid; j < NV; j += NTHREADS) {
      const float vk = Ai[k * NV + j], vp = Ai[pr * NV + j];
      if (pr != k) Ai[pr * NV + j] = vk;
      Ai[k * NV + j] = (j == k) ? ip : vp * ip;
    }
    __syncthreads();
    for (int r = tid; r < NV; r += NTHREADS) W[r] = Ai[r * NV + k];  // multipliers
    __syncthreads();
    for (int t = tid; t < NV * NV; t += NTHREADS) {
      const int r = t / NV, j = t % NV;
      if (r == k) continue;
      const float f = W[r];
      Ai[t] = (j == k) ? -f * ip : fmaf(-f, Ai[k * NV + j], Ai[t]);
    }
    __syncthreads();
  }
  for (int k = NV - 1; k >= 0; --k) {  // row interchanges become column interchanges
    const int p = piv[k];
    if (p != k)
      for (int r = tid; r < NV; r += NTHREADS) {
        const float t = Ai[r * NV + k];
        Ai[r * NV + k] = Ai[r * NV + p];
        Ai[r * NV + p] = t;
      }
    __syncthreads();
  }

  auto col_exponents = [&]() {  // eX[c] from the current X block
    for (int c = warp; c < CB; c += NWARP) {
      float mx = 0.f;
      for (int r = lane; r < NV; r += 32) mx = fmaxf(mx, fabsf(Xb[r * CB + c].hi));
      for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (lane == 0) eX[c] = oz_exponent(mx);
    }
  };
  auto slice_X = [&](int nnt) {
    auto getX = [&](int k, int n) { return k < NV ? Xb[k * CB + n] : df2{0.f, 0.f}; };
    auto sX = [&](int n) { return oz_scale(eX[n]); };
    for (int u = warp; u < KT * nnt; u += NWARP) {
      const int kt = u / nnt, nt = u % nnt;
      oz_slice_right_tile<OZS>(Xs + (kt * NTB + nt) * OZS * 32, 32, kt * 16, nt * 8, lane, getX, sX);
    }
  };

  // ---- blocks of right-hand sides
  for (int c0 = 0; c0 < NT + 1; c0 += CB) {
    const int nc = (NT + 1 - c0) < CB ? (NT + 1 - c0) : CB;
    const int nnt = (nc + 7) / 8;
    auto bval = [&](int r, int c) -> df2 {  // B' column or R_v, zero past the block
      const int col = c0 + c;
      if (c >= nc) return df2{0.f, 0.f};
      return col < NT ? Bd[r * NT + col] : df_from(R[r]);
    };
    for (int t = tid; t < NV * CB; t += NTHREADS) {
      const df2 b = bval(t / CB, t % CB);
      W[t] = (b.hi + b.lo) * sc[t / CB];
    }
    if (tid < 2) s_corr[tid] = 0.f;
    if (tid == 0) s_xmax = 0.f;
    __syncthreads();
    // X0 = sc Ai W
    cond_gemm_f32<NV, CB, RT, CT, NTHREADS>(Ai, W, [&](int r0, int cc0, float(&acc)[RT][CT]) {
#pragma unroll
      for (int i = 0; i < RT; ++i)
        if (r0 + i < NV)
#pragma unroll
          for (int j = 0; j < CT; ++j) Xb[(r0 + i) * CB + cc0 + j] = df2{acc[i][j] * sc[r0 + i], 0.f};
    });
    __syncthreads();
    col_exponents();
    __syncthreads();
    slice_X(nnt);
    __syncthreads();
    // r0 = B - A' X0 (exact slices), staged in W (the products read Xs, which Rk aliases)
    cond_oz_product<KT, NTB, OZS, NWARP>(slA, MTA, Xs, nnt, [&](int row, int col, const dfacc& v) {
      if (row < NV) {
        const df2 p = df_scaled(v, eA[row] + eX[col]);
        dfacc t;
        t.add(bval(row, col));
        t.add(df2{-p.hi, -p.lo});
        W[row * CB + col] = col < nc ? t.hi + t.lo : 0.f;
      }
    });
    __syncthreads();
    for (int t = tid; t < NV * CB; t += NTHREADS) {  // columns past the block stay zero
      const float rv = W[t];
      Rk[t] = rv;
      W[t] = rv * sc[t / CB];
    }
    __syncthreads();
    // two corrections: d_it = sc Ai W; X += d_it; between them r1 = r0 - A' d0 (FP32)
    for (int it = 0; it < 2; ++it) {
      cond_gemm_f32<NV, CB, RT, CT, NTHREADS>(Ai, W, [&](int r0, int cc0, float(&acc)[RT][CT]) {
        float cmax = 0.f, xmax = 0.f;
#pragma unroll
        for (int i = 0; i < RT; ++i)
          if (r0 + i < NV)
#pragma unroll
            for (int j = 0; j < CT; ++j) {
              const int t = (r0 + i) * CB + cc0 + j;
              const float corr = acc[i][j] * sc[r0 + i];
              dfacc u;
              u.add(Xb[t]);
              u.add(df2{corr, 0.f});
              const df2 xn = u.norm();
              Xb[t] = xn;
              Dk[t] = corr;
              cmax = fmaxf(cmax, fabsf(corr));
              xmax = fmaxf(xmax, fabsf(xn.hi));
            }
        atomicMax(reinterpret_cast<int*>(&s_corr[it]), __float_as_int(cmax));
        if (it == 1) atomicMax(reinterpret_cast<int*>(&s_xmax), __float_as_int(xmax));
      });
      __syncthreads();
      if (it == 1) break;
      cond_gemm_f32<NV, CB, RT, CT, NTHREADS>(Ah, Dk, [&](int r0, int cc0, float(&acc)[RT][CT]) {
#pragma unroll
        for (int i = 0; i < RT; ++i)
          if (r0 + i < NV)
#pragma unroll
            for (int j = 0; j < CT; ++j) {
              const int t = (r0 + i) * CB + cc0 + j;
              const float rv = Rk[t] - acc[i][j];
              Rk[t] = rv;
              W[t] = rv * sc[r0 + i];
            }
      });
      __syncthreads();
    }
    // The corrections contract the error by rho ~ |I - Ai A'| per sweep; the last one
    // measures the error before it, so the error left is ~ c_last^2 / c_prev.
    if (tid == 0) {
      const float cl = s_corr[1], cp = s_corr[0];
      if (!((double)cl * (double)cl <= 1e-10 * (double)s_xmax * (double)cp)) s_bad |= 4;
    }
    // store X and y for the recovery
    for (int t = tid; t < NV * CB; t += NTHREADS) {
      const int r = t / CB, c = t % CB, col = c0 + c;
      if (c < nc) {
        const double xv = df_val(Xb[t]);
        if (col < NT)
          Xg[r * NT + col] = xv;
        else
          yg[r] = xv;
      }
    }
    col_exponents();
    __syncthreads();
    slice_X(nnt);
    __syncthreads();
    // S[:, block] = D' - C' X ; g = R_t - C' y
    cond_oz_product<KT, NTB, OZS, NWARP>(slC, MTC, Xs, nnt, [&](int row, int col, const dfacc& v) {
      const int gc = c0 + col;
      if (row >= NT || col >= nc) return;
      const df2 p = df_scaled(v, eC[row] + eX[col]);
      dfacc t;
      if (gc < NT)
        t.add(Dd[row * NT + gc]);
      else
        t.add(df_from(R[NV + row]));
      t.add(df2{-p.hi, -p.lo});
      if (gc < NT)
        S[row * NT + gc] = t.value();
      else
        a.g[e * NT + row] = t.value();
    });
    __syncthreads();
  }
  if (tid == 0 && s_bad) atomicOr(a.status + e, s_bad);
}

}  // namespace hdg
