// Static condensation of one element on the FP32 pipe and the bf16 tensor cores
// (mixed form of Sec. 3.2's local elimination: S = D' - C' A'^{-1} B', g = R_t - C' A'^{-1} R_v).
//
// Inputs written by the mixed assembly, all double-float (hi, lo) pairs:
//   A' [NV][NV] and C' [NT][NV] in the chunk scratch, B' [NV][NT] in the recovery array,
//   D' [NT][NT] in the S array; R_v, R_t in FP64.
// Outputs (FP64): S over D', X = A'^{-1} B' over B' and y = A'^{-1} R_v, g.
//
// Two kernels, one CTA per element each:
//   k_condense_prep (small CTA, several per SM so that elements hide each other's latency):
//      Jacobi equilibration sc = |diag A'|^{-1/2}; FP32 Gauss-Jordan inverse with row
//      pivoting of (sc A' sc)^T in shared memory; FP32 copy of A'; row exponents and exact
//      bf16 slices (ozaki.cuh) of A' and C', fragment-native. All to a per-element scratch.
//   k_condense_tc, per block of CB = 32 right-hand sides (columns of B' and R_v):
//        X0 = sc Ai sc B                            FP32
//        r0 = B - A' X0                             exact slices on the tensor cores
//        d0 = sc Ai sc r0,  r1 = r0 - A'_hi d0      FP32 (d0 ~ rho |X|, rho ~ 1e-5)
//        d1 = sc Ai sc r1,  X = X0 + d0 + d1        double-float
//        S[:, block] = D' - C' X,  g = R_t - C' y   exact slices on the tensor cores
//      A status bit flags a block whose last correction is not below 1e-10 relative.
#pragma once
#include "assemble_fp64.cuh"
#include "ozaki.cuh"

#include <type_traits>

namespace hdg {

template <int N, int LD, int NTHREADS>
struct GJReg {
  static constexpr int NWARP = NTHREADS / 32, RW = (N + NWARP - 1) / NWARP, CQ = (N + 31) / 32;
  static_assert(RW * CQ <= 64, "register tile");
  // shared scratch (ints): pivot row of each step [N], step of each row [N], candidates [2 NWARP]
  static constexpr int smem_ints = 2 * N + 2 * NWARP;
  static constexpr int smem_floats = CQ * 32;  // the scaled pivot row
};

template <class C, int NTHREADS, int OZS>
struct CondTC {
  static constexpr int NV = C::NV, NT = C::NT;
  static constexpr int KT = (NV + 15) / 16;   // k tiles over the interior unknowns
  static constexpr int MTA = KT;              // row tiles of A'
  static constexpr int MTC = (NT + 15) / 16;  // row tiles of C'
  static constexpr int CB = 32, NTB = CB / 8;
  static constexpr int RT = NTHREADS >= 512 ? 2 : 4, CT = 4;  // FP32 register tile
  static constexpr int LDA = (NV + 3) / 4 * 4;  // leading dimension of the transposed FP32 matrices
  // A' and C' rows as the right operand (n tiles of 8 rows), X^T as the left operand
  // (row tiles of 16 block columns); fragment-native slices, [n tile][k tile][slice][lane]
  static constexpr int NTA = (NV + 7) / 8, NTC = (NT + 7) / 8, NMB = CB / 16;
  static constexpr size_t slice_u2 = (size_t)(NTA + NTC) * KT * OZS * 32;
  static constexpr size_t slice_uint4 = slice_u2 / 2;
  static constexpr size_t xs_bytes = sizeof(uint4) * KT * NMB * OZS * 32;
  static_assert(xs_bytes >= sizeof(float) * 2 * NV * CB, "residual buffers alias the slice buffer");
  static constexpr size_t bytes = sizeof(float) * (2 * NV * LDA + NV * CB + NV) + sizeof(df2) * (NV + NT) * CB +
                                  xs_bytes + sizeof(int) * (NV + MTA * 16 + MTC * 16 + CB) + 64;
  // per-element block written by k_condense_prep: Ai^T, A'^T [NV][LDA], sc [LDA], eA, eC
  static constexpr int PREP_AI = 0, PREP_AH = NV * LDA, PREP_SC = 2 * NV * LDA, PREP_EA = PREP_SC + LDA,
                       PREP_EC = PREP_EA + MTA * 16;
  static constexpr size_t prep_floats = (size_t)(PREP_EC + MTC * 16 + 3) / 4 * 4;
  static constexpr int PTH = 256;  // threads of the prep kernel
  using GJ = GJReg<NV, LDA, PTH>;
  static constexpr size_t prep_bytes =
      sizeof(float) * (NV * LDA + NV + GJ::smem_floats) + sizeof(int) * GJ::smem_ints + 64;
};

// out = A * W for an NV x CB block with A stored transposed (At[k][r] = A[r][k], leading
// dimension LDA, zero past NV): RT x CT register tiles, two vector loads per k. With SPLIT
// (one tile per thread at most) a barrier separates every read of Wm from the epilogues, so
// that they may overwrite Wm.
template <int NV, int LDA, int CB, int RT, int CT, int NTHREADS, bool SPLIT = false, class Epi>
HDG_DEVI void cond_gemm_f32(const float* __restrict__ At, const float* Wm, Epi epi) {
  static_assert(CT == 4 && (RT == 2 || RT == 4), "vector loads");
  constexpr int NRT = (NV + RT - 1) / RT, NCT = CB / CT;
  static_assert(!SPLIT || NRT * NCT <= NTHREADS, "one tile per thread");
  for (int tile = threadIdx.x; tile < (SPLIT ? NTHREADS : NRT * NCT); tile += NTHREADS) {
    const int r0 = (tile / NCT) * RT, c0 = (tile % NCT) * CT;
    const bool live = !SPLIT || tile < NRT * NCT;
    float acc[RT][CT] = {};
#pragma unroll 4
    for (int k = 0; k < (live ? NV : 0); ++k) {
      const float4 w = *reinterpret_cast<const float4*>(Wm + k * CB + c0);
      float av[RT];
      if constexpr (RT == 4) {
        const float4 v = *reinterpret_cast<const float4*>(At + k * LDA + r0);
        av[0] = v.x;
        av[1] = v.y;
        av[2] = v.z;
        av[3] = v.w;
      } else {
        const float2 v = *reinterpret_cast<const float2*>(At + k * LDA + r0);
        av[0] = v.x;
        av[1] = v.y;
      }
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        acc[i][0] = fmaf(av[i], w.x, acc[i][0]);
        acc[i][1] = fmaf(av[i], w.y, acc[i][1]);
        acc[i][2] = fmaf(av[i], w.z, acc[i][2]);
        acc[i][3] = fmaf(av[i], w.w, acc[i][3]);
      }
    }
    if constexpr (SPLIT) __syncthreads();
    if (live) epi(r0, c0, acc);
  }
}


// Steps k = 32 q .. 32 q + 31 of gj_inverse_reg (q: a compile-time register index).
template <int N, int NTHREADS, int q, int RW, int CQ>
HDG_DEVI void gj_steps(float (&a)[RW][CQ], unsigned& used, bool& ok, int* si, float* prow) {
  constexpr int NWARP = NTHREADS / 32;
  int* pk_of = si;
  int* k_of = si + N;
  int* crow = si + 2 * N;
  float* cval = reinterpret_cast<float*>(crow + NWARP);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll 1
  for (int kk = 0; kk < 32; ++kk) {
    const int k = 32 * q + kk;
    if (k >= N) break;
    float pv = 0.f;
    int pr = -1;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) {
      const int r = crow[w];
      const float v = cval[w];
      if (r >= 0 && (pr < 0 || fabsf(v) > fabsf(pv) || (fabsf(v) == fabsf(pv) && r < pr))) {
        pv = v;
        pr = r;
      }
    }
    if (!(fabsf(pv) > 0.f)) ok = false;
    const float ip = pv != 0.f ? 1.f / pv : 0.f;
    if (tid == 0) {
      pk_of[k] = pr;
      k_of[pr] = k;
    }
    if (warp == pr % NWARP) {  // the pivot row, scaled, for every warp
      const int pi = pr / NWARP;
      float v[CQ];
#pragma unroll
      for (int qq = 0; qq < CQ; ++qq) v[qq] = 0.f;
#pragma unroll
      for (int i = 0; i < RW; ++i)  // a select chain keeps a[][] in registers
#pragma unroll
        for (int qq = 0; qq < CQ; ++qq) v[qq] = i == pi ? a[i][qq] : v[qq];
#pragma unroll
      for (int qq = 0; qq < CQ; ++qq) prow[lane + 32 * qq] = (qq == q && lane == kk) ? ip : v[qq] * ip;
      used |= 1u << pi;
    }
    __syncthreads();
    float pk[CQ];
#pragma unroll
    for (int qq = 0; qq < CQ; ++qq) pk[qq] = prow[lane + 32 * qq];
    float bv = 0.f;
    int br = -1;
#pragma unroll
    for (int i = 0; i < RW; ++i) {
      const int r = warp + NWARP * i;
      if (r >= N) continue;
      const float f = __shfl_sync(0xffffffffu, a[i][q], kk);
      if (r == pr) {
#pragma unroll
        for (int qq = 0; qq < CQ; ++qq) a[i][qq] = pk[qq];
      } else {
#pragma unroll
        for (int qq = 0; qq < CQ; ++qq)
          a[i][qq] = (qq == q && lane == kk) ? -f * ip : fmaf(-f, pk[qq], a[i][qq]);
        if (!((used >> i) & 1u)) {  // candidate for column k + 1
          const float vn = kk < 31 ? a[i][q] : (q + 1 < CQ ? a[i][(q + 1) % CQ] : 0.f);
          if (br < 0 || fabsf(vn) > fabsf(bv)) {
            bv = vn;
            br = r;
          }
        }
      }
    }
    if (lane == ((kk + 1) & 31)) {
      cval[warp] = bv;
      crow[warp] = br;
    }
    __syncthreads();
  }
}

// Gauss-Jordan inverse with partial pivoting of an N x N FP32 matrix held in registers
// across the CTA: warp w holds rows w, w + NWARP, ... (RW of them), lane l the columns
// l, l + 32, ... (CQ). Rows are not moved: step k pivots on the row p_k with the largest
// |entry| in column k among the rows not yet pivoted (the lowest row on ties), scales it by
// 1/pivot and eliminates column k from every other row, storing -f/pivot in its place. The
// tableau's row p_k then holds the inverse's row k with the columns in pivot order:
// inv[k][p_j] = T[p_k][j]. G (shared memory, leading dimension LD) supplies the matrix and
// receives the inverse in natural order. The lane that updates column k+1 proposes the next
// pivot, so a step takes two barriers. Returns false on a zero pivot.
template <int N, int LD, int NTHREADS>
HDG_DEVI bool gj_inverse_reg(float* G, int* si, float* prow) {
  using Q = GJReg<N, LD, NTHREADS>;
  constexpr int NWARP = Q::NWARP, RW = Q::RW, CQ = Q::CQ;
  int* pk_of = si;          // [N] pivot row of step k
  int* k_of = si + N;       // [N] step at which row r pivoted
  int* crow = si + 2 * N;   // [NWARP] candidate row per warp
  float* cval = reinterpret_cast<float*>(crow + NWARP);  // [NWARP] its value
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float a[RW][CQ];
#pragma unroll
  for (int i = 0; i < RW; ++i)
#pragma unroll
    for (int q = 0; q < CQ; ++q) {
      const int r = warp + NWARP * i, c = lane + 32 * q;
      a[i][q] = (r < N && c < N) ? G[r * LD + c] : 0.f;
    }
  unsigned used = 0;  // bit i: this warp's row i has pivoted
  {                   // candidates for column 0 (lane 0)
    float bv = 0.f;
    int br = -1;
#pragma unroll
    for (int i = 0; i < RW; ++i)
      if (warp + NWARP * i < N && (br < 0 || fabsf(a[i][0]) > fabsf(bv))) {
        bv = a[i][0];
        br = warp + NWARP * i;
      }
    if (lane == 0) {
      cval[warp] = bv;
      crow[warp] = br;
    }
  }
  __syncthreads();
  bool ok = true;
  gj_steps<N, NTHREADS, 0>(a, used, ok, si, prow);
  if constexpr (CQ > 1) gj_steps<N, NTHREADS, 1 % CQ>(a, used, ok, si, prow);
  if constexpr (CQ > 2) gj_steps<N, NTHREADS, 2 % CQ>(a, used, ok, si, prow);
  if constexpr (CQ > 3) gj_steps<N, NTHREADS, 3 % CQ>(a, used, ok, si, prow);
  static_assert(CQ <= 4, "column groups");
  // inv[k_of[r]][pk_of[c]] = T[r][c]
#pragma unroll
  for (int i = 0; i < RW; ++i)
#pragma unroll
    for (int q = 0; q < CQ; ++q) {
      const int r = warp + NWARP * i, c = lane + 32 * q;
      if (r < N && c < N) G[k_of[r] * LD + pk_of[c]] = a[i][q];
    }
  __syncthreads();
  return ok;
}

// Exact-slice product of the rows of A' or C' (right operand, NTL tiles of 8 rows, sliced in
// global memory [NTL][KT][OZS][32]) with the block's X^T (left operand, nmt tiles of 16
// block columns, sliced in shared memory [KT][NMB][OZS][32]). Each warp owns one tile of 8
// rows across all the block's columns, so every right-operand fragment is read from L2 once
// per block; the next k tile's fragments load during this tile's products.
// epi(row, col, value_without_scales) per element (row of A' or C', block column).
// The right operand is stored with OZG >= OZS slices per tile; the first OZS are used. With
// PF each warp asks L2 for its next task's fragments (one contiguous run) while it works.
template <int KT, int NMB, int OZS, int NWARP, int OZG = OZS, bool PF = false, class Epi>
HDG_DEVI void cond_oz_product(const uint2* __restrict__ Rsl, int NTL, const uint4* Xs, int nmt, Epi epi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int task = warp; task < NTL; task += NWARP) {
    if constexpr (PF) {
      if (task + NWARP < NTL) {
        const char* nx = reinterpret_cast<const char*>(Rsl + (size_t)(task + NWARP) * KT * OZG * 32);
        constexpr int LINES = (KT * OZG * 32 * (int)sizeof(uint2)) / 128;
        for (int l = lane; l < LINES; l += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + l * 128));
      }
    }
    float acc[NMB][OZS][4];
#pragma unroll
    for (int m = 0; m < NMB; ++m)
#pragma unroll
      for (int d = 0; d < OZS; ++d)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][d][q] = 0.f;
    const uint2* Bt = Rsl + (size_t)task * KT * OZG * 32 + lane;
    uint2 b[OZS], bn[OZS];
#pragma unroll
    for (int s = 0; s < OZS; ++s) b[s] = Bt[s * 32];
#pragma unroll 1
    for (int kt = 0; kt < KT; ++kt) {
      if (kt + 1 < KT)  // next tile's fragments in flight during this tile's products
#pragma unroll
        for (int s = 0; s < OZS; ++s) bn[s] = Bt[((kt + 1) * OZG + s) * 32];
#pragma unroll
      for (int m = 0; m < NMB; ++m)
        if (m < nmt) {
          uint4 a[OZS];
#pragma unroll
          for (int s = 0; s < OZS; ++s) a[s] = Xs[((kt * NMB + m) * OZS + s) * 32 + lane];
          oz_mma_tile<OZS>(acc[m], a, b);
        }
#pragma unroll
      for (int s = 0; s < OZS; ++s) b[s] = bn[s];
    }
#pragma unroll
    for (int m = 0; m < NMB; ++m) {
      if (m >= nmt) break;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int col = m * 16 + (lane >> 2) + 8 * (q >> 1);
        const int row = task * 8 + 2 * (lane & 3) + (q & 1);
        epi(row, col, oz_combine<OZS>(acc[m], q));
      }
    }
  }
}

// defined in condense_t5.cuh (the tcgen05 operand layout)
template <class C, int OZS>
HDG_DEVI void prep_write_umma_slices(const AssembleArgs& a, int64_t le, const df2* Ap, const df2* Cp, const float* sc,
                                     const int* eA, const int* eC);

// UMMA = true writes the slices of A' P and C' P for k_condense_t5 (tcgen05 operand layout),
// otherwise fragment-native for the mma.sync kernels.
template <class C, int OZS, bool UMMA = false>
__global__ void __launch_bounds__(CondTC<C, 256, OZS>::PTH) k_condense_prep(AssembleArgs a) {
  using Q = CondTC<C, 256, OZS>;
  constexpr int NV = C::NV, NT = C::NT, KT = Q::KT, MTA = Q::MTA, MTC = Q::MTC, LDA = Q::LDA;
  constexpr int PTH = Q::PTH, NWARP = PTH / 32;
  extern __shared__ double smem_d[];
  float* G = reinterpret_cast<float*>(smem_d);  // [NV][LDA] A'^T, then (sc A' sc)^-T
  float* sc = G + NV * LDA;                     // [NV]
  float* prow = sc + NV;                        // the inverse's pivot row
  int* gsi = reinterpret_cast<int*>(prow + Q::GJ::smem_floats);
  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const df2* Ap = reinterpret_cast<const df2*>(a.Ap) + le * NV * NV;
  const df2* Cp = reinterpret_cast<const df2*>(a.Cp) + le * NT * NV;
  float* pre = a.prep + le * Q::prep_floats;
  int* eA = reinterpret_cast<int*>(pre + Q::PREP_EA);
  int* eC = reinterpret_cast<int*>(pre + Q::PREP_EC);

  // A'^T (FP32 high words) into shared memory by asynchronous copies, all in flight together;
  // the row exponents of C' meanwhile, then those of A' from shared memory
  for (int t = tid; t < NV * NV; t += PTH) {
    const int r = t / NV, k = t % NV;
    cp_async4(G + k * LDA + r, &Ap[t].hi);
  }
  cp_async_commit();
  if constexpr (LDA > NV)
    for (int t = tid; t < NV * (LDA - NV); t += PTH) G[(t / (LDA - NV)) * LDA + NV + t % (LDA - NV)] = 0.f;
  for (int r = NV + tid; r < MTA * 16; r += PTH) eA[r] = 0;
  cp_async_wait_all();
  __syncthreads();
  // equilibration sc = |diag A'|^-1/2; the column scales P (powers of two) of the slices
  for (int r = tid; r < LDA; r += PTH) {
    float v = 1.f;
    if (r < NV) {
      const float d = fabsf(G[r * LDA + r]);
      v = d > 0.f ? rsqrtf(d) : 1.f;
      sc[r] = v;
    }
    pre[Q::PREP_SC + r] = v;
  }
  __syncthreads();
  {  // row exponents of C' P: four rows per warp at a time, all their loads in flight together
    constexpr int RB = 4, KQ = (NV + 31) / 32;
    for (int r0 = warp * RB; r0 < MTC * 16; r0 += NWARP * RB) {
      float mx[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        mx[j] = 0.f;
        const int r = r0 + j;
#pragma unroll
        for (int m = 0; m < KQ; ++m) {
          const int k = lane + 32 * m;
          if (r < NT && k < NV) mx[j] = fmaxf(mx[j], fabsf(Cp[r * NV + k].hi) * oz_pow2_floor(sc[k]));
        }
      }
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        for (int off = 16; off > 0; off >>= 1) mx[j] = fmaxf(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], off));
        if (lane == 0 && r0 + j < MTC * 16) eC[r0 + j] = oz_exponent(mx[j]);
      }
    }
  }
  for (int r = warp; r < NV; r += NWARP) {  // row exponents of A' P
    float mx = 0.f;
    for (int k = lane; k < NV; k += 32) mx = fmaxf(mx, fabsf(G[k * LDA + r]) * oz_pow2_floor(sc[k]));
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) eA[r] = oz_exponent(mx);
  }
  {  // A'^T out
    const float4* src = reinterpret_cast<const float4*>(G);
    float4* dst = reinterpret_cast<float4*>(pre + Q::PREP_AH);
    for (int t = tid; t < NV * LDA / 4; t += PTH) dst[t] = src[t];
  }
  __syncthreads();
  for (int t = tid; t < NV * LDA; t += PTH) {
    const int k = t / LDA, r = t % LDA;
    G[t] = r < NV ? G[t] * sc[r] * sc[k] : 0.f;
  }
  __syncthreads();
  // slices of the rows of A' and C' as the right operand (one warp per 16 x 8 tile)
  if constexpr (UMMA) {
    prep_write_umma_slices<C, OZS>(a, le, Ap, Cp, sc, eA, eC);
  } else {
    constexpr int NTA = Q::NTA, NTC = Q::NTC;
    uint2* sl = reinterpret_cast<uint2*>(a.oz) + le * Q::slice_u2;
    auto colP = [&](df2 v, int k) {  // A'[n][k] P[k], C'[n][k] P[k]: exact
      const float pk = oz_pow2_floor(sc[k]);
      return df2{v.hi * pk, v.lo * pk};
    };
    auto getA = [&](int k, int n) { return (n < NV && k < NV) ? colP(Ap[n * NV + k], k) : df2{0.f, 0.f}; };
    auto getC = [&](int k, int n) { return (n < NT && k < NV) ? colP(Cp[n * NV + k], k) : df2{0.f, 0.f}; };
    auto sA = [&](int n) { return oz_scale(eA[n]); };
    auto sC = [&](int n) { return oz_scale(eC[n]); };
    for (int u = warp; u < (NTA + NTC) * KT; u += NWARP) {
      const int nt = u / KT, kt = u % KT;
      if (nt < NTA)
        oz_slice_right_tile<OZS>(sl + (size_t)u * OZS * 32, 32, kt * 16, nt * 8, lane, getA, sA);
      else
        oz_slice_right_tile<OZS>(sl + (size_t)u * OZS * 32, 32, kt * 16, (nt - NTA) * 8, lane, getC, sC);
    }
  }
  // inverse of the transposed equilibrated matrix
  const bool ok = gj_inverse_reg<NV, LDA, PTH>(G, gsi, prow);
  float* ai = pre + Q::PREP_AI;
  for (int t = tid; t < NV * LDA; t += PTH) ai[t] = (t % LDA) < NV ? G[t] : 0.f;
  if (tid == 0 && !ok) atomicOr(a.status + e, HDG_STATUS_SINGULAR);
}

template <class C, int NTHREADS, int OZS>
__global__ void __launch_bounds__(NTHREADS) k_condense_tc(AssembleArgs a) {
  using Q = CondTC<C, NTHREADS, OZS>;
  constexpr int NV = C::NV, NT = C::NT, KT = Q::KT, MTA = Q::MTA, MTC = Q::MTC, CB = Q::CB;
  constexpr int RT = Q::RT, CT = Q::CT, LDA = Q::LDA, NWARP = NTHREADS / 32;
  extern __shared__ double smem_d[];
  df2* Ds = reinterpret_cast<df2*>(smem_d);                 // [NT][CB] D' columns of the block
  df2* Xb = Ds + NT * CB;                                   // [NV][CB] current X block
  uint4* Xs = reinterpret_cast<uint4*>(Xb + NV * CB);       // [KT][NMB][OZS][32] slices of X^T
  float* Rk = reinterpret_cast<float*>(Xs);                 // [NV][CB] residual (aliases Xs)
  float* Dk = Rk + NV * CB;                                 // [NV][CB] correction (aliases Xs)
  // FP32 matrices stored transposed ([k][r], leading dimension LDA, zero past NV)
  float* Ai = reinterpret_cast<float*>(reinterpret_cast<char*>(Xs) + Q::xs_bytes);  // (sc A' sc)^-T
  float* Ah = Ai + NV * LDA;                                // A'^T (FP32)
  float* W = Ah + NV * LDA;                                 // [NV][CB]
  float* sc = W + NV * CB;                                  // [NV]
  int* eA = reinterpret_cast<int*>(sc + NV);                // [MTA*16] row exponents of A'
  int* eC = eA + MTA * 16;                                  // [MTC*16] row exponents of C'
  int* eX = eC + MTC * 16;                                  // [CB] column exponents of the X block
  __shared__ int s_bad;
  __shared__ float s_corr[2], s_xmax;
  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint2* slA = reinterpret_cast<const uint2*>(a.oz) + le * Q::slice_u2;
  const uint2* slC = slA + (size_t)Q::NTA * KT * OZS * 32;
  double* Xg = a.recov + e * (int64_t)(NV * NT + NV);  // B' (double-float) in, X out
  const df2* Bd = reinterpret_cast<const df2*>(Xg);
  double* yg = Xg + NV * NT;
  double* S = a.S + e * (int64_t)NT * NT;  // D' (double-float) in, S out
  const df2* Dd = reinterpret_cast<const df2*>(S);
  const double* R = a.R + e * (int64_t)(NV + NT);

  // ---- the element's prepared operands: Ai^T, A'^T, sc, row exponents
  {
    const float* pre = a.prep + le * Q::prep_floats;
    const float4* src = reinterpret_cast<const float4*>(pre);
    float4* dst = reinterpret_cast<float4*>(Ai);  // Ai and Ah are contiguous, as in the block
    for (int t = tid; t < 2 * NV * LDA / 4; t += NTHREADS) dst[t] = src[t];
    for (int r = tid; r < NV; r += NTHREADS) sc[r] = pre[Q::PREP_SC + r];
    const int* ex = reinterpret_cast<const int*>(pre + Q::PREP_EA);
    for (int r = tid; r < (MTA + MTC) * 16; r += NTHREADS) eA[r] = ex[r];  // eC follows eA
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();

  auto col_exponents = [&]() {  // eX[c] from the current X block, rows scaled by P^-1
    for (int c = warp; c < CB; c += NWARP) {
      float mx = 0.f;
      for (int r = lane; r < NV; r += 32) mx = fmaxf(mx, fabsf(Xb[r * CB + c].hi) / oz_pow2_floor(sc[r]));
      for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (lane == 0) eX[c] = oz_exponent(mx);
    }
  };
  auto slice_X = [&](int nmt) {  // (P^-1 X)^T of the block as the left operand
    auto getX = [&](int c, int k) {
      if (k >= NV) return df2{0.f, 0.f};
      const float ip = 1.f / oz_pow2_floor(sc[k]);
      const df2 x = Xb[k * CB + c];
      return df2{x.hi * ip, x.lo * ip};
    };
    auto sX = [&](int c) { return oz_scale(eX[c]); };
    for (int u = warp; u < KT * nmt; u += NWARP) {
      const int kt = u / nmt, m = u % nmt;
      oz_slice_left_tile<OZS>(Xs + (kt * Q::NMB + m) * OZS * 32, 32, m * 16, kt * 16, lane, getX, sX);
    }
  };

  // ---- blocks of right-hand sides
  for (int c0 = 0; c0 < NT + 1; c0 += CB) {
    const int nc = (NT + 1 - c0) < CB ? (NT + 1 - c0) : CB;
    const int nmt = (nc + 15) / 16;
    // the block's D' columns, read by the Schur epilogue, copied in the background meanwhile
    for (int t = tid; t < NT * CB; t += NTHREADS) {
      const int r = t / CB, c = t % CB;
      if (c < nc && c0 + c < NT) cp_async8(Ds + t, Dd + (size_t)r * NT + c0 + c);
    }
    cp_async_commit();
    auto bval = [&](int r, int c) -> df2 {  // B' column or R_v, zero past the block
      const int col = c0 + c;
      if (c >= nc) return df2{0.f, 0.f};
      return col < NT ? Bd[r * NT + col] : df_from(R[r]);
    };
    {  // all of a thread's B' loads in flight together
      constexpr int NWI = (NV * CB + NTHREADS - 1) / NTHREADS;
      df2 bv[NWI];
#pragma unroll
      for (int x = 0; x < NWI; ++x) {
        const int t = tid + x * NTHREADS;
        bv[x] = t < NV * CB ? bval(t / CB, t % CB) : df2{0.f, 0.f};
      }
#pragma unroll
      for (int x = 0; x < NWI; ++x) {
        const int t = tid + x * NTHREADS;
        if (t < NV * CB) W[t] = (bv[x].hi + bv[x].lo) * sc[t / CB];
      }
    }
    if (tid < 2) s_corr[tid] = 0.f;
    if (tid == 0) s_xmax = 0.f;
    __syncthreads();
    // X0 = sc Ai W
    cond_gemm_f32<NV, LDA, CB, RT, CT, NTHREADS>(Ai, W, [&](int r0, int cc0, float(&acc)[RT][CT]) {
#pragma unroll
      for (int i = 0; i < RT; ++i)
        if (r0 + i < NV)
#pragma unroll
          for (int j = 0; j < CT; ++j) Xb[(r0 + i) * CB + cc0 + j] = df2{acc[i][j] * sc[r0 + i], 0.f};
    });
    __syncthreads();
    col_exponents();
    __syncthreads();
    slice_X(nmt);
    __syncthreads();
    // r0 = B - A' X0 (exact slices), staged in W (the products read Xs, which Rk aliases)
    cond_oz_product<KT, Q::NMB, OZS, NWARP>(slA, Q::NTA, Xs, nmt, [&](int row, int col, const dfacc& v) {
      if (row < NV) {
        const df2 p = oz_scaled(v, eA[row] + eX[col]);
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
      cond_gemm_f32<NV, LDA, CB, RT, CT, NTHREADS>(Ai, W, [&](int r0, int cc0, float(&acc)[RT][CT]) {
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
      cond_gemm_f32<NV, LDA, CB, RT, CT, NTHREADS>(Ah, Dk, [&](int r0, int cc0, float(&acc)[RT][CT]) {
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
      if (!((double)cl * (double)cl <= (double)a.refine_tol * (double)s_xmax * (double)cp)) s_bad |= HDG_STATUS_REFINE;
    }
    // store X and y for the recovery
    for (int t = tid; t < NV * CB; t += NTHREADS) {
      const int r = t / CB, c = t % CB, col = c0 + c;
      if (c < nc) {
        const double xv = df_to_f64(Xb[t].hi, Xb[t].lo);
        if (col < NT)
          Xg[r * NT + col] = xv;
        else
          yg[r] = xv;
      }
    }
    col_exponents();
    __syncthreads();
    slice_X(nmt);
    cp_async_wait_all();
    __syncthreads();
    // S[:, block] = D' - C' X ; g = R_t - C' y
    cond_oz_product<KT, Q::NMB, OZS, NWARP>(slC, Q::NTC, Xs, nmt, [&](int row, int col, const dfacc& v) {
      const int gc = c0 + col;
      if (row >= NT || col >= nc) return;
      const df2 p = oz_scaled(v, eC[row] + eX[col]);
      dfacc t;
      if (gc < NT)
        t.add(Ds[row * CB + col]);
      else
        t.add(df_from(R[NV + row]));
      t.add(df2{-p.hi, -p.lo});
      if (gc < NT)
        S[row * NT + gc] = df_to_f64(t.hi, t.lo);
      else
        a.g[e * NT + row] = df_to_f64(t.hi, t.lo);
    });
    __syncthreads();
  }
  if (tid == 0 && s_bad) atomicOr(a.status + e, s_bad);
}

// ------------------------------------------------------------------------------------
// k_condense_tc2: the condensation of k_condense_tc in blocks of CB = 16 right-hand sides
// and without the FP32 copy of A': the second residual r1 = r0 - A' d0 comes from the first
// OZR = 4 exact slices of A' and of d0 on the tensor cores. Slices hold an entry to a power
// of two below its row's (column's) largest, not below itself as FP32 does: with three the
// small entries of A' lose about two digits against FP32 and X misses 1e-10; four give
// 2^-33 of the largest, as accurate as the FP32 product. About 108 KB of shared memory, so
// that two CTAs share an SM and one hides the other's latency. Launched with two CTAs per
// element (grid 2 ne).
// ------------------------------------------------------------------------------------
template <class C, int NTHREADS, int OZS>
struct CondTC2 {
  static constexpr int NV = C::NV, NT = C::NT;
  static constexpr int KT = (NV + 15) / 16, MTA = KT, MTC = (NT + 15) / 16;
  static constexpr int CB = 16, NMB = 1;
  static constexpr int RT = 2, CT = 4;
  static constexpr int LDA = (NV + 3) / 4 * 4;
  static constexpr int NTA = (NV + 7) / 8, NTC = (NT + 7) / 8;
  static constexpr int OZR = 4;
  static constexpr size_t xs_bytes = sizeof(uint4) * KT * NMB * OZS * 32;
  static constexpr size_t rk_bytes = sizeof(float) * NV * CB;  // r0, then the slices of d0
  static_assert(rk_bytes % 16 == 0 && rk_bytes + sizeof(uint4) * KT * NMB * OZR * 32 <= xs_bytes,
                "r0 and the slices of d0 share the X slice buffer");
  static constexpr size_t bytes = sizeof(df2) * (NT + NV) * CB + xs_bytes +
                                  sizeof(float) * (NV * LDA + NV * CB + NV) + sizeof(int) * (MTA * 16 + MTC * 16 + CB) +
                                  64;
};

template <class C, int NTHREADS, int OZS>
__global__ void __launch_bounds__(NTHREADS, 2) k_condense_tc2(AssembleArgs a) {
  // every block re-reads the slices of A' and C', and two elements per SM keep about as many
  // of them in flight as L2 holds: each warp asks L2 for its next task's fragments
  constexpr bool PF = true;
  using Q = CondTC2<C, NTHREADS, OZS>;
  using P = CondTC<C, 256, OZS>;  // the prep block and the slices of A', C'
  constexpr int NV = C::NV, NT = C::NT, KT = Q::KT, MTA = Q::MTA, MTC = Q::MTC, CB = Q::CB, OZR = Q::OZR;
  constexpr int RT = Q::RT, CT = Q::CT, LDA = Q::LDA, NWARP = NTHREADS / 32;
  static_assert(LDA == P::LDA, "prep layout");
  extern __shared__ double smem_d[];
  df2* Ds = reinterpret_cast<df2*>(smem_d);                                         // [NT][CB] D' columns
  df2* Xb = Ds + NT * CB;                                                           // [NV][CB] X block
  uint4* Xs = reinterpret_cast<uint4*>(Xb + NV * CB);                               // [KT][OZS][32] X^T slices
  float* Rk = reinterpret_cast<float*>(Xs);                                         // [NV][CB] r0 (aliases Xs)
  uint4* Xd = reinterpret_cast<uint4*>(reinterpret_cast<char*>(Xs) + Q::rk_bytes);  // [KT][OZR][32] d0^T slices
  float* Ai = reinterpret_cast<float*>(reinterpret_cast<char*>(Xs) + Q::xs_bytes);  // (sc A' sc)^-T [NV][LDA]
  float* W = Ai + NV * LDA;                                                         // [NV][CB]
  float* sc = W + NV * CB;                                                          // [NV]
  int* eA = reinterpret_cast<int*>(sc + NV);                                        // [MTA*16]
  int* eC = eA + MTA * 16;                                                          // [MTC*16]
  int* eX = eC + MTC * 16;                                                          // [CB]
  __shared__ int s_bad;
  __shared__ float s_corr[2], s_xmax;
  // two CTAs per element, on the even and the odd blocks of right-hand sides: the slices of
  // A' and C' that every block re-reads are then live for half as many elements at a time
  const int64_t le = blockIdx.x >> 1;
  const int half = (int)(blockIdx.x & 1);
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint2* slA = reinterpret_cast<const uint2*>(a.oz) + le * P::slice_u2;
  const uint2* slC = slA + (size_t)P::NTA * KT * OZS * 32;
  double* Xg = a.recov + e * (int64_t)(NV * NT + NV);  // B' (double-float) in, X out
  const df2* Bd = reinterpret_cast<const df2*>(Xg);
  double* yg = Xg + NV * NT;
  double* S = a.S + e * (int64_t)NT * NT;  // D' (double-float) in, S out
  const df2* Dd = reinterpret_cast<const df2*>(S);
  const double* R = a.R + e * (int64_t)(NV + NT);

  {  // the element's prepared operands: Ai^T, sc, row exponents
    const float* pre = a.prep + le * P::prep_floats;
    const float4* src = reinterpret_cast<const float4*>(pre + P::PREP_AI);
    float4* dst = reinterpret_cast<float4*>(Ai);
    for (int t = tid; t < NV * LDA / 4; t += NTHREADS) dst[t] = src[t];
    for (int r = tid; r < NV; r += NTHREADS) sc[r] = pre[P::PREP_SC + r];
    const int* ex = reinterpret_cast<const int*>(pre + P::PREP_EA);
    for (int r = tid; r < (MTA + MTC) * 16; r += NTHREADS) eA[r] = ex[r];  // eC follows eA
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();

  auto col_exponents = [&](auto get) {  // eX[c] = exponent of max_r |get(r, c)|
    for (int c = warp; c < CB; c += NWARP) {
      float mx = 0.f;
      for (int r = lane; r < NV; r += 32) mx = fmaxf(mx, fabsf(get(r, c)));
      for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (lane == 0) eX[c] = oz_exponent(mx);
    }
  };
  auto sX = [&](int c) { return oz_scale(eX[c]); };
  // the products slice P^-1 X and P^-1 d0 (P: powers of two from sc) against A' P and C' P
  auto ipow = [&](int r) { return 1.f / oz_pow2_floor(sc[r]); };
  auto xhi = [&](int r, int c) { return Xb[r * CB + c].hi * ipow(r); };
  auto getXs = [&](int c, int k) {
    if (k >= NV) return df2{0.f, 0.f};
    const float ip = ipow(k);
    const df2 x = Xb[k * CB + c];
    return df2{x.hi * ip, x.lo * ip};
  };

  // W = sc B for the block at column cb: all of a thread's loads in flight together
  auto w_init = [&](int cb) {
    const int ncb = (NT + 1 - cb) < CB ? (NT + 1 - cb) : CB;
    constexpr int NWI = (NV * CB + NTHREADS - 1) / NTHREADS;
    df2 bv[NWI];
#pragma unroll
    for (int x = 0; x < NWI; ++x) {
      const int t = tid + x * NTHREADS, r = t / CB, c = t % CB, col = cb + c;
      bv[x] = (t >= NV * CB || c >= ncb) ? df2{0.f, 0.f} : (col < NT ? Bd[r * NT + col] : df_from(R[r]));
    }
#pragma unroll
    for (int x = 0; x < NWI; ++x) {
      const int t = tid + x * NTHREADS;
      if (t < NV * CB) W[t] = (bv[x].hi + bv[x].lo) * sc[t / CB];
    }
  };
  if (half * CB < NT + 1) w_init(half * CB);
  for (int c0 = half * CB; c0 < NT + 1; c0 += 2 * CB) {
    const int nc = (NT + 1 - c0) < CB ? (NT + 1 - c0) : CB;
    // the block's D' columns, read by the Schur epilogue, copied in the background meanwhile
    for (int t = tid; t < NT * CB; t += NTHREADS) {
      const int r = t / CB, c = t % CB;
      if (c < nc && c0 + c < NT) cp_async8(Ds + t, Dd + (size_t)r * NT + c0 + c);
    }
    cp_async_commit();
    auto bval = [&](int r, int c) -> df2 {  // B' column or R_v, zero past the block
      const int col = c0 + c;
      if (c >= nc) return df2{0.f, 0.f};
      return col < NT ? Bd[r * NT + col] : df_from(R[r]);
    };
    if (tid < 2) s_corr[tid] = 0.f;
    if (tid == 0) s_xmax = 0.f;
    __syncthreads();
    // X0 = sc Ai W
    cond_gemm_f32<NV, LDA, CB, RT, CT, NTHREADS>(Ai, W, [&](int r0, int cc0, float(&acc)[RT][CT]) {
#pragma unroll
      for (int i = 0; i < RT; ++i)
        if (r0 + i < NV)
#pragma unroll
          for (int j = 0; j < CT; ++j) Xb[(r0 + i) * CB + cc0 + j] = df2{acc[i][j] * sc[r0 + i], 0.f};
    });
    __syncthreads();
    col_exponents(xhi);
    __syncthreads();
    for (int kt = warp; kt < KT; kt += NWARP) oz_slice_left_tile<OZS>(Xs + kt * OZS * 32, 32, 0, kt * 16, lane, getXs, sX);
    __syncthreads();
    // r0 = B - A' X0 (exact slices) into W
    cond_oz_product<KT, 1, OZS, NWARP, OZS, PF>(slA, Q::NTA, Xs, 1, [&](int row, int col, const dfacc& v) {
      if (row < NV) {
        const df2 p = oz_scaled(v, eA[row] + eX[col]);
        dfacc t;
        t.add(bval(row, col));
        t.add(df2{-p.hi, -p.lo});
        W[row * CB + col] = col < nc ? t.hi + t.lo : 0.f;
      }
    });
    __syncthreads();
    for (int t = tid; t < NV * CB; t += NTHREADS) {  // Rk = r0 (the X slices are done), W = sc r0
      const float rv = W[t];
      Rk[t] = rv;
      W[t] = rv * sc[t / CB];
    }
    __syncthreads();
    // d0 = sc Ai W, in place in W; X += d0
    cond_gemm_f32<NV, LDA, CB, RT, CT, NTHREADS, true>(Ai, W, [&](int r0, int cc0, float(&acc)[RT][CT]) {
      float cmax = 0.f;
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
            Xb[t] = u.norm();
            W[t] = corr;
            cmax = fmaxf(cmax, fabsf(corr));
          }
      atomicMax(reinterpret_cast<int*>(&s_corr[0]), __float_as_int(cmax));
    });
    __syncthreads();
    // r1 = r0 - A' d0 from four slices of each, W = sc r1
    col_exponents([&](int r, int c) { return W[r * CB + c] * ipow(r); });
    __syncthreads();
    for (int kt = warp; kt < KT; kt += NWARP) {
      auto getD = [&](int c, int k) { return df2{k < NV ? W[k * CB + c] * ipow(k) : 0.f, 0.f}; };
      oz_slice_left_tile<OZR>(Xd + kt * OZR * 32, 32, 0, kt * 16, lane, getD, sX);
    }
    __syncthreads();
    cond_oz_product<KT, 1, OZR, NWARP, OZS, PF>(slA, Q::NTA, Xd, 1, [&](int row, int col, const dfacc& v) {
      if (row < NV) {
        const df2 p = oz_scaled(v, eA[row] + eX[col]);
        W[row * CB + col] = col < nc ? ((Rk[row * CB + col] - p.hi) - p.lo) * sc[row] : 0.f;
      }
    });
    __syncthreads();
    // d1 = sc Ai W; X += d1
    cond_gemm_f32<NV, LDA, CB, RT, CT, NTHREADS>(Ai, W, [&](int r0, int cc0, float(&acc)[RT][CT]) {
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
            cmax = fmaxf(cmax, fabsf(corr));
            xmax = fmaxf(xmax, fabsf(xn.hi));
          }
      atomicMax(reinterpret_cast<int*>(&s_corr[1]), __float_as_int(cmax));
      atomicMax(reinterpret_cast<int*>(&s_xmax), __float_as_int(xmax));
    });
    __syncthreads();
    // the error left after the second correction is ~ c_last^2 / c_prev
    if (tid == 0) {
      const float cl = s_corr[1], cp = s_corr[0];
      if (!((double)cl * (double)cl <= (double)a.refine_tol * (double)s_xmax * (double)cp)) s_bad |= HDG_STATUS_REFINE;
    }
    // store X and y for the recovery
    for (int t = tid; t < NV * CB; t += NTHREADS) {
      const int r = t / CB, c = t % CB, col = c0 + c;
      if (c < nc) {
        const double xv = df_to_f64(Xb[t].hi, Xb[t].lo);
        if (col < NT)
          Xg[r * NT + col] = xv;
        else
          yg[r] = xv;
      }
    }
    col_exponents(xhi);
    __syncthreads();
    for (int kt = warp; kt < KT; kt += NWARP) oz_slice_left_tile<OZS>(Xs + kt * OZS * 32, 32, 0, kt * 16, lane, getXs, sX);
    cp_async_wait_all();
    __syncthreads();
    // S[:, block] = D' - C' X ; g = R_t - C' y
    cond_oz_product<KT, 1, OZS, NWARP, OZS, PF>(slC, Q::NTC, Xs, 1, [&](int row, int col, const dfacc& v) {
      const int gc = c0 + col;
      if (row >= NT || col >= nc) return;
      const df2 p = oz_scaled(v, eC[row] + eX[col]);
      dfacc t;
      if (gc < NT)
        t.add(Ds[row * CB + col]);
      else
        t.add(df_from(R[NV + row]));
      t.add(df2{-p.hi, -p.lo});
      if (gc < NT)
        S[row * NT + gc] = df_to_f64(t.hi, t.lo);
      else
        a.g[e * NT + row] = df_to_f64(t.hi, t.lo);
    });
    // W is free since the last correction: warps done with their Schur tasks fill it for
    // this CTA's next block while the others finish
    if (c0 + 2 * CB < NT + 1) w_init(c0 + 2 * CB);
    __syncthreads();
  }
  if (tid == 0 && s_bad) atomicOr(a.status + e, s_bad);
}

}  // namespace hdg
