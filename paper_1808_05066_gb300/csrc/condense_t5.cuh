// Static condensation of the mixed form on the fifth-generation tensor cores: tcgen05.mma with
// accumulators in tensor memory (TMEM), operands in shared memory, the element's prepared
// slices streamed in by bulk asynchronous copies (cp.async.bulk) that complete on mbarriers.
//
// The arithmetic is that of k_condense_tc2 (Sec. 3.2 local elimination, S = D' - C' A'^{-1} B',
// g = R_t - C' A'^{-1} R_v, X refined to FP64 accuracy), per block of NB right-hand sides:
//   X0 = sc Ai sc B                      FP32 (CUDA cores)
//   r0 = B - A' X0                       21 exact slice products   (tcgen05, 6 TMEM accumulators)
//   d0 = sc Ai sc r0, X = X0 + d0        FP32
//   r1 = r0 - A' d0                      10 products of 4 slices   (tcgen05, 4 accumulators)
//   d1 = sc Ai sc r1, X += d1            FP32
//   S = D' - C' X, g = R_t - C' y        21 exact slice products per 128-row tile of C'
// Every product is (A' P)(P^-1 X) with P the power-of-two Jacobi scales (exact). Each slice
// diagonal d = s + t has its own FP32 accumulator in TMEM; every partial sum is an integer below
// 2^24 in the diagonal's unit, so the accumulation is exact, and the diagonals are combined in
// double-float in the epilogue (as in ozaki.cuh).
//
// Operand layouts (tcgen05 "no swizzle, K-major"): an R x 16 tile of bf16 is stored as core
// matrices of 8 rows x 16 bytes, [row group][k group (2)][8 rows][8 entries]; the leading byte
// offset (next k group) is 128, the stride byte offset (next row group) 256.
//   A operand: 128 rows of A' P or C' P (M = 128) x one k step of 16 interior unknowns, one
//              4 KB block per slice; prepared per element by k_condense_prep<..., true> as
//              [tile (A', C' rows 0-127, C' rows 128-255)][k step][slice][4 KB].
//   B operand: NB columns of P^-1 X (N = NB) x 16, written by the warps into shared memory,
//              [k step][slice][NB x 16 bf16].
// TMEM: D row i = lane i, column j = column base + j (M = 128, cta_group::1); accumulator of
// diagonal d for tile mt at column (mt * OZS + d) * NB.
//
// One CTA of 256 threads per element, one CTA per SM (shared memory), 512 TMEM columns. Thread 0
// issues the bulk copies (a ring of NSLOT stages of one k step x all slices, up to NSLOT - 1 jobs
// ahead) and the MMAs; the FP32 inverse stays in shared memory for the GEMMs; all waits
// are bounded: a wait that gives up sets HDG_STATUS_TIMEOUT, the kernel lets its own copies and
// MMAs drain (with a bounded wait), frees its TMEM and returns.
#pragma once
#include "condense_tc.cuh"
#include "ptx_async.cuh"

namespace hdg {

// ---------------------------------------------------------------------------------------------
// PTX wrappers (the mbarrier and bulk-copy ones are in ptx_async.cuh)
// ---------------------------------------------------------------------------------------------
HDG_DEVI void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
HDG_DEVI void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets (16-byte units),
// the fixed version bits 0b001 at [46, 49), no swizzle.
HDG_DEVI uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: D in FP32, A and B bf16, both K-major, N and M.
template <int M, int N>
struct UmmaIdesc {
  static_assert(M == 128 && N % 16 == 0 && N >= 16 && N <= 256, "cta_group::1 shape");
  static constexpr uint32_t value = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                                    ((uint32_t)(M >> 4) << 24);
};
HDG_DEVI void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives once on `bar` when every tcgen05 operation this thread issued before has completed.
HDG_DEVI void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 8 consecutive FP32 columns of the warp's 32 TMEM lanes (lane i of the warp: TMEM lane
// 32 (warp % 4) + i); waits for the load.
HDG_DEVI void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// Byte offset of entry (row, k) (k < 16) of an R x 16 K-major tile in the core-matrix layout.
HDG_DEVI uint32_t umma_off(int row, int k) {
  return (uint32_t)((((row >> 3) * 2 + (k >> 3)) * 8 + (row & 7)) * 16 + (k & 7) * 2);
}

// Slices of the pair (v0, v1) (adjacent k, k even) written as bf16x2 to S slice blocks.
template <int S>
HDG_DEVI void umma_put_pair(unsigned char* blk, uint32_t blk_stride, uint32_t off, df2 v0, df2 v1, float scale) {
  float a[S], b[S];
  oz_split<S>(v0, scale, a);
  oz_split<S>(v1, scale, b);
#pragma unroll
  for (int s = 0; s < S; ++s) *reinterpret_cast<unsigned*>(blk + s * blk_stride + off) = oz_pack2(a[s], b[s]);
}

// ---------------------------------------------------------------------------------------------
// sizes and layout
// ---------------------------------------------------------------------------------------------
template <class C, int OZS>
struct CondT5 {
  static constexpr int NV = C::NV, NT = C::NT;
  static_assert(NV <= 128 && NT <= 256, "one 128-row tile of A', two of C'");
  static constexpr int KT = (NV + 15) / 16;            // k steps of 16 interior unknowns
  static constexpr int MTC = (NT + 127) / 128;         // 128-row tiles of C'
  static constexpr int NTILE = 1 + MTC;
  static constexpr int NB = 32;                        // right-hand sides per block
  static constexpr int OZR = 4;                        // slices of the second residual
  static constexpr int NSLOT = 3;                      // stages of the A-operand ring
  static constexpr int NTH = 256;
  static constexpr uint32_t TILE = 128 * 16 * 2;      // one slice of one k step of one tile
  static constexpr uint32_t BTILE = NB * 16 * 2;      // one slice of one k step of the X block
  static constexpr int TMEM_COLS = 512;
  static_assert(MTC * OZS * NB <= TMEM_COLS, "Schur accumulators fit in TMEM");
  // per element: [tile][k step][slice][TILE]
  static constexpr size_t slice_bytes = (size_t)NTILE * KT * OZS * TILE;
  static constexpr int LDA = (NV + 3) / 4 * 4;
  // jobs of one block: r0 (A', KT steps, OZS slices), r1 (A', KT, OZR), S (C' tiles, KT x MTC, OZS)
  static constexpr int NJOB = KT * (2 + MTC);
  // shared memory
  static constexpr size_t a_bytes = (size_t)NSLOT * OZS * TILE;
  static constexpr size_t b_bytes = (size_t)KT * OZS * BTILE;
  static constexpr size_t ai_bytes = sizeof(float) * NV * LDA;  // the FP32 inverse, read by every GEMM
  static constexpr size_t bytes = a_bytes + b_bytes + sizeof(df2) * NV * NB + sizeof(float) * 2 * NV * NB +
                                  ai_bytes + sizeof(float) * 128 + sizeof(int) * (128 + 128 * MTC + NB) +
                                  sizeof(uint64_t) * (2 * NSLOT + 1) + 64;
};

// The prep kernel's slices of A' P (tile 0) and C' P (tiles 1, 2) in the tcgen05 operand layout,
// rows scaled by their exponents eA / eC (2^(8 - E)), zero past the matrices.
template <class C, int OZS>
HDG_DEVI void prep_write_umma_slices(const AssembleArgs& a, int64_t le, const df2* Ap, const df2* Cp, const float* sc,
                                     const int* eA, const int* eC) {
  using Q = CondT5<C, OZS>;
  constexpr int NV = C::NV, NT = C::NT, KT = Q::KT, NTILE = Q::NTILE;
  unsigned char* dst = reinterpret_cast<unsigned char*>(a.oz) + (size_t)le * Q::slice_bytes;
  auto get = [&](int tile, int r, int k) -> df2 {
    if (k >= NV) return df2{0.f, 0.f};
    df2 v;
    if (tile == 0) {
      if (r >= NV) return df2{0.f, 0.f};
      v = Ap[r * NV + k];
    } else {
      const int rc = (tile - 1) * 128 + r;
      if (rc >= NT) return df2{0.f, 0.f};
      v = Cp[rc * NV + k];
    }
    const float pk = oz_pow2_floor(sc[k]);
    return df2{v.hi * pk, v.lo * pk};
  };
  for (int it = threadIdx.x; it < NTILE * KT * 128 * 8; it += blockDim.x) {
    const int kp = it & 7, r = (it >> 3) & 127, kt = ((it >> 10) % KT), tile = (it >> 10) / KT;
    const int k = kt * 16 + 2 * kp;
    int E;
    if (tile == 0)
      E = r < NV ? eA[r] : 0;
    else
      E = (tile - 1) * 128 + r < NT ? eC[(tile - 1) * 128 + r] : 0;
    umma_put_pair<OZS>(dst + (size_t)(tile * KT + kt) * OZS * Q::TILE, Q::TILE, umma_off(r, 2 * kp), get(tile, r, k),
                       get(tile, r, k + 1), oz_scale(E));
  }
}

// ---------------------------------------------------------------------------------------------
// k_condense_t5
// ---------------------------------------------------------------------------------------------
template <class C, int OZS>
__global__ void __launch_bounds__(256, 1) k_condense_t5(AssembleArgs a) {
  using Q = CondT5<C, OZS>;
  using P = CondTC<C, 256, OZS>;  // the prep block (Ai, sc, exponents)
  constexpr int NV = C::NV, NT = C::NT, KT = Q::KT, MTC = Q::MTC, NB = Q::NB, OZR = Q::OZR;
  constexpr int NSLOT = Q::NSLOT, NTH = Q::NTH, NWARP = NTH / 32, LDA = Q::LDA;
  constexpr uint32_t TILE = Q::TILE, BTILE = Q::BTILE;
  constexpr uint32_t IDESC = UmmaIdesc<128, NB>::value;
  constexpr int WAIT = 1 << 22;  // polls of a bounded wait (about a second with the back-off)
  static_assert(LDA == P::LDA, "prep layout");
  extern __shared__ __align__(128) unsigned char smem_t5[];
  unsigned char* As = smem_t5;                                            // [NSLOT][OZS][TILE]
  unsigned char* Bs = As + Q::a_bytes;                                    // [KT][OZS][BTILE]
  df2* Xb = reinterpret_cast<df2*>(Bs + Q::b_bytes);                      // [NV][NB]
  float* W = reinterpret_cast<float*>(Xb + NV * NB);                      // [NV][NB]
  float* Rk = W + NV * NB;                                                // [NV][NB] r0
  float* Ai = Rk + NV * NB;                                               // (sc A' sc)^-T [NV][LDA]
  float* sc = Ai + NV * LDA;                                              // [128]
  int* eA = reinterpret_cast<int*>(sc + 128);                             // [128]
  int* eC = eA + 128;                                                     // [128 MTC]
  int* eX = eC + 128 * MTC;                                               // [NB]
  uint64_t* full = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(eX + NB) + 7) & ~(uintptr_t)7);
  uint64_t* empty = full + NSLOT;
  uint64_t* accb = empty + NSLOT;
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad, s_fail;
  __shared__ float s_corr[2], s_xmax;

  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned char* slices = reinterpret_cast<const unsigned char*>(a.oz) + (size_t)le * Q::slice_bytes;
  const float* pre = a.prep + le * P::prep_floats;
  double* Xg = a.recov + e * (int64_t)(NV * NT + NV);
  const df2* Bd = reinterpret_cast<const df2*>(Xg);
  double* yg = Xg + NV * NT;
  double* S = a.S + e * (int64_t)NT * NT;
  const df2* Dd = reinterpret_cast<const df2*>(S);
  const double* R = a.R + e * (int64_t)(NV + NT);

  {
    const float4* src = reinterpret_cast<const float4*>(pre + P::PREP_AI);
    float4* dst = reinterpret_cast<float4*>(Ai);
    for (int t = tid; t < NV * LDA / 4; t += NTH) dst[t] = src[t];
  }
  for (int r = tid; r < 128; r += NTH) {
    sc[r] = r < NV ? pre[P::PREP_SC + r] : 1.f;
    eA[r] = r < NV ? reinterpret_cast<const int*>(pre + P::PREP_EA)[r] : 0;
  }
  for (int r = tid; r < 128 * MTC; r += NTH) eC[r] = r < NT ? reinterpret_cast<const int*>(pre + P::PREP_EC)[r] : 0;
  if (tid == 0) {
    s_bad = 0;
    s_fail = 0;
    for (int i = 0; i < 2 * NSLOT + 1; ++i) mbar_init(full + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(Q::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  // ---- the job stream of thread 0 (producer of the A-operand ring and MMA issuer)
  const int nblk = (NT + 1 + NB - 1) / NB;
  const int njobs = nblk * Q::NJOB;
  int next_load = 0, issued = 0;  // thread 0 only
  uint32_t acc_phase = 0;         // uniform
  auto job_src = [&](int J, uint32_t* bytes) {
    const int j = J % Q::NJOB;
    int tile, kt, nsl;
    if (j < KT) {
      tile = 0, kt = j, nsl = OZS;
    } else if (j < 2 * KT) {
      tile = 0, kt = j - KT, nsl = OZR;
    } else {
      const int u = j - 2 * KT;
      tile = 1 + u % MTC, kt = u / MTC, nsl = OZS;
    }
    *bytes = nsl * TILE;
    return slices + ((size_t)(tile * KT + kt) * OZS) * TILE;
  };
  // thread 0: loads jobs ahead of the MMAs, at most NSLOT - 2 past the last one issued, so that
  // a refill waits only for MMAs queued before the ones the tensor cores are working on
  auto produce = [&]() {
    while (next_load < njobs && next_load < issued + NSLOT - 1) {
      const int slot = next_load % NSLOT, use = next_load / NSLOT;
      if (use > 0 && !mbar_wait(empty + slot, (use - 1) & 1, WAIT)) {
        s_fail = 1;
        return;
      }
      uint32_t bytes;
      const unsigned char* src = job_src(next_load, &bytes);
      mbar_arrive_expect_tx(full + slot, bytes);
      if (!(a.stall_first_copy && next_load == 0))  // the test hook leaves this phase incomplete
        bulk_g2s(As + (size_t)slot * OZS * TILE, src, bytes, full + slot);
      ++next_load;
    }
  };
  // thread 0: waits for job J's operands and issues its slice products into the accumulators
  // of `tile` (columns acc0 + d NB); npair products with s + t < nsl
  auto issue = [&](int J, int nsl, uint32_t acc0, int kt) {
    const int slot = J % NSLOT;
    if (s_fail || !mbar_wait(full + slot, (J / NSLOT) & 1, WAIT)) {
      s_fail = 1;
      return;
    }
    tc_fence_after();
    const uint32_t abase = smem_u32(As + (size_t)slot * OZS * TILE), bbase = smem_u32(Bs + (size_t)kt * OZS * BTILE);
    for (int s = 0; s < nsl; ++s)
      for (int t = 0; s + t < nsl; ++t)
        umma_bf16(tmem + acc0 + (uint32_t)((s + t) * NB), umma_desc(abase + s * TILE, 128, 256),
                  umma_desc(bbase + t * BTILE, 128, 256), IDESC, (kt > 0 || s > 0) ? 1u : 0u);
    umma_commit(empty + slot);
    ++issued;
    produce();
  };
  // all threads: the accumulators of the phase are complete
  auto acc_ready = [&]() {
    if (tid == 0) {
      umma_commit(accb);
      produce();  // the next phase's first operands, meanwhile
    }
    const bool ok = mbar_wait(accb, acc_phase & 1, WAIT);
    ++acc_phase;
    if (!ok) s_fail = 1;
    tc_fence_after();
    __syncthreads();  // s_fail is uniform from here
  };
  // the diagonals of one accumulator column as a double-float (without row / column scales)
  auto combine = [&](const float (&v)[OZS]) {
    dfacc r;
    float w = 1.f / 65536.f;
#pragma unroll
    for (int d = 0; d < OZS; ++d) {
      r.add(df2{v[d] * w, 0.f});
      w *= (1.f / 256.f);
    }
    return r;
  };
  // epilogue over one tile's accumulators: f(row in tile, column, value without scales); warp w
  // takes TMEM lanes 32 (w % 4).. and columns 16 (w / 4)..+16 of the block
  auto epilogue = [&](uint32_t acc0, int nacc, auto f) {
    const int q = warp & 3, ch = warp >> 2;
    const int row = 32 * q + lane;
#pragma unroll 1
    for (int c8 = 0; c8 < 2; ++c8) {
      const int col0 = 16 * ch + 8 * c8;
      float v[OZS][8];
#pragma unroll
      for (int d = 0; d < OZS; ++d) {
        if (d < nacc)
          tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + acc0 + (uint32_t)(d * NB + col0), v[d]);
        else
#pragma unroll
          for (int j = 0; j < 8; ++j) v[d][j] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float u[OZS];
#pragma unroll
        for (int d = 0; d < OZS; ++d) u[d] = v[d][j];
        f(row, col0 + j, combine(u));
      }
    }
  };
  auto ipow = [&](int r) { return 1.f / oz_pow2_floor(sc[r]); };
  auto col_exponents = [&](auto get) {  // eX[c] = exponent of max_r |get(r, c)|
    for (int c = warp; c < NB; c += NWARP) {
      float mx = 0.f;
      for (int r = lane; r < NV; r += 32) mx = fmaxf(mx, fabsf(get(r, c)));
      for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (lane == 0) eX[c] = oz_exponent(mx);
    }
  };
  // slices of the block (P^-1 times get) into the B operand: nsl slices
  auto slice_B = [&](auto get, auto nslc) {
    constexpr int NSL = decltype(nslc)::value;
    for (int it = tid; it < KT * NB * 8; it += NTH) {
      const int kp = it & 7, c = (it >> 3) % NB, kt = (it >> 3) / NB;
      const int k = kt * 16 + 2 * kp;
      const df2 v0 = get(k, c), v1 = get(k + 1, c);
      umma_put_pair<NSL>(Bs + (size_t)kt * OZS * BTILE, BTILE, umma_off(c, 2 * kp), v0, v1, oz_scale(eX[c]));
    }
  };

  int blk = 0;
  for (int c0 = 0; c0 < NT + 1; c0 += NB, ++blk) {
    const int nc = (NT + 1 - c0) < NB ? (NT + 1 - c0) : NB;
    const int J0 = blk * Q::NJOB;
    auto bval = [&](int r, int c) -> df2 {
      const int col = c0 + c;
      if (c >= nc) return df2{0.f, 0.f};
      return col < NT ? Bd[r * NT + col] : df_from(R[r]);
    };
    if (tid == 0) produce();
    for (int t = tid; t < NV * NB; t += NTH) W[t] = [&] { const df2 b = bval(t / NB, t % NB); return (b.hi + b.lo) * sc[t / NB]; }();
    if (tid < 2) s_corr[tid] = 0.f;
    if (tid == 0) s_xmax = 0.f;
    __syncthreads();
    // X0 = sc Ai W
    cond_gemm_f32<NV, LDA, NB, 4, 4, NTH>(Ai, W, [&](int r0, int cc0, float(&acc)[4][4]) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (r0 + i < NV)
#pragma unroll
          for (int j = 0; j < 4; ++j) Xb[(r0 + i) * NB + cc0 + j] = df2{acc[i][j] * sc[r0 + i], 0.f};
    });
    __syncthreads();
    col_exponents([&](int r, int c) { return Xb[r * NB + c].hi * ipow(r); });
    __syncthreads();
    auto getX = [&](int k, int c) {
      if (k >= NV) return df2{0.f, 0.f};
      const float ip = ipow(k);
      const df2 x = Xb[k * NB + c];
      return df2{x.hi * ip, x.lo * ip};
    };
    slice_B(getX, std::integral_constant<int, OZS>{});
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // r0 = B - A' X0
    if (tid == 0) {
      tc_fence_after();
      for (int kt = 0; kt < KT; ++kt) issue(J0 + kt, OZS, 0, kt);
    }
    acc_ready();
    if (s_fail) break;
    epilogue(0, OZS, [&](int row, int col, const dfacc& v) {
      if (row < NV) {
        const df2 p = oz_scaled(v, eA[row] + eX[col]);
        dfacc t;
        t.add(bval(row, col));
        t.add(df2{-p.hi, -p.lo});
        const float rv = col < nc ? t.hi + t.lo : 0.f;
        Rk[row * NB + col] = rv;
        W[row * NB + col] = rv * sc[row];
      }
    });
    tc_fence_before();
    __syncthreads();
    // d0 = sc Ai W in place; X += d0
    cond_gemm_f32<NV, LDA, NB, 4, 4, NTH, true>(Ai, W, [&](int r0, int cc0, float(&acc)[4][4]) {
      float cmax = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (r0 + i < NV)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int t = (r0 + i) * NB + cc0 + j;
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
    // r1 = r0 - A' d0 from four slices of each
    col_exponents([&](int r, int c) { return W[r * NB + c] * ipow(r); });
    __syncthreads();
    slice_B([&](int k, int c) { return df2{k < NV ? W[k * NB + c] * ipow(k) : 0.f, 0.f}; },
            std::integral_constant<int, OZR>{});
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int kt = 0; kt < KT; ++kt) issue(J0 + KT + kt, OZR, 0, kt);
    }
    acc_ready();
    if (s_fail) break;
    epilogue(0, OZR, [&](int row, int col, const dfacc& v) {
      if (row < NV) {
        const df2 p = oz_scaled(v, eA[row] + eX[col]);
        W[row * NB + col] = col < nc ? ((Rk[row * NB + col] - p.hi) - p.lo) * sc[row] : 0.f;
      }
    });
    tc_fence_before();
    __syncthreads();
    // d1 = sc Ai W; X += d1
    cond_gemm_f32<NV, LDA, NB, 4, 4, NTH>(Ai, W, [&](int r0, int cc0, float(&acc)[4][4]) {
      float cmax = 0.f, xmax = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (r0 + i < NV)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int t = (r0 + i) * NB + cc0 + j;
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
    if (tid == 0) {  // the error left after the second correction is ~ c_last^2 / c_prev
      const float cl = s_corr[1], cp = s_corr[0];
      if (!((double)cl * (double)cl <= (double)a.refine_tol * (double)s_xmax * (double)cp)) s_bad |= HDG_STATUS_REFINE;
    }
    for (int t = tid; t < NV * NB; t += NTH) {  // X and y for the recovery
      const int r = t / NB, c = t % NB, col = c0 + c;
      if (c < nc) {
        const double xv = df_to_f64(Xb[t].hi, Xb[t].lo);
        if (col < NT)
          Xg[r * NT + col] = xv;
        else
          yg[r] = xv;
      }
    }
    col_exponents([&](int r, int c) { return Xb[r * NB + c].hi * ipow(r); });
    __syncthreads();
    slice_B(getX, std::integral_constant<int, OZS>{});
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // S = D' - C' X, g = R_t - C' y: both 128-row tiles of C' per k step
    if (tid == 0) {
      tc_fence_after();
      for (int kt = 0; kt < KT; ++kt)
        for (int mt = 0; mt < MTC; ++mt) issue(J0 + 2 * KT + kt * MTC + mt, OZS, (uint32_t)(mt * OZS * NB), kt);
    }
    acc_ready();
    if (s_fail) break;
    for (int mt = 0; mt < MTC; ++mt)
      epilogue((uint32_t)(mt * OZS * NB), OZS, [&](int rt, int col, const dfacc& v) {
        const int row = mt * 128 + rt, gc = c0 + col;
        if (row >= NT || col >= nc) return;
        const df2 p = oz_scaled(v, eC[row] + eX[col]);
        dfacc t;
        if (gc < NT)
          t.add(Dd[(size_t)row * NT + gc]);
        else
          t.add(df_from(R[NV + row]));
        t.add(df2{-p.hi, -p.lo});
        if (gc < NT)
          S[(size_t)row * NT + gc] = df_to_f64(t.hi, t.lo);
        else
          a.g[e * NT + row] = df_to_f64(t.hi, t.lo);
      });
    tc_fence_before();
    __syncthreads();
  }
  // drain: every copy issued has landed and every MMA has completed before TMEM is freed
  if (tid == 0) {
    for (int J = issued; J < next_load; ++J) mbar_wait(full + J % NSLOT, (J / NSLOT) & 1, WAIT);
    umma_commit(accb);
  }
  mbar_wait(accb, acc_phase & 1, WAIT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Q::TMEM_COLS) : "memory");
  }
  if (tid == 0 && (s_bad || s_fail)) atomicOr(a.status + e, s_bad | (s_fail ? HDG_STATUS_TIMEOUT : 0));
}

}  // namespace hdg
