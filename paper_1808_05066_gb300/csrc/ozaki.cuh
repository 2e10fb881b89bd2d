// Exact-slice products on the bf16 tensor cores (warp-level mma.sync m16n8k16).
//
// A double-float operand is split, with one power-of-two scale per row (left operand) or
// per column (right operand), into S slices whose values are integers of at most 8
// significant bits:
//     a = 2^(E-8) * sum_s alpha_s 2^(-8 s),   |alpha_0| <= 256, |alpha_s>0| <= 128,
// which leaves a remainder below 2^(E-8S-1) (E: the exponent of the row's largest entry).
// Integers of 8 bits are exact in bf16 and their products exact in FP32, so for a
// contraction length K <= 128 every partial sum of
//     Q_d = sum_{s+t=d} sum_k alpha_s(i,k) beta_t(k,j),   d = 0 .. S-1,
// stays an integer below 2^24 and the tensor core's FP32 accumulator holds it exactly.
// The product is then  c_ij = 2^(E_i+F_j-16) sum_d 2^(-8d) Q_d(i,j), combined in
// double-float. Dropping the diagonals d >= S bounds the error by about
// 2^(-8S) * K * max|a_i.| * max|b_.j| (2^-40 for S = 5, 2^-48 for S = 6).
//
// Fragments are stored "fragment-native": the 4 (left) or 2 (right) 32-bit registers a lane
// holds for one 16x16 / 16x8 tile of one slice are contiguous, so a warp loads a tile with
// one 16-byte (8-byte) access per lane.
#pragma once
#include <cuda_bf16.h>

#include "dfloat.cuh"

namespace hdg {

// Integer-valued floats with |x| <= 256 are exact in bf16.
HDG_DEVI unsigned oz_pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}

// Exponent E with max|x| < 2^E (0 for an all-zero row), and the slicing scale 2^(8-E).
HDG_DEVI int oz_exponent(float amax) {
  int E = 0;
  if (amax > 0.f) frexpf(amax, &E);
  return E;
}
HDG_DEVI float oz_scale(int E) { return ldexpf(1.f, 8 - E); }  // per row / column, not per entry

// The power of two P with P <= s < 2P (s > 0). The condensation's products A' X and C' X are
// sliced as (A' P)(P^-1 X) with P from the Jacobi scales of A': the scaling is exact, and it
// evens out the entries of a row of A' (and of a column of X), which each share one slice scale.
HDG_DEVI float oz_pow2_floor(float s) {
  int E = 0;
  frexpf(s, &E);
  return ldexpf(1.f, E - 1);
}

// Slices of one double-float value, scaled by a power of two (|v| scale <= 256).
// Slice 0 is the nearest integer to the high word h; the low word l joins the remainder
// (|r| <= 1/2) in one exact two-sum (t, e). Slices 1 and 2 peel t exactly (scale by 2^8,
// subtract the nearest integer); the two-sum's error e, scaled to the unit of slice 3, is
// added there (|e| <= 1/2 at that unit, so the slice stays within 128; the rounding of that
// addition is below 2^-49 of 2^E); slices 3.. peel what is left. Every slice after the first
// lies in [-128, 128] and the represented value differs from v by less than 2^(E-48).
template <int S>
HDG_DEVI void oz_split(df2 v, float scale, float (&out)[S]) {
  const float h = v.hi * scale, l = v.lo * scale;
  const float q0 = rintf(h);
  out[0] = q0;
  const float r = h - q0;  // exact
  float t = r + l;         // two-sum: t + e = r + l exactly
  const float bb = t - r;
  float e = (r - (t - bb)) + (l - bb);
#pragma unroll
  for (int i = 1; i < S; ++i) {
    t *= 256.f;
    if (i <= 3) e *= 256.f;
    if (i == 3) t += e;
    const float q = rintf(t);
    out[i] = q;
    t -= q;  // exact: |t - q| <= 1/2
  }
}

// Left-operand tile (16 rows x 16 k): element (rr, kk) lives in lane (rr%8)*4 + (kk%8)/2,
// register (rr/8) + 2*(kk/8), half kk%2.  Writes the S slices of the lane's 8 elements.
// get(r, k) returns the element as df2 (zero outside the matrix); rscale(r) its row scale.
template <int S, class Get, class RScale>
HDG_DEVI void oz_slice_left_tile(uint4* dst, int slice_stride, int r0, int k0, int lane, Get get, RScale rscale) {
  const int ra = r0 + (lane >> 2), rb = ra + 8;
  const int ka = k0 + 2 * (lane & 3);
  const float sa = rscale(ra), sb = rscale(rb);
  float v[8][S];
  oz_split<S>(get(ra, ka), sa, v[0]);
  oz_split<S>(get(ra, ka + 1), sa, v[1]);
  oz_split<S>(get(rb, ka), sb, v[2]);
  oz_split<S>(get(rb, ka + 1), sb, v[3]);
  oz_split<S>(get(ra, ka + 8), sa, v[4]);
  oz_split<S>(get(ra, ka + 9), sa, v[5]);
  oz_split<S>(get(rb, ka + 8), sb, v[6]);
  oz_split<S>(get(rb, ka + 9), sb, v[7]);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    uint4 w;
    w.x = oz_pack2(v[0][s], v[1][s]);
    w.y = oz_pack2(v[2][s], v[3][s]);
    w.z = oz_pack2(v[4][s], v[5][s]);
    w.w = oz_pack2(v[6][s], v[7][s]);
    dst[s * slice_stride + lane] = w;
  }
}

// Right-operand tile (16 k x 8 columns): element (kk, nn) lives in lane nn*4 + (kk%8)/2,
// register kk/8, half kk%2.
template <int S, class Get, class CScale>
HDG_DEVI void oz_slice_right_tile(uint2* dst, int slice_stride, int k0, int n0, int lane, Get get, CScale cscale) {
  const int n = n0 + (lane >> 2);
  const int ka = k0 + 2 * (lane & 3);
  const float sc = cscale(n);
  float v[4][S];
  oz_split<S>(get(ka, n), sc, v[0]);
  oz_split<S>(get(ka + 1, n), sc, v[1]);
  oz_split<S>(get(ka + 8, n), sc, v[2]);
  oz_split<S>(get(ka + 9, n), sc, v[3]);
#pragma unroll
  for (int s = 0; s < S; ++s) dst[s * slice_stride + lane] = make_uint2(oz_pack2(v[0][s], v[1][s]), oz_pack2(v[2][s], v[3][s]));
}

HDG_DEVI void oz_mma(float (&c)[4], const uint4& a, const uint2& b) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
}

// The S(S+1)/2 slice products of one k-tile, accumulated per diagonal d = s + t.
template <int S>
HDG_DEVI void oz_mma_tile(float (&acc)[S][4], const uint4 (&a)[S], const uint2 (&b)[S]) {
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int t = 0; t + s < S; ++t) oz_mma(acc[s + t], a[s], b[t]);
}

// Combines the diagonals of one accumulator element: sum_d 2^(-8(d+2)) Q_d in double-float
// (every term is exact in FP32), without the row and column scales.
template <int S>
HDG_DEVI dfacc oz_combine(const float (&acc)[S][4], int q) {
  dfacc r;
  float w = 1.f / 65536.f;
#pragma unroll
  for (int d = 0; d < S; ++d) {
    r.add(df2{acc[d][q] * w, 0.f});
    w *= (1.f / 256.f);
  }
  return r;
}

// 2^e as a float for |e| <= 126 (built from the exponent field).
HDG_DEVI float oz_pow2(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __int_as_float((e + 127) << 23);
}

// v * 2^e as a double-float (the row and column scales of a slice product). Two factors
// keep e over the whole float range.
HDG_DEVI df2 oz_scaled(const dfacc& v, int e) {
  const int e1 = e / 2, e2 = e - e1;
  const float p1 = oz_pow2(e1), p2 = oz_pow2(e2);
  const df2 n = v.norm();
  return {n.hi * p1 * p2, n.lo * p1 * p2};
}

// Asynchronous 16-byte copies global -> shared (cp.async, L2 only) and their completion.
HDG_DEVI void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
HDG_DEVI void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
HDG_DEVI void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Asynchronous 4-byte copy global -> shared (cp.async, L1-allocating).
HDG_DEVI void cp_async4(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

// Asynchronous 8-byte copy global -> shared (cp.async, L1-allocating).
HDG_DEVI void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

}  // namespace hdg
