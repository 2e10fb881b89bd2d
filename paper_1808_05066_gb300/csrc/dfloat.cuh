// Double-float arithmetic: a value is an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, about 48 significant bits. Products use the exact FMA residual
// of hi*hi (Dekker's product with a fused multiply-add); sums use Knuth's branch-free
// two-sum. On GB300 the FP32 pipe issues ~62x the FP64 rate, so a double-float
// multiply-accumulate (~12 FP32 operations) is ~5x faster than an FP64 one while
// keeping a relative error near 2^-44 per operation.
#pragma once
#include "hdg_device.cuh"

namespace hdg {

struct __align__(8) df2 {
  float hi, lo;
};

HDG_DEVI df2 df_from(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return {h, l};
}
HDG_DEVI double df_val(df2 a) { return (double)a.hi + (double)a.lo; }

// Accumulator kept unnormalised: hi collects the leading parts exactly (two-sum), lo the
// rounding errors and the cross products.
struct dfacc {
  float hi = 0.f, lo = 0.f;
  HDG_DEVI void mac(const df2& a, const df2& b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s = hi + p;
    float bb = s - hi;
    float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += err + e;
  }
  HDG_DEVI void add(const df2& a) {
    float s = hi + a.hi;
    float bb = s - hi;
    float err = (hi - (s - bb)) + (a.hi - bb);
    hi = s;
    lo += err + a.lo;
  }
  HDG_DEVI double value() const { return (double)hi + (double)lo; }
  HDG_DEVI df2 norm() const {
    float s = hi + lo;
    return {s, lo - (s - hi)};
  }
};

// Exact double of a float built from its bit fields on the integer pipe (the FP64 pipe of
// GB300 runs at 1/64 of the FP32 rate); zero and normal numbers; other classes take the
// conversion instruction.
HDG_DEVI double f32_to_f64_bits(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (ex == 0u && (u << 1) == 0u) return __longlong_as_double((long long)sign);
  if (ex == 0u || ex == 0xffu) return (double)x;
  const unsigned long long bits = sign | ((unsigned long long)(ex + 896u) << 52) |  // 1023 - 127
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// hi + lo of a double-float in FP64: one FP64 addition.
HDG_DEVI double df_to_f64(float hi, float lo) { return f32_to_f64_bits(hi) + f32_to_f64_bits(lo); }

}  // namespace hdg
