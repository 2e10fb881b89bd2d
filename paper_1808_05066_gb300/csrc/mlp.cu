// Per-face MLP that predicts the trace update of the next implicit step, used to
// warm-start Newton (no counterpart in the paper; it serves the Newton solve of the
// method, which stays the judge: the converged answer is the same either way).
//
// Network: x (NIN) -> tanh(W1 x + b1) (NH) -> tanh(W2 h1 + b2) (NH) -> W3 h2 + b3 (NOUT).
// Weights are used in BF16 with FP32 accumulation; an FP32 master copy and the Adam
// moments live in the same parameter buffer:
//   params [P] FP32 master | m [P] | v [P] | w16 [P] BF16 copy used by the kernels,
// P = NH*NIN + NH + NH*NH + NH + NOUT*NH + NOUT, laid out as W1 (row-major [NH][NIN]),
// b1, W2 [NH][NH], b2, W3 [NOUT][NH], b3.
//
// Features of face F (canonical node order), all as differences so the map is
// invariant to the state level: [V_side0 - vhat^n | V_side1 - vhat^n | dvhat^n |
// dvhat^{n-1}] at the NFN face nodes, standardised by per-feature mean and scale.
#include <cuda_bf16.h>

#include <cstdint>

#include "ctx.hpp"

namespace hdg {

namespace {

constexpr int MAXH = 64;  // hidden width supported by the register-resident kernels

__host__ __device__ inline int64_t mlp_params(int nin, int nh, int nout) {
  return (int64_t)nh * nin + nh + (int64_t)nh * nh + nh + (int64_t)nout * nh + nout;
}

// SplitMix64 counter-based generator (Steele, Lea & Flood 2014), used for the initial weights.
__device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_mlp_init(float* params, int nin, int nh, int nout, uint64_t seed) {
  const int64_t P = mlp_params(nin, nh, nout);
  float* m = params + P;
  float* v = m + P;
  __nv_bfloat16* w16 = reinterpret_cast<__nv_bfloat16*>(v + P);
  const int64_t o1 = (int64_t)nh * nin, o2 = o1 + nh, o3 = o2 + (int64_t)nh * nh, o4 = o3 + nh,
                o5 = o4 + (int64_t)nout * nh;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x) {
    float val = 0.f;
    int fan_in = 0, fan_out = 0;
    if (t < o1) {
      fan_in = nin;
      fan_out = nh;
    } else if (t >= o2 && t < o3) {
      fan_in = nh;
      fan_out = nh;
    } else if (t >= o4 && t < o5) {
      fan_in = nh;
      fan_out = nout;
    }
    if (fan_in) {  // Glorot-uniform
      const double u = (double)(splitmix64(seed * 0x100000001B3ull + (uint64_t)t) >> 11) * (1.0 / 9007199254740992.0);
      const double lim = ::sqrt(6.0 / (double)(fan_in + fan_out));
      val = (float)((2.0 * u - 1.0) * lim);
      if (t >= o4) val *= 0.1f;  // small output layer: the start predicts ~0 correction
    }
    params[t] = val;
    m[t] = 0.f;
    v[t] = 0.f;
    w16[t] = __float2bfloat16_rn(val);
  }
}

// Face features [F][4][NFN][M] (float), standardised: (raw - mean) / std.
__global__ void k_mlp_features(const double* V, const double* Vhat, const double* dvh1, const double* dvh2,
                               const int* fs_elem, const int* fs_loc, const int* fnodes, int64_t F, int NFN, int M,
                               int NP, int NF, const float* mean, const float* stdv, float* feat) {
  const int per = NFN * M;
  const int nin = 4 * per;
  const int64_t n = F * per;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t Fi = t / per;
    const int r = (int)(t % per), c = r / M, i = r % M;
    const double vh = Vhat[t];
    float* out = feat + Fi * nin;
    for (int side = 0; side < 2; ++side) {
      const int64_t e = fs_elem[2 * Fi + side];
      const int loc = fs_loc[(2 * Fi + side) * NFN + c];  // f * NFN + local face node
      const int f = loc / NFN, cl = loc % NFN;
      const int a = fnodes[f * NFN + cl];
      const double v = V[(e * NP + a) * M + i];
      const int k = side * per + r;
      out[k] = (float)((v - vh - mean[k]) / stdv[k]);
    }
    out[2 * per + r] = (float)((dvh1[t] - mean[2 * per + r]) / stdv[2 * per + r]);
    out[3 * per + r] = (float)((dvh2[t] - mean[3 * per + r]) / stdv[3 * per + r]);
  }
}

template <int NIN, int NH, int NOUT>
__device__ inline void mlp_forward_one(const __nv_bfloat16* w, const float* x, float* h1, float* h2, float* y) {
  const __nv_bfloat16* W1 = w;
  const __nv_bfloat16* b1 = W1 + NH * NIN;
  const __nv_bfloat16* W2 = b1 + NH;
  const __nv_bfloat16* b2 = W2 + NH * NH;
  const __nv_bfloat16* W3 = b2 + NH;
  const __nv_bfloat16* b3 = W3 + NOUT * NH;
#pragma unroll 4
  for (int j = 0; j < NH; ++j) {
    float s = __bfloat162float(b1[j]);
    for (int k = 0; k < NIN; ++k) s = fmaf(__bfloat162float(W1[j * NIN + k]), x[k], s);
    h1[j] = tanhf(s);
  }
#pragma unroll 4
  for (int j = 0; j < NH; ++j) {
    float s = __bfloat162float(b2[j]);
    for (int k = 0; k < NH; ++k) s = fmaf(__bfloat162float(W2[j * NH + k]), h1[k], s);
    h2[j] = tanhf(s);
  }
  for (int j = 0; j < NOUT; ++j) {
    float s = __bfloat162float(b3[j]);
    for (int k = 0; k < NH; ++k) s = fmaf(__bfloat162float(W3[j * NH + k]), h2[k], s);
    y[j] = s;
  }
}

// Forward for a batch: one thread per sample, BF16 weights staged in shared memory.
template <int NIN, int NH, int NOUT>
__global__ void __launch_bounds__(128) k_mlp_forward(const float* params, const float* x, int64_t B, float* y) {
  constexpr int P = NH * NIN + NH + NH * NH + NH + NOUT * NH + NOUT;
  __shared__ __nv_bfloat16 w[P];
  const __nv_bfloat16* w16 = reinterpret_cast<const __nv_bfloat16*>(params + 3 * (int64_t)P);
  for (int t = threadIdx.x; t < P; t += blockDim.x) w[t] = w16[t];
  __syncthreads();
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  float xin[NIN], h1[NH], h2[NH], out[NOUT];
  for (int k = 0; k < NIN; ++k) xin[k] = x[b * NIN + k];
  mlp_forward_one<NIN, NH, NOUT>(w, xin, h1, h2, out);
  for (int j = 0; j < NOUT; ++j) y[b * NOUT + j] = out[j];
}

// Forward on the tensor cores: each warp takes 16 samples, and a layer out = act W^T + b is a
// 16 x N product over K in steps of 16 (mma.sync m16n8k16, bf16 operands, FP32 accumulation).
// The FP32 activations enter as two bf16 parts, hi = bf16(a) and lo = bf16(a - hi), which carry
// them to about 2^-16 relative; the weights are the BF16 copy, exactly as in the scalar kernel.
HDG_DEVI void mlp_mma(float (&c)[4], const uint4& a, const uint2& b) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
}

// the bf16 pairs (x0, x1) of hi and lo parts (x0 in the low half)
HDG_DEVI void mlp_split2(float x0, float x1, unsigned& hi, unsigned& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const unsigned*>(&h);
  lo = *reinterpret_cast<const unsigned*>(&l);
}

constexpr int kTcLd = MAXH + 4;  // row stride (floats) of a warp's activation tile

// One layer of 16 samples: out[16][N] = f(in[16][K] W^T + b), W [N][K] row-major (bf16, shared).
// Fragment layout of m16n8k16 (g = lane / 4, t = lane % 4): A rows g, g + 8 at columns 2t, 2t + 1
// and 2t + 8, 2t + 9 of the k tile; B (col-major) rows 2t, 2t + 1 and 2t + 8, 2t + 9 of column g;
// C rows g, g + 8 at columns 2t, 2t + 1.
template <int K, int N, bool TANH>
HDG_DEVI void mlp_layer_tc(const __nv_bfloat16* W, const __nv_bfloat16* bias, const float* in, float* out,
                           int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
  for (int nt = 0; nt < N / 8; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16* Wn = W + (nt * 8 + g) * K;
#pragma unroll
    for (int kt = 0; kt < K / 16; ++kt) {
      const int k0 = kt * 16 + 2 * t;
      uint4 hi, lo;
      mlp_split2(in[g * kTcLd + k0], in[g * kTcLd + k0 + 1], hi.x, lo.x);
      mlp_split2(in[(g + 8) * kTcLd + k0], in[(g + 8) * kTcLd + k0 + 1], hi.y, lo.y);
      mlp_split2(in[g * kTcLd + k0 + 8], in[g * kTcLd + k0 + 9], hi.z, lo.z);
      mlp_split2(in[(g + 8) * kTcLd + k0 + 8], in[(g + 8) * kTcLd + k0 + 9], hi.w, lo.w);
      uint2 b;
      b.x = *reinterpret_cast<const unsigned*>(Wn + k0);
      b.y = *reinterpret_cast<const unsigned*>(Wn + k0 + 8);
      mlp_mma(c, hi, b);
      mlp_mma(c, lo, b);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = g + 8 * (q >> 1), col = nt * 8 + 2 * t + (q & 1);
      const float v = c[q] + __bfloat162float(bias[col]);
      out[row * kTcLd + col] = TANH ? tanhf(v) : v;
    }
  }
  __syncwarp();
}

template <int NIN, int NH, int NOUT>
__global__ void __launch_bounds__(64) k_mlp_forward_tc(const float* params, const float* x, int64_t B, float* y) {
  static_assert(NIN % 16 == 0 && NH % 16 == 0 && NOUT % 8 == 0 && NIN <= MAXH && NH <= MAXH, "tile shape");
  constexpr int P = NH * NIN + NH + NH * NH + NH + NOUT * NH + NOUT;
  constexpr int WPB = 2;  // warps per block (static shared memory below 48 KB)
  __shared__ __align__(16) __nv_bfloat16 w[P + 8];
  __shared__ float act[WPB][2][16 * kTcLd];
  const __nv_bfloat16* w16 = reinterpret_cast<const __nv_bfloat16*>(params + 3 * (int64_t)P);
  for (int t = threadIdx.x; t < P; t += blockDim.x) w[t] = w16[t];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b0 = ((int64_t)blockIdx.x * WPB + warp) * 16;
  float* a0 = act[warp][0];
  float* a1 = act[warp][1];
  for (int t = lane; t < 16 * NIN; t += 32) {
    const int r = t / NIN, k = t % NIN;
    a0[r * kTcLd + k] = b0 + r < B ? x[(b0 + r) * NIN + k] : 0.f;
  }
  __syncthreads();
  const __nv_bfloat16* W1 = w;
  const __nv_bfloat16* bb1 = W1 + NH * NIN;
  const __nv_bfloat16* W2 = bb1 + NH;
  const __nv_bfloat16* bb2 = W2 + NH * NH;
  const __nv_bfloat16* W3 = bb2 + NH;
  const __nv_bfloat16* bb3 = W3 + NOUT * NH;
  mlp_layer_tc<NIN, NH, true>(W1, bb1, a0, a1, lane);
  mlp_layer_tc<NH, NH, true>(W2, bb2, a1, a0, lane);
  mlp_layer_tc<NH, NOUT, false>(W3, bb3, a0, a1, lane);
  for (int t = lane; t < 16 * NOUT; t += 32) {
    const int r = t / NOUT, j = t % NOUT;
    if (b0 + r < B) y[(b0 + r) * NOUT + j] = a1[r * kTcLd + j];
  }
}

// Forward + backward of the mean-squared error (mean over the batch and the NOUT
// outputs). A block takes SB samples: one thread per sample runs the forward and
// back-propagates to the pre-activation gradients, kept in shared memory; then all
// threads form the weight gradients as sums over the block's samples and add them to
// grad [P] (FP32) with one atomic per parameter and block. loss [1] accumulates.
template <int NIN, int NH, int NOUT, int SB>
struct GradSmem {
  static constexpr int P = NH * NIN + NH + NH * NH + NH + NOUT * NH + NOUT;
  static constexpr size_t bytes = sizeof(float) * (size_t)SB * (NIN + 4 * NH + NOUT) + sizeof(__nv_bfloat16) * P + 16;
};

template <int NIN, int NH, int NOUT, int SB>
__global__ void __launch_bounds__(128) k_mlp_grad(const float* params, const float* x, const float* target, int64_t B,
                                                int64_t b0_all, int64_t Btot, float* grad, float* loss) {
  constexpr int P = NH * NIN + NH + NH * NH + NH + NOUT * NH + NOUT;
  extern __shared__ float smf[];
  float* xs = smf;                 // [SB][NIN]
  float* h1 = xs + SB * NIN;       // [SB][NH]
  float* h2 = h1 + SB * NH;        // [SB][NH]
  float* dz1 = h2 + SB * NH;       // [SB][NH]
  float* dz2 = dz1 + SB * NH;      // [SB][NH]
  float* dy = dz2 + SB * NH;       // [SB][NOUT]
  __nv_bfloat16* w = reinterpret_cast<__nv_bfloat16*>(dy + SB * NOUT);
  __shared__ float lsum;
  const __nv_bfloat16* w16 = reinterpret_cast<const __nv_bfloat16*>(params + 3 * (int64_t)P);
  for (int t = threadIdx.x; t < P; t += blockDim.x) w[t] = w16[t];
  if (threadIdx.x == 0) lsum = 0.f;
  __syncthreads();
  const __nv_bfloat16* W2 = w + NH * NIN + NH;
  const __nv_bfloat16* W3 = W2 + NH * NH + NH;
  const int64_t base = (int64_t)blockIdx.x * SB;
  const int nb_here = (int)((B - base) < SB ? (B - base) : SB);
  if ((int)threadIdx.x < SB) {
    const int sb = threadIdx.x;
    float* xr = xs + sb * NIN;
    float* a1 = h1 + sb * NH;
    float* a2 = h2 + sb * NH;
    float* d1 = dz1 + sb * NH;
    float* d2 = dz2 + sb * NH;
    float* dyr = dy + sb * NOUT;
    if (sb < nb_here) {
      const int64_t b = b0_all + base + sb;
      for (int k = 0; k < NIN; ++k) xr[k] = x[b * NIN + k];
      float out[NOUT];
      mlp_forward_one<NIN, NH, NOUT>(w, xr, a1, a2, out);
      const float inv = 1.f / ((float)Btot * (float)NOUT);
      float l = 0.f;
      for (int j = 0; j < NOUT; ++j) {
        const float d = out[j] - target[b * NOUT + j];
        l += d * d;
        dyr[j] = 2.f * d * inv;
      }
      atomicAdd(&lsum, l * inv);
      for (int k = 0; k < NH; ++k) {
        float s = 0.f;
        for (int j = 0; j < NOUT; ++j) s = fmaf(__bfloat162float(W3[j * NH + k]), dyr[j], s);
        d2[k] = s * (1.f - a2[k] * a2[k]);
      }
      for (int k = 0; k < NH; ++k) {
        float s = 0.f;
        for (int j = 0; j < NH; ++j) s = fmaf(__bfloat162float(W2[j * NH + k]), d2[j], s);
        d1[k] = s * (1.f - a1[k] * a1[k]);
      }
    } else {  // padding samples contribute nothing
      for (int k = 0; k < NIN; ++k) xr[k] = 0.f;
      for (int k = 0; k < NH; ++k) a1[k] = a2[k] = d1[k] = d2[k] = 0.f;
      for (int j = 0; j < NOUT; ++j) dyr[j] = 0.f;
    }
  }
  __syncthreads();
  // weight gradients: sums over the block's samples
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    const float *L, *Rr;
    int ldl, ldr, j, k;
    bool bias = false;
    int p = t;
    if (p < NH * NIN) {
      j = p / NIN; k = p % NIN; L = dz1; ldl = NH; Rr = xs; ldr = NIN;
    } else if ((p -= NH * NIN) < NH) {
      j = p; k = 0; L = dz1; ldl = NH; Rr = nullptr; ldr = 0; bias = true;
    } else if ((p -= NH) < NH * NH) {
      j = p / NH; k = p % NH; L = dz2; ldl = NH; Rr = h1; ldr = NH;
    } else if ((p -= NH * NH) < NH) {
      j = p; k = 0; L = dz2; ldl = NH; Rr = nullptr; ldr = 0; bias = true;
    } else if ((p -= NH) < NOUT * NH) {
      j = p / NH; k = p % NH; L = dy; ldl = NOUT; Rr = h2; ldr = NH;
    } else {
      p -= NOUT * NH;
      j = p; k = 0; L = dy; ldl = NOUT; Rr = nullptr; ldr = 0; bias = true;
    }
    float s = 0.f;
    for (int sb = 0; sb < SB; ++sb) s = fmaf(L[sb * ldl + j], bias ? 1.f : Rr[sb * ldr + k], s);
    atomicAdd(grad + t, s);
  }
  if (threadIdx.x == 0) atomicAdd(loss, lsum);
}

// Adam on the FP32 master weights, then refresh the BF16 copy.
__global__ void k_mlp_adam(float* params, const float* grad, int64_t P, float lr, float beta1, float beta2, float eps,
                           int step) {
  float* m = params + P;
  float* v = m + P;
  __nv_bfloat16* w16 = reinterpret_cast<__nv_bfloat16*>(v + P);
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x) {
    const float g = grad[t];
    const float mt = beta1 * m[t] + (1.f - beta1) * g;
    const float vt = beta2 * v[t] + (1.f - beta2) * g * g;
    m[t] = mt;
    v[t] = vt;
    const float p = params[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    params[t] = p;
    w16[t] = __float2bfloat16_rn(p);
  }
}

// vhat_out = vhat + dvh1 + pred * tscale (per output component of a face)
__global__ void k_mlp_apply(const double* Vhat, const double* dvh1, const float* pred, const float* tscale,
                            const float* tmean, int64_t F, int per, double* out) {
  const int64_t n = F * per;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % per);
    out[t] = Vhat[t] + dvh1[t] + ((double)pred[t] * (double)tscale[r] + (double)tmean[r]);
  }
}

template <int NIN, int NH, int NOUT>
int launch_grad(const float* params, const float* x, const float* target, int64_t B, float* grad, float* loss,
                cudaStream_t s) {
  constexpr int SB = 64;
  using G = GradSmem<NIN, NH, NOUT, SB>;
  HDG_CK(cudaFuncSetAttribute(k_mlp_grad<NIN, NH, NOUT, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)G::bytes));
  // grid limited to 65535 blocks per launch: split very large batches
  const int64_t per_launch = (int64_t)65535 * SB;
  for (int64_t b0 = 0; b0 < B; b0 += per_launch) {
    const int64_t nbat = (B - b0) < per_launch ? (B - b0) : per_launch;
    k_mlp_grad<NIN, NH, NOUT, SB><<<(unsigned)((nbat + SB - 1) / SB), 128, G::bytes, s>>>(params, x, target, nbat,
                                                                                        b0, B, grad, loss);
  }
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

// Column statistics of x [B][n]: mean and standard deviation (FP64 accumulation; a
// deviation below 1e-30 is reported as 1 so that standardising leaves the column as is).
__global__ void k_mlp_stats(const float* x, int64_t B, int n, float* mean, float* stdv) {
  const int col = blockIdx.x;
  double s = 0.0, s2 = 0.0;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
    const double v = x[b * n + col];
    s += v;
    s2 += v * v;
  }
  __shared__ double ps[256], ps2[256];
  ps[threadIdx.x] = s;
  ps2[threadIdx.x] = s2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      ps[threadIdx.x] += ps[threadIdx.x + w];
      ps2[threadIdx.x] += ps2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = ps[0] / (double)B;
    const double var = ps2[0] / (double)B - m * m;
    const double sd = var > 1e-60 ? ::sqrt(var) : 1.0;
    mean[col] = (float)m;
    stdv[col] = (float)sd;
  }
}

__global__ void k_mlp_standardize(float* x, int64_t B, int n, const float* mean, const float* stdv) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < B * n; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % n);
    x[t] = (x[t] - mean[c]) / stdv[c];
  }
}

// Raw training target: the correction of the extrapolated trace update,
// (vhat^{n+1} - vhat^n) - dvhat^n.
__global__ void k_mlp_target(int64_t n, const double* vh_next, const double* vh, const double* dvh1, float* out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (float)((vh_next[t] - vh[t]) - dvh1[t]);
}

inline unsigned nb(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

}  // namespace

}  // namespace hdg

using namespace hdg;

#define MLP_DISPATCH(NIN, NH, NOUT, ...) \
  if (nin == NIN && nh == NH && nout == NOUT) { __VA_ARGS__; }

extern "C" {

int64_t hdg_mlp_param_count(int nin, int nh, int nout) { return mlp_params(nin, nh, nout); }

int hdg_mlp_init(float* params, int nin, int nh, int nout, uint64_t seed, void* stream) {
  if (!params || nin <= 0 || nh <= 0 || nh > MAXH || nout <= 0) {
    set_error("hdg_mlp_init: invalid argument");
    return HDG_ERR_INVALID_ARG;
  }
  k_mlp_init<<<nb(mlp_params(nin, nh, nout)), 256, 0, (cudaStream_t)stream>>>(params, nin, nh, nout, seed);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int hdg_mlp_features(hdg_ctx_t ctx, const double* V, const double* Vhat, const double* dvh1, const double* dvh2,
                     const float* mean, const float* stdv, float* feat, void* stream) {
  if (!ctx || !V || !Vhat || !dvh1 || !dvh2 || !mean || !stdv || !feat) {
    set_error("hdg_mlp_features: null argument");
    return HDG_ERR_INVALID_ARG;
  }
  if (ctx->pm) {
    set_error("hdg_mlp_features: not built for meshes of mixed degree");
    return HDG_ERR_UNSUPPORTED;
  }
  if (ctx->scheme || !ctx->h_bface.empty()) {
    set_error("hdg_mlp_features: the per-face network works on two-sided face traces (periodic HDG) only");
    return HDG_ERR_UNSUPPORTED;
  }
  k_mlp_features<<<nb(ctx->ntrace), 256, 0, (cudaStream_t)stream>>>(
      V, Vhat, dvh1, dvh2, ctx->d_fs_elem, ctx->d_fs_loc, ctx->T.fnodes, ctx->F, ctx->NFN, ctx->M, ctx->NP, ctx->NF,
      mean, stdv, feat);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int hdg_mlp_forward(const float* params, int nin, int nh, int nout, const float* x, int64_t B, float* y,
                    void* stream) {
  if (!params || !x || !y || B < 0) {
    set_error("hdg_mlp_forward: invalid argument");
    return HDG_ERR_INVALID_ARG;
  }
  if (B == 0) return HDG_OK;
  const unsigned g = (unsigned)((B + 127) / 128);
  cudaStream_t s = (cudaStream_t)stream;
  // 64-64-16 (2D p = 3) on the tensor cores, 32 samples per block; 48-32-12 keeps the scalar kernel
  // (its output width is not a multiple of the tile's 8 columns)
  const unsigned g32 = (unsigned)((B + 31) / 32);
  MLP_DISPATCH(64, 64, 16, (k_mlp_forward_tc<64, 64, 16><<<g32, 64, 0, s>>>(params, x, B, y));
               HDG_CK(cudaGetLastError()); return HDG_OK)
  MLP_DISPATCH(48, 32, 12, (k_mlp_forward<48, 32, 12><<<g, 128, 0, s>>>(params, x, B, y)); HDG_CK(cudaGetLastError());
               return HDG_OK)
  set_error("hdg_mlp_forward: network size not compiled in");
  return HDG_ERR_UNSUPPORTED;
}

int hdg_mlp_train_step(float* params, float* grad, int nin, int nh, int nout, const float* x, const float* target,
                       int64_t B, float lr, int step, float* loss, void* stream) {
  if (!params || !grad || !x || !target || !loss || B <= 0 || step < 1) {
    set_error("hdg_mlp_train_step: invalid argument");
    return HDG_ERR_INVALID_ARG;
  }
  const int64_t P = mlp_params(nin, nh, nout);
  cudaStream_t s = (cudaStream_t)stream;
  HDG_CK(cudaMemsetAsync(grad, 0, sizeof(float) * P, s));
  HDG_CK(cudaMemsetAsync(loss, 0, sizeof(float), s));
  bool done = false;
  int rc = HDG_OK;
  MLP_DISPATCH(64, 64, 16, rc = launch_grad<64, 64, 16>(params, x, target, B, grad, loss, s); done = true)
  MLP_DISPATCH(48, 32, 12, rc = launch_grad<48, 32, 12>(params, x, target, B, grad, loss, s); done = true)
  if (rc) return rc;
  if (!done) {
    set_error("hdg_mlp_train_step: network size not compiled in");
    return HDG_ERR_UNSUPPORTED;
  }
  k_mlp_adam<<<nb(P), 256, 0, s>>>(params, grad, P, lr, 0.9f, 0.999f, 1e-8f, step);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int hdg_mlp_gradient(const float* params, float* grad, int nin, int nh, int nout, const float* x, const float* target,
                     int64_t B, float* loss, void* stream) {
  if (!params || !grad || !x || !target || !loss || B <= 0) {
    set_error("hdg_mlp_gradient: invalid argument");
    return HDG_ERR_INVALID_ARG;
  }
  const int64_t P = mlp_params(nin, nh, nout);
  cudaStream_t s = (cudaStream_t)stream;
  HDG_CK(cudaMemsetAsync(grad, 0, sizeof(float) * P, s));
  HDG_CK(cudaMemsetAsync(loss, 0, sizeof(float), s));
  MLP_DISPATCH(64, 64, 16, return launch_grad<64, 64, 16>(params, x, target, B, grad, loss, s))
  MLP_DISPATCH(48, 32, 12, return launch_grad<48, 32, 12>(params, x, target, B, grad, loss, s))
  set_error("hdg_mlp_gradient: network size not compiled in");
  return HDG_ERR_UNSUPPORTED;
}

int hdg_mlp_stats(const float* x, int64_t B, int n, float* mean, float* stdv, void* stream) {
  if (!x || !mean || !stdv || B <= 0 || n <= 0) {
    set_error("hdg_mlp_stats: invalid argument");
    return HDG_ERR_INVALID_ARG;
  }
  k_mlp_stats<<<n, 256, 0, (cudaStream_t)stream>>>(x, B, n, mean, stdv);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int hdg_mlp_standardize(float* x, int64_t B, int n, const float* mean, const float* stdv, void* stream) {
  if (!x || !mean || !stdv || B < 0 || n <= 0) {
    set_error("hdg_mlp_standardize: invalid argument");
    return HDG_ERR_INVALID_ARG;
  }
  k_mlp_standardize<<<nb(B * n), 256, 0, (cudaStream_t)stream>>>(x, B, n, mean, stdv);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int hdg_mlp_target(int64_t n, const double* vhat_next, const double* vhat, const double* dvhat1, float* out,
                   void* stream) {
  if (!vhat_next || !vhat || !dvhat1 || !out || n < 0) {
    set_error("hdg_mlp_target: invalid argument");
    return HDG_ERR_INVALID_ARG;
  }
  k_mlp_target<<<nb(n), 256, 0, (cudaStream_t)stream>>>(n, vhat_next, vhat, dvhat1, out);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int hdg_mlp_apply_trace(hdg_ctx_t ctx, const double* Vhat, const double* dvh1, const float* pred, const float* tmean,
                        const float* tscale, double* Vhat_out, void* stream) {
  if (!ctx || !Vhat || !dvh1 || !pred || !tmean || !tscale || !Vhat_out) {
    set_error("hdg_mlp_apply_trace: null argument");
    return HDG_ERR_INVALID_ARG;
  }
  if (ctx->pm) {
    set_error("hdg_mlp_apply_trace: not built for meshes of mixed degree");
    return HDG_ERR_UNSUPPORTED;
  }
  if (ctx->scheme || !ctx->h_bface.empty()) {
    set_error("hdg_mlp_apply_trace: the per-face network works on two-sided face traces (periodic HDG) only");
    return HDG_ERR_UNSUPPORTED;
  }
  k_mlp_apply<<<nb(ctx->ntrace), 256, 0, (cudaStream_t)stream>>>(Vhat, dvh1, pred, tscale, tmean, ctx->F,
                                                                 ctx->NFN * ctx->M, Vhat_out);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

}  // extern "C"
