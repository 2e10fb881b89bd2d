// Trace-space operations around the condensed local problems:
//   * BDF history and primitive -> entropy-variable conversion (element data),
//   * the assembled trace operator K = sum_e P_e^T S_e P_e applied element by element
//     and its right-hand side -sum_e P_e^T g_e (Sec. 3.2: only vhat is coupled),
//   * recovery of the interior update dV_e = -y_e - X_e P_e dVhat,
//   * the Newton residual norm,
//   * the trace solve: restarted GMRES(30) with right face-block Jacobi preconditioning,
//     or an assembled dense LU with partial pivoting for small systems.
// All vectors in the trace space are [F][Nf][m] (canonical face-node order).
#include <algorithm>
#include <cstring>
#include <cmath>
#include <vector>

#include "ctx.hpp"
#include "dfloat.cuh"
#include "ptx_async.cuh"

namespace hdg {

namespace {

constexpr int kThreads = 256;

inline unsigned nblocks(int64_t n, int t = kThreads) {
  int64_t b = (n + t - 1) / t;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Block sum; result valid in thread 0.
__device__ double block_sum(double v) {
  __shared__ double part[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) part[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < (int)((blockDim.x + 31) >> 5) ? part[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// ---------------------------------------------------------------- element data
template <int D>
__global__ void k_prim_to_entropy(const double* prim, int64_t n, double gamma, double* v) {
  constexpr int M = D + 2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double* P = prim + t * M;
    double rho = P[0], p = P[M - 1], vv = 0.0;
    for (int i = 0; i < D; ++i) vv += P[1 + i] * P[1 + i];
    double rhoE = p / (gamma - 1.0) + 0.5 * rho * vv;
    double s = ::log(p) - gamma * ::log(rho);
    double* o = v + t * M;
    o[0] = -s + gamma + 1.0 - (gamma - 1.0) * rhoE / p;
    for (int i = 0; i < D; ++i) o[1 + i] = (gamma - 1.0) * rho * P[1 + i] / p;
    o[M - 1] = -(gamma - 1.0) * rho / p;
  }
}

template <int D>
__global__ void k_history(DevTables T, const double* geo, int GEO, int NP, int NG, const double* V0,
                          const double* V1, double c0, double c1, double gamma, double* hist) {
  constexpr int M = D + 2;
  extern __shared__ double sh[];
  double* u = sh;  // [NG][M]
  const int64_t e = blockIdx.x;
  const double detJ = geo[e * GEO + D * D];
  for (int g = threadIdx.x; g < NG; g += blockDim.x) {
    double acc[M];
    for (int i = 0; i < M; ++i) acc[i] = 0.0;
    for (int which = 0; which < 2; ++which) {
      const double* Vs = which == 0 ? V0 : V1;
      const double c = which == 0 ? c0 : c1;
      if (!Vs) continue;
      double v[M];
      for (int i = 0; i < M; ++i) {
        double s = 0.0;
        for (int b = 0; b < NP; ++b) s += T.Phi[g * NP + b] * Vs[(e * NP + b) * M + i];
        v[i] = s;
      }
      double rho, vel[D], p;
      prim_of_v<D>(v, gamma, rho, vel, p);
      double uu[M];
      cons_and_flux<D>(rho, vel, p, gamma, uu, (double(*)[D]) nullptr);
      for (int i = 0; i < M; ++i) acc[i] += c * uu[i];
    }
    for (int i = 0; i < M; ++i) u[g * M + i] = acc[i] * T.W[g] * detJ;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NP * M; t += blockDim.x) {
    int a = t / M, i = t % M;
    double s = 0.0;
    for (int g = 0; g < NG; ++g) s += T.Phi[g * NP + a] * u[g * M + i];
    hist[e * NP * M + t] = s;
  }
}

// ---------------------------------------------------------------- trace operator
// rhs[F][c][i] = -sum_sides g_e[loc * M + i]
__global__ void k_trace_gather(const int* fs_elem, const int* fs_loc, int64_t F, int NFN, int M, int NT,
                               const double* ge, double scale, double* out, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  const int64_t n = F * NFN * M;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t Fi = t / (NFN * M);
    int c = (int)((t / M) % NFN), i = (int)(t % M);
    double s = 0.0;
    for (int side = 0; side < 2; ++side) {
      int64_t e = fs_elem[2 * Fi + side];
      if (e < 0) continue;  // a boundary face has one side
      int loc = fs_loc[(2 * Fi + side) * NFN + c];
      s += ge[e * NT + loc * M + i];
    }
    out[t] = scale * s;
  }
}

// w_e = S_e x_e from the double-float copy of S, in double-float arithmetic on the FP32 pipe
// (exact products by FMA residuals, two-sum accumulation; ~2^-46 relative per product). S streams
// through shared memory by bulk asynchronous copies: a persistent CTA walks its elements
// (e = blockIdx.x, + gridDim.x, ...) in chunks of CR rows (the last one ragged); thread 0 keeps
// kMvStages chunks in flight on an mbarrier ring and refills a slot once every warp has passed it;
// the warps read rows from shared memory (row r: lanes over columns, then a warp sum). No thread
// issues a global load of S, so the copy engine sets the pace. A wait that gives up (about a
// second) sets *err, writes NaN for the element and ends the CTA once its own copies have drained
// (bounded as well).
constexpr int kMvStages = 4;
constexpr int kMvCtasPerSm = 3;
constexpr int kMvChunkBytes = 12800;
constexpr int kMvWaitPolls = 4 * 1000 * 1000;  // ~1 s at 256 ns per poll
__global__ void __launch_bounds__(256) k_elem_matvec_df(const df2* __restrict__ Sdf, const double* x,
                                                        const int* tgidx, int64_t E, int NT, int M, int CR,
                                                        int nchunk, double* w, int* err, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  extern __shared__ __align__(128) df2 smf[];
  __shared__ uint64_t full[kMvStages];
  __shared__ int s_fail;
  const size_t chunk_entries = (size_t)CR * NT;
  df2* xs = smf + kMvStages * chunk_entries;  // [NT]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int64_t my_elems = blockIdx.x < E ? (E - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t Q = my_elems * nchunk;  // chunks of this CTA, in order
  if (Q == 0) return;
  auto chunk_rows = [&](int k) { return k == nchunk - 1 ? NT - (nchunk - 1) * CR : CR; };
  auto issue = [&](int64_t q) {  // thread 0: chunk q into slot q % kMvStages
    const int64_t e = blockIdx.x + (q / nchunk) * gridDim.x;
    const int k = (int)(q % nchunk);
    const uint32_t bytes = (uint32_t)(sizeof(df2) * chunk_rows(k) * NT);
    uint64_t* bar = full + (q % kMvStages);
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(smf + (q % kMvStages) * chunk_entries, Sdf + (e * NT + (int64_t)k * CR) * NT, bytes, bar);
  };
  if (tid == 0) {
    for (int i = 0; i < kMvStages; ++i) mbar_init(full + i, 1);
    fence_mbar_init();
  }
  __syncthreads();
  int64_t issued = 0;
  if (tid == 0)
    for (; issued < Q && issued < kMvStages; ++issued) issue(issued);
  for (int64_t q = 0; q < Q; ++q) {
    const int64_t e = blockIdx.x + (q / nchunk) * gridDim.x;
    const int k = (int)(q % nchunk);
    if (tid == 0) s_fail = 0;
    if (k == 0) {  // the element's x, gathered once (the previous element is done with xs)
      const int nfc = NT / M;
      for (int t = tid; t < NT; t += blockDim.x) xs[t] = df_from(x[(int64_t)tgidx[e * nfc + t / M] * M + t % M]);
    }
    __syncthreads();
    if (!mbar_wait(full + (q % kMvStages), (uint32_t)((q / kMvStages) & 1), kMvWaitPolls)) s_fail = 1;
    __syncthreads();
    if (s_fail) {  // give up: NaN for the element, let the copies in flight land, leave
      for (int t = tid; t < NT; t += blockDim.x) w[e * NT + t] = __longlong_as_double(0x7ff8000000000000LL);
      if (tid == 0) {
        atomicExch(err, 1);
        for (int64_t p = q; p < issued; ++p)
          mbar_wait(full + (p % kMvStages), (uint32_t)((p / kMvStages) & 1), kMvWaitPolls);
      }
      return;
    }
    const int rows = chunk_rows(k);
    const df2* chunk = smf + (q % kMvStages) * chunk_entries;
    for (int r = wid; r < rows; r += nw) {
      dfacc a;
      for (int c = lane; c < NT; c += 32) a.mac(chunk[r * NT + c], xs[c]);
      for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, a.hi, off), ol = __shfl_down_sync(0xffffffffu, a.lo, off);
        a.add(df2{oh, ol});
      }
      if (lane == 0) w[e * NT + (int64_t)k * CR + r] = a.value();
    }
    __syncthreads();  // every warp is done with the slot (and with xs for the last chunk)
    if (tid == 0 && issued < Q) {
      fence_proxy_async();
      issue(issued);
      ++issued;
    }
  }
}

// EDG (continuous trace): out[t][i] = scale * sum over the local occurrences o of node t of
// ge[o * M + i], o = e NF NFN + f NFN + c (CSR ptr / occ)
__global__ void k_node_gather(const int* ptr, const int* occ, int64_t nnode, int M, const double* ge, double scale,
                              double* out, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  const int64_t n = nnode * M;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = t / M;
    const int i = (int)(t % M);
    double s = 0.0;
    for (int o = ptr[node]; o < ptr[node + 1]; ++o) s += ge[(int64_t)occ[o] * M + i];
    out[t] = scale * s;
  }
}

// w_e = S_e x_e in FP64, one warp per row, x_e gathered into shared memory. On GB300 this is
// bound by the FP64 pipe (one FMA per 8-byte entry), not by HBM: the GMRES iterations use the
// double-float copy of S (k_elem_matvec_df) and keep this one for the residuals.
__global__ void k_elem_matvec(const double* S, const double* x, const int* tgidx, int NT, int M, double* w, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  extern __shared__ double xs[];
  const int64_t e = blockIdx.x;
  const int nfc = NT / M;
  for (int t = threadIdx.x; t < NT; t += blockDim.x) {
    int fc = t / M, i = t % M;
    xs[t] = x[(int64_t)tgidx[e * nfc + fc] * M + i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* Se = S + e * (int64_t)NT * NT;
  for (int r = wid; r < NT; r += nw) {
    double s = 0.0;
    for (int c = lane; c < NT; c += 32) s += Se[(int64_t)r * NT + c] * xs[c];
    s = warp_sum(s);
    if (lane == 0) w[e * NT + r] = s;
  }
}

// The double-float copy of S: entry i = hi + lo (hi = S rounded to FP32, lo = the rest rounded),
// 8 bytes an entry as in FP64, about 48 significant bits.
__global__ void k_split_df(const double* S, int64_t n, df2* out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = df_from(S[t]);
}

// dV_e = -y_e - X_e P_e dVhat
__global__ void k_recover(const double* recov, const double* dvh, const int* tgidx, int NV, int NT, int M,
                          double* dV) {
  extern __shared__ double xs[];
  const int64_t e = blockIdx.x;
  const int nfc = NT / M;
  for (int t = threadIdx.x; t < NT; t += blockDim.x) {
    int fc = t / M, i = t % M;
    xs[t] = dvh[(int64_t)tgidx[e * nfc + fc] * M + i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* X = recov + e * (int64_t)(NV * NT + NV);
  const double* y = X + (int64_t)NV * NT;
  for (int r = wid; r < NV; r += nw) {
    double s = 0.0;
    for (int c = lane; c < NT; c += 32) s += X[(int64_t)r * NT + c] * xs[c];
    s = warp_sum(s);
    if (lane == 0) dV[e * NV + r] = -y[r] - s;
  }
}

__global__ void k_sumsq_elem_rows(const double* R, int64_t E, int stride, int n, double* out) {
  double s = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < E * n; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = t / n;
    double v = R[e * stride + (t % n)];
    s += v * v;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

__global__ void k_sumsq_trace_residual(const double* R, const int* fs_elem, const int* fs_loc, int64_t F, int NFN,
                                       int M, int NV, int NT, double* out) {
  double s = 0.0;
  const int64_t n = F * NFN * M;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t Fi = t / (NFN * M);
    int c = (int)((t / M) % NFN), i = (int)(t % M);
    double v = 0.0;
    for (int side = 0; side < 2; ++side) {
      int64_t e = fs_elem[2 * Fi + side];
      if (e < 0) continue;
      int loc = fs_loc[(2 * Fi + side) * NFN + c];
      v += R[e * (int64_t)(NV + NT) + NV + loc * M + i];
    }
    s += v * v;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

// EDG: sum of squares of the assembled trace residual sum_e P_e^T R_t,e
__global__ void k_sumsq_node_residual(const double* R, const int* ptr, const int* occ, int64_t nnode, int M, int NV,
                                      int NT, double* out) {
  const int nfc = NT / M;
  double s = 0.0;
  const int64_t n = nnode * M;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = t / M;
    const int i = (int)(t % M);
    double v = 0.0;
    for (int o = ptr[node]; o < ptr[node + 1]; ++o) {
      const int64_t e = occ[o] / nfc;
      const int fc = occ[o] % nfc;
      v += R[e * (int64_t)(NV + NT) + NV + fc * M + i];
    }
    s += v * v;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

// ---------------------------------------------------------------- vector ops
__global__ void k_axpy(int64_t n, double a, const double* x, double* y) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    y[t] += a * x[t];
}
__global__ void k_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = a * x[t] + b * y[t];
}
__global__ void k_scale_copy(int64_t n, double a, const double* x, double* y) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    y[t] = a * x[t];
}
// out[j] = basis_j . w for j < nb (blockIdx.y = j)
__global__ void k_multidot(int64_t n, const double* basis, int64_t ld, const double* w, double* out, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  const int j = blockIdx.y;
  const double* b = basis + j * ld;
  double s = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    s += b[t] * w[t];
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(out + j, s);
}
// w -= sum_j h[j] basis_j
__global__ void k_multiaxpy(int64_t n, const double* basis, int64_t ld, const double* h, int nb, double* w, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double s = w[t];
    for (int j = 0; j < nb; ++j) s -= h[j] * basis[j * ld + t];
    w[t] = s;
  }
}

// ---------------------------------------------------------------- device-resident Arnoldi
// The state of one GMRES(m) restart cycle in device memory: the Hessenberg matrix in its
// rotated (triangular) form, the Givens rotations, the rotated right-hand side gv, the current
// column h and its second Gram-Schmidt pass h2, |w|^2, and the cycle's progress. The kernels of
// the m Arnoldi steps of a cycle are enqueued (or replayed as one CUDA graph) without a host
// round trip; once a step reaches the tolerance or the iteration limit it sets `done`, and the
// kernels of the remaining steps return at once.
constexpr int kGmM = 30;
struct GmState {
  double H[(kGmM + 1) * kGmM];  // H[i * m + j]
  double cs[kGmM], sn[kGmM], gv[kGmM + 1];
  double h[kGmM + 2], h2[kGmM + 2], y[kGmM];
  double wn2, hnext, bnorm, rtol, rel;
  int done, jdone, total, max_it;
};

__global__ void k_gm_zero(double* a, int n, const int* skip) {
  if (*skip) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = 0.0;
}

// step j: h += h2 (the two Gram-Schmidt passes), h[j+1] = |w|, the previous rotations on h, the
// new rotation, the rotated right-hand side, column j of H, the residual estimate and the stop test
__global__ void k_gm_givens(GmState* st, int j, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || st->done) return;
  double* h = st->h;
  for (int i = 0; i <= j; ++i) h[i] += st->h2[i];
  const double hn = ::sqrt(st->wn2);
  h[j + 1] = hn;
  st->hnext = hn;
  for (int i = 0; i < j; ++i) {
    const double t = st->cs[i] * h[i] + st->sn[i] * h[i + 1];
    h[i + 1] = -st->sn[i] * h[i] + st->cs[i] * h[i + 1];
    h[i] = t;
  }
  const double den = ::hypot(h[j], h[j + 1]);
  st->cs[j] = den > 0.0 ? h[j] / den : 1.0;
  st->sn[j] = den > 0.0 ? h[j + 1] / den : 0.0;
  h[j] = den;
  h[j + 1] = 0.0;
  st->gv[j + 1] = -st->sn[j] * st->gv[j];
  st->gv[j] = st->cs[j] * st->gv[j];
  for (int i = 0; i <= j; ++i) st->H[i * m + j] = h[i];
  st->rel = ::fabs(st->gv[j + 1]) / st->bnorm;
  st->total += 1;
  st->jdone = j + 1;
  if (st->rel <= st->rtol || st->total >= st->max_it || j + 1 == m) st->done = 1;
}

// the next basis vector w / h[j+1] (not needed once the cycle is done)
__global__ void k_gm_scale(const GmState* st, int64_t n, const double* w, double* vnext) {
  if (st->done || !(st->hnext > 0.0)) return;
  const double inv = 1.0 / st->hnext;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    vnext[t] = inv * w[t];
}

// y = H^{-1} gv on the jdone completed steps (back substitution)
__global__ void k_gm_solve(GmState* st, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int jd = st->jdone;
  for (int i = jd - 1; i >= 0; --i) {
    double t = st->gv[i];
    for (int k = i + 1; k < jd; ++k) t -= st->H[i * m + k] * st->y[k];
    st->y[i] = t / st->H[i * m + i];
  }
}

// x += sum_{j < *nb} c[j] basis_j (the count read on the device)
__global__ void k_multiaxpy_add_dev(int64_t n, const double* basis, int64_t ld, const double* c, const int* nb,
                                    double* x) {
  const int k = *nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double s = x[t];
    for (int j = 0; j < k; ++j) s += c[j] * basis[j * ld + t];
    x[t] = s;
  }
}

// ---------------------------------------------------------------- face-block Jacobi
// K_FF (canonical order) = sum_sides S_e[loc rows, loc cols]; LU with partial pivoting, then
// the inverse column by column (thread t: K_FF x = e_t), stored transposed, fac[F][j][i] =
// K_FF^{-1}[i][j], so that applying it reads whole rows of fac (B <= kMaxFaceBlock).
constexpr int kMaxFaceBlock = 64;
__global__ void k_face_block_factor(const double* S, const int* fs_elem, const int* fs_loc, int NFN, int M, int NT,
                                    double* fac) {
  extern __shared__ double A[];  // [B][B], then X [B][B] (column t of the inverse in X[.][t])
  __shared__ int s_p;
  __shared__ int s_piv[kMaxFaceBlock];
  const int B = NFN * M;
  const int64_t Fi = blockIdx.x;
  for (int t = threadIdx.x; t < B * B; t += blockDim.x) {
    int r = t / B, c = t % B;
    int cr = r / M, ir = r % M, cc = c / M, ic = c % M;
    double s = 0.0;
    for (int side = 0; side < 2; ++side) {
      int64_t e = fs_elem[2 * Fi + side];
      if (e < 0) continue;
      int lr = fs_loc[(2 * Fi + side) * NFN + cr] * M + ir;
      int lc = fs_loc[(2 * Fi + side) * NFN + cc] * M + ic;
      s += S[e * (int64_t)NT * NT + (int64_t)lr * NT + lc];
    }
    A[t] = s;
  }
  __syncthreads();
  for (int k = 0; k < B; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int r = k + threadIdx.x; r < B; r += 32) {
        double v = fabs(A[r * B + k]);
        if (v > best) {
          best = v;
          bi = r;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        double ob = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) {
        s_p = bi;
        s_piv[k] = bi;
      }
    }
    __syncthreads();
    int p = s_p;
    if (p != k)
      for (int j = threadIdx.x; j < B; j += blockDim.x) {
        double t = A[k * B + j];
        A[k * B + j] = A[p * B + j];
        A[p * B + j] = t;
      }
    __syncthreads();
    double d = A[k * B + k];
    double inv = d != 0.0 ? 1.0 / d : 0.0;
    for (int r = k + 1 + threadIdx.x; r < B; r += blockDim.x) A[r * B + k] *= inv;
    __syncthreads();
    int rem = B - k - 1;
    for (int t = threadIdx.x; t < rem * rem; t += blockDim.x) {
      int r = k + 1 + t / rem, c = k + 1 + t % rem;
      A[r * B + c] -= A[r * B + k] * A[k * B + c];
    }
    __syncthreads();
  }
  double* X = A + B * B;
  for (int t = threadIdx.x; t < B; t += blockDim.x) {  // column t of the inverse
    for (int i = 0; i < B; ++i) X[i * B + t] = i == t ? 1.0 : 0.0;
    for (int k = 0; k < B; ++k) {  // the row swaps of the factorisation, in order
      const int p = s_piv[k];
      if (p != k) {
        const double tmp = X[k * B + t];
        X[k * B + t] = X[p * B + t];
        X[p * B + t] = tmp;
      }
    }
    for (int k = 0; k < B; ++k) {  // unit lower triangle
      const double xk = X[k * B + t];
      for (int r = k + 1; r < B; ++r) X[r * B + t] -= A[r * B + k] * xk;
    }
    for (int k = B - 1; k >= 0; --k) {  // upper triangle
      const double d = A[k * B + k];
      const double xk = d != 0.0 ? X[k * B + t] / d : 0.0;
      X[k * B + t] = xk;
      for (int r = 0; r < k; ++r) X[r * B + t] -= A[r * B + k] * xk;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < B * B; t += blockDim.x) {
    const int j = t / B, i = t % B;
    fac[Fi * (int64_t)B * B + t] = X[i * B + j];
  }
}

// z_F = K_FF^{-1} r_F from the stored inverse (fac[F][j][i] = K_FF^{-1}[i][j]), one warp per face:
// lane i accumulates row i over j, every load a coalesced run of one stored row
__global__ void k_face_block_apply(const double* fac, int64_t F, int B, const double* r, double* z, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  extern __shared__ double xs[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t Fi = (int64_t)blockIdx.x * nw + wid;
  if (Fi >= F) return;
  double* rs = xs + wid * B;
  for (int t = lane; t < B; t += 32) rs[t] = r[Fi * B + t];
  __syncwarp();
  const double* A = fac + Fi * (int64_t)B * B;
  const bool h0 = lane < B, h1 = lane + 32 < B;
  double a0 = 0.0, a1 = 0.0;
#pragma unroll 5
  for (int j = 0; j < B; ++j) {
    const double rj = rs[j];
    if (h0) a0 += A[j * B + lane] * rj;
    if (h1) a1 += A[j * B + 32 + lane] * rj;
  }
  if (h0) z[Fi * B + lane] = a0;
  if (h1) z[Fi * B + 32 + lane] = a1;
}

// ---------------------------------------------------------------- EDG node-block Jacobi
// K_tt (M x M) = sum over pairs of local occurrences (e, fc), (e, fc') of node t in the same
// element of S_e[fc M + i][fc' M + j]; inverted by Gauss-Jordan with partial pivoting. One thread
// per node (M <= 5).
__global__ void k_node_block_factor(const double* S, const int* ptr, const int* occ, int64_t nnode, int M, int NT,
                                    double* binv) {
  const int nfc = NT / M;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnode; t += (int64_t)gridDim.x * blockDim.x) {
    double A[5][10];
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < 2 * M; ++j) A[i][j] = (j == M + i) ? 1.0 : 0.0;
    for (int o1 = ptr[t]; o1 < ptr[t + 1]; ++o1) {
      const int64_t e = occ[o1] / nfc;
      const int f1 = occ[o1] % nfc;
      const double* Se = S + e * (int64_t)NT * NT;
      for (int o2 = ptr[t]; o2 < ptr[t + 1]; ++o2) {
        if (occ[o2] / nfc != e) continue;
        const int f2 = occ[o2] % nfc;
        for (int i = 0; i < M; ++i)
          for (int j = 0; j < M; ++j) A[i][j] += Se[(int64_t)(f1 * M + i) * NT + f2 * M + j];
      }
    }
    for (int k = 0; k < M; ++k) {
      int p = k;
      for (int r = k + 1; r < M; ++r)
        if (fabs(A[r][k]) > fabs(A[p][k])) p = r;
      if (p != k)
        for (int j = 0; j < 2 * M; ++j) {
          const double tmp = A[k][j];
          A[k][j] = A[p][j];
          A[p][j] = tmp;
        }
      const double d = A[k][k];
      const double inv = d != 0.0 ? 1.0 / d : 0.0;
      for (int j = 0; j < 2 * M; ++j) A[k][j] *= inv;
      for (int r = 0; r < M; ++r) {
        if (r == k) continue;
        const double f = A[r][k];
        for (int j = 0; j < 2 * M; ++j) A[r][j] -= f * A[k][j];
      }
    }
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) binv[(t * M + i) * M + j] = A[i][M + j];
  }
}

// z_t = K_tt^{-1} r_t for every node (z and r distinct)
__global__ void k_node_block_apply(const double* binv, int64_t nnode, int M, const double* r, double* z, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  const int64_t n = nnode * M;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = t / M;
    const int i = (int)(t % M);
    double s = 0.0;
    for (int j = 0; j < M; ++j) s += binv[(node * M + i) * M + j] * r[node * M + j];
    z[t] = s;
  }
}

// ---------------------------------------------------------------- dense direct solver
__global__ void k_dense_scatter(const double* S, const int* tgidx, int64_t E, int NT, int M, int64_t n, double* K) {
  const int nfc = NT / M;
  const int64_t tot = E * (int64_t)NT * NT;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = t / ((int64_t)NT * NT);
    int r = (int)((t / NT) % NT), c = (int)(t % NT);
    int64_t gr = (int64_t)tgidx[e * nfc + r / M] * M + r % M;
    int64_t gc = (int64_t)tgidx[e * nfc + c / M] * M + c % M;
    atomicAdd(K + gr * n + gc, S[t]);
  }
}
__global__ void k_dense_pivot(double* K, int64_t n, int64_t k, int* piv, int* bad) {
  __shared__ double bv[1024];
  __shared__ int64_t bi[1024];
  double best = -1.0;
  int64_t idx = k;
  for (int64_t r = k + threadIdx.x; r < n; r += blockDim.x) {
    double v = fabs(K[r * n + k]);
    if (v > best) {
      best = v;
      idx = r;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = idx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      double ov = bv[threadIdx.x + s];
      int64_t oi = bi[threadIdx.x + s];
      if (ov > bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = ov;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int64_t p = bi[0];
  if (threadIdx.x == 0) {
    piv[k] = (int)p;
    if (!(bv[0] > 0.0)) *bad = 1;
  }
  if (p != k)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      double t = K[k * n + j];
      K[k * n + j] = K[p * n + j];
      K[p * n + j] = t;
    }
}
__global__ void k_dense_scale(double* K, int64_t n, int64_t k) {
  const double d = K[k * n + k];
  const double inv = d != 0.0 ? 1.0 / d : 0.0;
  for (int64_t r = k + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    K[r * n + k] *= inv;
}
__global__ void k_dense_update(double* K, int64_t n, int64_t k) {
  const int64_t rem = n - k - 1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rem * rem; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = k + 1 + t / rem, c = k + 1 + t % rem;
    K[r * n + c] -= K[r * n + k] * K[k * n + c];
  }
}
// forward / backward substitution in one block
__global__ void k_dense_solve(const double* K, const int* piv, int64_t n, double* x) {
  if (threadIdx.x == 0)
    for (int64_t k = 0; k < n; ++k) {
      int64_t p = piv[k];
      if (p != k) {
        double t = x[k];
        x[k] = x[p];
        x[p] = t;
      }
    }
  __syncthreads();
  for (int64_t k = 0; k < n; ++k) {
    double xk = x[k];
    for (int64_t r = k + 1 + threadIdx.x; r < n; r += blockDim.x) x[r] -= K[r * n + k] * xk;
    __syncthreads();
  }
  for (int64_t k = n - 1; k >= 0; --k) {
    if (threadIdx.x == 0) x[k] /= K[k * n + k];
    __syncthreads();
    double xk = x[k];
    for (int64_t r = threadIdx.x; r < k; r += blockDim.x) x[r] -= K[r * n + k] * xk;
    __syncthreads();
  }
}

}  // namespace

// ================================================================ host launchers
// Source term s of d u/dt + div(F + G) = s given at the element nodes: its nodal interpolant
// s_h enters R_v as -(s_h, w)_K, which the residual takes with the history, so the kernel adds
// c (s_h, phi_a)_K = c sum_g W_g |J_e| phi_a(x_g) sum_b phi_b(x_g) s[e][b] to hist[e][a].
// One CTA per element; the values of s_h at the volume points are staged in shared memory.
__global__ void k_source_weak(DevTables T, const double* geo, int GEO, int detj_at, int NP, int NG, int M,
                              const double* src, double c, double* hist) {
  extern __shared__ double sh[];  // [NG][M]
  const int64_t e = blockIdx.x;
  const double w = c * geo[e * GEO + detj_at];
  for (int t = threadIdx.x; t < NG * M; t += blockDim.x) {
    const int g = t / M, i = t % M;
    double s = 0.0;
    for (int b = 0; b < NP; ++b) s += T.Phi[g * NP + b] * src[(e * NP + b) * M + i];
    sh[t] = s * T.W[g] * w;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NP * M; t += blockDim.x) {
    const int a = t / M, i = t % M;
    double s = 0.0;
    for (int g = 0; g < NG; ++g) s += T.Phi[g * NP + a] * sh[g * M + i];
    hist[e * NP * M + t] += s;
  }
}

int launch_prim_to_entropy(hdg_ctx* ctx, const double* prim, int64_t n, double* v, cudaStream_t s) {
  if (n <= 0) return HDG_OK;
  if (ctx->dim == 2)
    k_prim_to_entropy<2><<<nblocks(n), kThreads, 0, s>>>(prim, n, ctx->ph.gamma, v);
  else
    k_prim_to_entropy<3><<<nblocks(n), kThreads, 0, s>>>(prim, n, ctx->ph.gamma, v);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int launch_history(hdg_ctx* ctx, const double* V0, const double* V1, double c0, double c1, double* hist,
                   cudaStream_t s) {
  if (ctx->pm) return pm_history(ctx, V0, V1, c0, c1, hist, s);
  size_t sm = sizeof(double) * ctx->NG * ctx->M;
  if (ctx->dim == 2)
    k_history<2><<<(unsigned)ctx->E, 128, sm, s>>>(ctx->T, ctx->d_geo, ctx->GEO, ctx->NP, ctx->NG, V0, V1, c0, c1,
                                                   ctx->ph.gamma, hist);
  else
    k_history<3><<<(unsigned)ctx->E, 128, sm, s>>>(ctx->T, ctx->d_geo, ctx->GEO, ctx->NP, ctx->NG, V0, V1, c0, c1,
                                                   ctx->ph.gamma, hist);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int launch_source_weak(hdg_ctx* ctx, const double* src, double c, double* hist, cudaStream_t s) {
  if (ctx->pm) return HDG_ERR_UNSUPPORTED;
  if (ctx->E <= 0) return HDG_OK;
  const size_t sm = sizeof(double) * ctx->NG * ctx->M;
  k_source_weak<<<(unsigned)ctx->E, 128, sm, s>>>(ctx->T, ctx->d_geo, ctx->GEO, ctx->dim * ctx->dim, ctx->NP, ctx->NG,
                                                  ctx->M, src, c, hist);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int launch_trace_rhs(hdg_ctx* ctx, const double* g, double* rhs, cudaStream_t s) {
  if (ctx->pm) return pm_gather(ctx, g, -1.0, rhs, s);
  if (ctx->scheme)
    k_node_gather<<<nblocks(ctx->ntrace), kThreads, 0, s>>>(ctx->d_tr_ptr, ctx->d_tr_occ, ctx->n_tnodes, ctx->M, g,
                                                           -1.0, rhs, nullptr);
  else
    k_trace_gather<<<nblocks(ctx->ntrace), kThreads, 0, s>>>(ctx->d_fs_elem, ctx->d_fs_loc, ctx->F, ctx->NFN, ctx->M,
                                                            ctx->NT, g, -1.0, rhs, nullptr);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

static int launch_gather(hdg_ctx* ctx, const double* work, double* y, cudaStream_t s, const int* skip = nullptr) {
  if (ctx->pm) return pm_gather(ctx, work, 1.0, y, s, skip);
  if (ctx->scheme)
    k_node_gather<<<nblocks(ctx->ntrace), kThreads, 0, s>>>(ctx->d_tr_ptr, ctx->d_tr_occ, ctx->n_tnodes, ctx->M, work,
                                                           1.0, y, skip);
  else
    k_trace_gather<<<nblocks(ctx->ntrace), kThreads, 0, s>>>(ctx->d_fs_elem, ctx->d_fs_loc, ctx->F, ctx->NFN, ctx->M,
                                                            ctx->NT, work, 1.0, y, skip);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int launch_trace_matvec(hdg_ctx* ctx, const double* S, const double* x, double* y, double* work, cudaStream_t s,
                        const int* skip) {
  if (ctx->pm) {
    if (int rc = pm_elem_matvec(ctx, S, x, work, s, skip)) return rc;
    return pm_gather(ctx, work, 1.0, y, s, skip);
  }
  k_elem_matvec<<<(unsigned)ctx->E, 256, sizeof(double) * ctx->NT, s>>>(S, x, ctx->d_tgidx, ctx->NT, ctx->M, work,
                                                                        skip);
  return launch_gather(ctx, work, y, s, skip);
}

// y = K x from the double-float copy of S (see k_elem_matvec_df)
// shared memory of k_elem_matvec_df; its attribute, the SM count and the error flag are set up
// on first use (before any stream capture: none of these steps may be captured)
static size_t matvec_df_smem(const hdg_ctx* ctx, int* CR, int* nchunk) {
  const int NT = ctx->NT;
  *CR = std::max(1, std::min(NT, kMvChunkBytes / (int)(sizeof(df2) * NT)));
  *nchunk = (NT + *CR - 1) / *CR;
  return sizeof(df2) * ((size_t)kMvStages * *CR * NT + NT);
}

static int prepare_matvec_df(hdg_ctx* ctx) {
  int CR, nchunk;
  const size_t smem = matvec_df_smem(ctx, &CR, &nchunk);
  if (!ctx->attr_matvec) {  // per context, hence per device
    HDG_CK(cudaFuncSetAttribute(k_elem_matvec_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (!ctx->num_sms) HDG_CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    if (!ctx->d_mv_err) {
      HDG_CK(cudaMalloc(&ctx->d_mv_err, sizeof(int)));
      HDG_CK(cudaMemset(ctx->d_mv_err, 0, sizeof(int)));
    }
    ctx->attr_matvec = true;
  }
  return HDG_OK;
}

static int launch_trace_matvec_df(hdg_ctx* ctx, const df2* Sdf, const double* x, double* y, double* work,
                                  cudaStream_t s, const int* skip = nullptr) {
  if (int rc = prepare_matvec_df(ctx)) return rc;
  const int NT = ctx->NT;
  int CR, nchunk;
  const size_t smem = matvec_df_smem(ctx, &CR, &nchunk);
  const int64_t grid = std::min<int64_t>(ctx->E, (int64_t)kMvCtasPerSm * ctx->num_sms);
  k_elem_matvec_df<<<(unsigned)grid, 256, smem, s>>>(Sdf, x, ctx->d_tgidx, ctx->E, NT, ctx->M, CR, nchunk, work,
                                                      ctx->d_mv_err, skip);
  return launch_gather(ctx, work, y, s, skip);
}

int launch_recover(hdg_ctx* ctx, const double* recov, const double* dVhat, double* dV, cudaStream_t s) {
  if (ctx->pm) return pm_recover(ctx, recov, dVhat, dV, s);
  k_recover<<<(unsigned)ctx->E, 256, sizeof(double) * ctx->NT, s>>>(recov, dVhat, ctx->d_tgidx, ctx->NV, ctx->NT,
                                                                   ctx->M, dV);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
  if (n <= 0) return HDG_OK;
  k_axpby<<<nblocks(n), kThreads, 0, s>>>(n, a, x, b, y, out);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  k_axpy<<<nblocks(n), kThreads, 0, s>>>(n, a, x, y);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

static int ensure_red(hdg_ctx* ctx) {
  if (!ctx->d_red) {
    HDG_CK(cudaMalloc(&ctx->d_red, sizeof(double) * 128));
    HDG_CK(cudaMallocHost(&ctx->h_red, sizeof(double) * 128));
  }
  return HDG_OK;
}

int residual_norm(hdg_ctx* ctx, const double* R, double* norm, cudaStream_t s) {
  int rc = ensure_red(ctx);
  if (rc) return rc;
  HDG_CK(cudaMemsetAsync(ctx->d_red, 0, sizeof(double) * 2, s));
  if (ctx->pm) {
    if ((rc = pm_sumsq(ctx, R, ctx->d_red, s))) return rc;
  } else {
  k_sumsq_elem_rows<<<nblocks(ctx->E * (int64_t)ctx->NV), kThreads, 0, s>>>(R, ctx->E, ctx->NV + ctx->NT, ctx->NV,
                                                                           ctx->d_red);
  if (ctx->scheme)
    k_sumsq_node_residual<<<nblocks(ctx->ntrace), kThreads, 0, s>>>(R, ctx->d_tr_ptr, ctx->d_tr_occ, ctx->n_tnodes,
                                                                   ctx->M, ctx->NV, ctx->NT, ctx->d_red + 1);
  else
    k_sumsq_trace_residual<<<nblocks(ctx->ntrace), kThreads, 0, s>>>(R, ctx->d_fs_elem, ctx->d_fs_loc, ctx->F,
                                                                    ctx->NFN, ctx->M, ctx->NV, ctx->NT, ctx->d_red + 1);
  }
  HDG_CK(cudaGetLastError());
  HDG_CK(cudaMemcpyAsync(ctx->h_red, ctx->d_red, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  HDG_CK(cudaStreamSynchronize(s));
  *norm = std::sqrt(ctx->h_red[0] + ctx->h_red[1]);
  return HDG_OK;
}

// ---------------------------------------------------------------- dense solve
static int dense_solve(hdg_ctx* ctx, const double* S, const double* g, double* dVhat, double* final_res,
                       cudaStream_t s) {
  const int64_t n = ctx->ntrace;
  if ((size_t)n != ctx->dense_n) {
    if (ctx->d_dense) cudaFree(ctx->d_dense);
    if (ctx->d_dpiv) cudaFree(ctx->d_dpiv);
    ctx->d_dense = nullptr;
    ctx->d_dpiv = nullptr;
    ctx->dense_n = 0;
    HDG_CK(cudaMalloc(&ctx->d_dense, sizeof(double) * n * n));
    HDG_CK(cudaMalloc(&ctx->d_dpiv, sizeof(int) * (n + 1)));
    ctx->dense_n = (size_t)n;
    if (ctx->lu_graph_exec) {  // the recorded graph refers to the old buffers
      cudaGraphExecDestroy(ctx->lu_graph_exec);
      ctx->lu_graph_exec = nullptr;
    }
  }
  int rc = ensure_red(ctx);
  if (rc) return rc;
  double* K = ctx->d_dense;
  int* bad = ctx->d_dpiv + n;
  HDG_CK(cudaMemsetAsync(K, 0, sizeof(double) * n * n, s));
  HDG_CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
  if (ctx->pm) {
    if ((rc = pm_dense_scatter(ctx, S, n, K, s))) return rc;
  } else {
    k_dense_scatter<<<nblocks(ctx->E * (int64_t)ctx->NT * ctx->NT), kThreads, 0, s>>>(S, ctx->d_tgidx, ctx->E,
                                                                                     ctx->NT, ctx->M, n, K);
  }
  // LU with partial pivoting: 3 launches per pivot, recorded once per context into a CUDA
  // graph (on a context-owned stream, so the caller's stream may be the legacy default
  // stream) and replayed on the caller's stream.
  if (!ctx->lu_graph_exec) {
    cudaStream_t cap = nullptr;
    HDG_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    HDG_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    for (int64_t k = 0; k < n; ++k) {
      k_dense_pivot<<<1, 1024, 0, cap>>>(K, n, k, ctx->d_dpiv, bad);
      if (k + 1 < n) {
        k_dense_scale<<<nblocks(n - k - 1), kThreads, 0, cap>>>(K, n, k);
        k_dense_update<<<nblocks((n - k - 1) * (n - k - 1)), kThreads, 0, cap>>>(K, n, k);
      }
    }
    cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture (dense LU)");
    ce = cudaGraphInstantiate(&ctx->lu_graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      ctx->lu_graph_exec = nullptr;
      return cuda_fail(ce, "cudaGraphInstantiate (dense LU)");
    }
  }
  {
    LaunchScope ls(ctx, HDG_KERNEL_TRACE, s);
    HDG_CK(cudaGraphLaunch(ctx->lu_graph_exec, s));
  }
  rc = launch_trace_rhs(ctx, g, dVhat, s);
  if (rc) return rc;
  k_dense_solve<<<1, 1024, 0, s>>>(K, ctx->d_dpiv, n, dVhat);
  HDG_CK(cudaGetLastError());
  int hbad = 0;
  HDG_CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  HDG_CK(cudaStreamSynchronize(s));
  if (hbad) {
    set_error("trace_solve: singular assembled trace matrix");
    return HDG_ERR_SINGULAR;
  }
  *final_res = 0.0;
  return HDG_OK;
}

// ---------------------------------------------------------------- GMRES
static int gmres_solve(hdg_ctx* ctx, const double* S, const double* g, double* x, double rtol, int max_it,
                       int* iters, double* final_res, cudaStream_t s) {
  const int m = kGmM;
  const int64_t n = ctx->ntrace;
  const int B = ctx->NFN * ctx->M;
  // workspace: basis V (m+1) n, Z (precond of current basis vector) n, w n, b n, elem work E*NT
  const size_t elem_work = ctx->pm ? (size_t)ctx->mesh->m.toff.back() : (size_t)ctx->E * ctx->NT;
  const size_t need = sizeof(double) * ((size_t)(m + 1) * n + 3 * (size_t)n + elem_work);
  if (ctx->sw_bytes < need) {
    if (ctx->d_sw) cudaFree(ctx->d_sw);
    ctx->d_sw = nullptr;
    ctx->sw_bytes = 0;
    HDG_CK(cudaMalloc(&ctx->d_sw, need));
    ctx->sw_bytes = need;
  }
  if (ctx->pm) {
    if (!ctx->d_pc) HDG_CK(cudaMalloc(&ctx->d_pc, sizeof(double) * ctx->pm->pc_len));
  } else if (ctx->scheme) {
    if (!ctx->d_pcn) HDG_CK(cudaMalloc(&ctx->d_pcn, sizeof(double) * ctx->n_tnodes * ctx->M * ctx->M));
  } else {
    if (B > kMaxFaceBlock || 2 * sizeof(double) * B * B > 48 * 1024) {  // factor + inverse in shared memory
      set_error("trace_solve: face block larger than the preconditioner supports");
      return HDG_ERR_UNSUPPORTED;
    }
    if (!ctx->d_pc) HDG_CK(cudaMalloc(&ctx->d_pc, sizeof(double) * ctx->F * B * B));
  }
  int rc = ensure_red(ctx);
  if (rc) return rc;
  double* Vb = ctx->d_sw;
  double* zt = Vb + (size_t)(m + 1) * n;
  double* w = zt + n;
  double* b = w + n;
  double* ew = b + n;
  if (ctx->pm) {  // mixed degrees: face blocks of each face's own size
    if ((rc = pm_face_factor(ctx, S, ctx->d_pc, s))) return rc;
  } else if (ctx->scheme)  // EDG: node-block Jacobi
    k_node_block_factor<<<nblocks(ctx->n_tnodes), kThreads, 0, s>>>(S, ctx->d_tr_ptr, ctx->d_tr_occ, ctx->n_tnodes,
                                                                    ctx->M, ctx->NT, ctx->d_pcn);
  else  // HDG: face-block Jacobi
    k_face_block_factor<<<(unsigned)ctx->F, 64, 2 * sizeof(double) * B * B, s>>>(S, ctx->d_fs_elem, ctx->d_fs_loc,
                                                                               ctx->NFN, ctx->M, ctx->NT, ctx->d_pc);
  // the double-float copy of S for the Arnoldi products (the restart and final residuals use S
  // itself); without room for it every product is the FP64 one
  const size_t sdf_bytes = sizeof(df2) * (size_t)ctx->E * ctx->NT * ctx->NT;
  if (!ctx->pm && ctx->sdf_bytes < sdf_bytes && !ctx->sdf_unavailable) {
    if (ctx->d_Sdf) cudaFree(ctx->d_Sdf);
    ctx->d_Sdf = nullptr;
    ctx->sdf_bytes = 0;
    if (cudaMalloc(&ctx->d_Sdf, sdf_bytes) == cudaSuccess) {
      ctx->sdf_bytes = sdf_bytes;
    } else {
      cudaGetLastError();  // out of memory is not an error here
      ctx->d_Sdf = nullptr;
      ctx->sdf_unavailable = true;
    }
  }
  const df2* Sdf = nullptr;
  if (ctx->d_Sdf && !ctx->pm) {
    const int64_t ns = (int64_t)ctx->E * ctx->NT * ctx->NT;
    k_split_df<<<nblocks(ns), kThreads, 0, s>>>(S, ns, static_cast<df2*>(ctx->d_Sdf));
    Sdf = static_cast<const df2*>(ctx->d_Sdf);
  }
  auto arnoldi_matvec = [&](const double* xin, double* yout, cudaStream_t st, const int* skip) {
    return Sdf ? launch_trace_matvec_df(ctx, Sdf, xin, yout, ew, st, skip)
               : launch_trace_matvec(ctx, S, xin, yout, ew, st, skip);
  };
  rc = launch_trace_rhs(ctx, g, b, s);
  if (rc) return rc;
  const int wpb = 8;
  auto precond = [&](const double* r, double* z, cudaStream_t st, const int* skip) {
    if (ctx->pm)
      pm_face_apply(ctx, ctx->d_pc, r, z, st, skip);
    else if (ctx->scheme)
      k_node_block_apply<<<nblocks(n), kThreads, 0, st>>>(ctx->d_pcn, ctx->n_tnodes, ctx->M, r, z, skip);
    else
      k_face_block_apply<<<(unsigned)((ctx->F + wpb - 1) / wpb), 32 * wpb, sizeof(double) * wpb * B, st>>>(
          ctx->d_pc, ctx->F, B, r, z, skip);
  };
  auto dot_host = [&](const double* basis, int nb, const double* v, double* out) -> int {
    HDG_CK(cudaMemsetAsync(ctx->d_red, 0, sizeof(double) * nb, s));
    dim3 grid(std::min<unsigned>(nblocks(n), 1024), nb);
    k_multidot<<<grid, kThreads, 0, s>>>(n, basis, n, v, ctx->d_red, nullptr);
    HDG_CK(cudaGetLastError());
    HDG_CK(cudaMemcpyAsync(ctx->h_red, ctx->d_red, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    HDG_CK(cudaStreamSynchronize(s));
    for (int i = 0; i < nb; ++i) out[i] = ctx->h_red[i];
    return HDG_OK;
  };
  // the device state of a cycle and the kernels of one cycle: step j preconditions basis
  // vector j, applies the operator, orthogonalises twice against the basis (classical
  // Gram-Schmidt), takes |w|, updates the rotations and the residual estimate, and writes basis
  // vector j + 1; every step's kernels return at once once `done` is set
  if (!ctx->d_gm) {
    HDG_CK(cudaMalloc(&ctx->d_gm, sizeof(GmState)));
    HDG_CK(cudaMallocHost(&ctx->h_gm, sizeof(GmState)));
    std::memset(ctx->h_gm, 0, sizeof(GmState));
  }
  GmState* gm = static_cast<GmState*>(ctx->d_gm);
  const int* done = &gm->done;
  if (Sdf && (rc = prepare_matvec_df(ctx))) return rc;
  auto enqueue_cycle = [&](cudaStream_t st) -> int {
    const dim3 dgrid1(std::min<unsigned>(nblocks(n), 1024), 1);
    for (int j = 0; j < m; ++j) {
      precond(Vb + (size_t)j * n, zt, st, done);
      if (int r2 = arnoldi_matvec(zt, w, st, done)) return r2;
      for (int pass = 0; pass < 2; ++pass) {
        double* hp = pass == 0 ? gm->h : gm->h2;
        k_gm_zero<<<1, 64, 0, st>>>(hp, j + 1, done);
        k_multidot<<<dim3(dgrid1.x, j + 1), kThreads, 0, st>>>(n, Vb, n, w, hp, done);
        k_multiaxpy<<<nblocks(n), kThreads, 0, st>>>(n, Vb, n, hp, j + 1, w, done);
      }
      k_gm_zero<<<1, 64, 0, st>>>(&gm->wn2, 1, done);
      k_multidot<<<dgrid1, kThreads, 0, st>>>(n, w, n, w, &gm->wn2, done);
      k_gm_givens<<<1, 32, 0, st>>>(gm, j, m);
      k_gm_scale<<<nblocks(n), kThreads, 0, st>>>(gm, n, w, Vb + (size_t)(j + 1) * n);
    }
    k_gm_solve<<<1, 32, 0, st>>>(gm, m);
    HDG_CK(cudaMemsetAsync(w, 0, sizeof(double) * n, st));
    k_multiaxpy_add_dev<<<nblocks(n), kThreads, 0, st>>>(n, Vb, n, gm->y, &gm->jdone, w);
    precond(w, zt, st, nullptr);
    k_axpy<<<nblocks(n), kThreads, 0, st>>>(n, 1.0, zt, x);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
  };
  // the cycle as a CUDA graph, captured once for these buffers and replayed; if the capture
  // fails the same kernels are launched one by one
  const void* key[6] = {S, x, ctx->d_sw, Sdf, ctx->d_pc, ctx->d_pcn};
  if (ctx->gm_graph && !std::equal(key, key + 6, ctx->gm_key)) {
    cudaGraphExecDestroy(ctx->gm_graph);
    ctx->gm_graph = nullptr;
  }
  if (!ctx->gm_graph && !ctx->gm_graph_failed) {
    if (!ctx->gm_stream) HDG_CK(cudaStreamCreateWithFlags(&ctx->gm_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(ctx->gm_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const int rcap = ok ? enqueue_cycle(ctx->gm_stream) : HDG_OK;
    ok = cudaStreamEndCapture(ctx->gm_stream, &graph) == cudaSuccess && ok && rcap == HDG_OK;
    if (ok && cudaGraphInstantiate(&ctx->gm_graph, graph, 0) != cudaSuccess) {
      ctx->gm_graph = nullptr;
      ok = false;
    }
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
      cudaGetLastError();  // a failed capture is not an error of the solve
      ctx->gm_graph_failed = true;
    } else {
      std::copy(key, key + 6, ctx->gm_key);
    }
  }
  auto run_cycle = [&]() -> int {
    if (ctx->gm_graph) {
      LaunchScope ls(ctx, HDG_KERNEL_TRACE, s);
      HDG_CK(cudaGraphLaunch(ctx->gm_graph, s));
      ++ctx->gm_replays;
      return HDG_OK;
    }
    return enqueue_cycle(s);
  };
  HDG_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  double bn2;
  rc = dot_host(b, 1, b, &bn2);
  if (rc) return rc;
  const double bnorm = std::sqrt(bn2);
  *iters = 0;
  if (bnorm == 0.0) {
    *final_res = 0.0;
    return HDG_OK;
  }
  double rel = 1.0;
  int total = 0;
  bool first = true;
  // each cycle starts from the FP64 residual r = b - K x, which also decides convergence (the
  // Arnoldi products may use the double-float copy of S, whose residual estimate is not trusted)
  for (;;) {
    if (first) {
      HDG_CK(cudaMemcpyAsync(w, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    } else {
      rc = launch_trace_matvec(ctx, S, x, w, ew, s);
      if (rc) return rc;
      k_scale_copy<<<nblocks(n), kThreads, 0, s>>>(n, -1.0, w, w);
      k_axpy<<<nblocks(n), kThreads, 0, s>>>(n, 1.0, b, w);
    }
    first = false;
    double rn2;
    rc = dot_host(w, 1, w, &rn2);
    if (rc) return rc;
    double beta = std::sqrt(rn2);
    rel = beta / bnorm;
    if (rel <= rtol || total >= max_it) break;
    k_scale_copy<<<nblocks(n), kThreads, 0, s>>>(n, 1.0 / beta, w, Vb);
    // one restart cycle on the device: its starting state, the m Arnoldi steps (replayed as a
    // graph when one could be captured), the back substitution and x += M^{-1} V y
    GmState& hs = *static_cast<GmState*>(ctx->h_gm);
    hs.gv[0] = beta;
    hs.bnorm = bnorm;
    hs.rtol = rtol;
    hs.rel = rel;
    hs.done = 0;
    hs.jdone = 0;
    hs.total = total;
    hs.max_it = max_it;
    HDG_CK(cudaMemcpyAsync(gm, &hs, sizeof(GmState), cudaMemcpyHostToDevice, s));
    if ((rc = run_cycle())) return rc;
    HDG_CK(cudaMemcpyAsync(&hs, gm, sizeof(GmState), cudaMemcpyDeviceToHost, s));
    HDG_CK(cudaStreamSynchronize(s));
    total = hs.total;
    ++ctx->gm_cycles;
  }
  *final_res = rel;  // of the last FP64 residual
  *iters = total;
  if (ctx->d_mv_err) {  // a staged matvec gave up a copy wait
    int flag = 0;
    HDG_CK(cudaMemcpy(&flag, ctx->d_mv_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      HDG_CK(cudaMemset(ctx->d_mv_err, 0, sizeof(int)));
      set_error("trace_solve: a bulk copy of the trace operator did not complete");
      return HDG_ERR_TIMEOUT;
    }
  }
  if (*final_res > rtol * 10.0) {
    set_error("trace_solve: GMRES did not converge");
    return HDG_ERR_NOT_CONVERGED;
  }
  return HDG_OK;
}

int trace_solve(hdg_ctx* ctx, const double* S, const double* g, double* dVhat, int method, double rtol, int max_it,
                int* iters, double* final_res, cudaStream_t s) {
  if (method == HDG_SOLVER_AUTO) method = ctx->ntrace <= 4096 ? HDG_SOLVER_DENSE : HDG_SOLVER_GMRES;
  if (method == HDG_SOLVER_DENSE) {
    if (ctx->ntrace > 16384) {
      set_error("trace_solve: dense solver limited to n_trace <= 16384");
      return HDG_ERR_INVALID_ARG;
    }
    *iters = 1;
    return dense_solve(ctx, S, g, dVhat, final_res, s);
  }
  return gmres_solve(ctx, S, g, dVhat, rtol, max_it, iters, final_res, s);
}

}  // namespace hdg
