// Trace-space operations on meshes of mixed degree (the packed per-element layout of
// hdg_mesh_copy_layout): BDF history, the assembled trace operator K = sum_e P_e^T S_e P_e and its
// right-hand side, the face-block Jacobi preconditioner with blocks of each face's own size, the
// dense assembly, the interior recovery and the residual norm. The same operations as trace.cu
// for one degree; only the addressing differs (element e's trace vector has nt_e unknowns, face by
// face in its local face-node order; the trace node t = face_node_off[F] + c has one local
// occurrence per side of F).
#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.hpp"
#include "pclass.hpp"

namespace hdg {

namespace {

constexpr int kThreads = 256;
constexpr int M5 = 5, NF4 = 4;

inline unsigned nblk(int64_t n, int t = kThreads) {
  int64_t b = (n + t - 1) / t;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

__device__ __forceinline__ double wsum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

__device__ double bsum(double v) {
  __shared__ double part[32];
  v = wsum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) part[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < (int)((blockDim.x + 31) >> 5) ? part[lane] : 0.0;
    s = wsum(s);
  }
  return s;
}

// hist_e[a][i] = sum_g W_g |J| phi_a(x_g) (c0 u(v0) + c1 u(v1))_i at element e's own rule
__global__ void k_pm_history(PMixDev p, const double* geo, const double* V0, const double* V1, double c0, double c1,
                             double gamma, double* hist) {
  extern __shared__ double u[];  // [NG][M]
  const int64_t e = blockIdx.x;
  const PClassDev& T = p.tab[p.cls[e]];
  const int NP = T.d.NP, NG = T.d.NG;
  const double detJ = geo[e * (3 * 3 + 1 + NF4 * 4) + 9];
  const int64_t vo = p.voff[e];
  for (int g = threadIdx.x; g < NG; g += blockDim.x) {
    double acc[M5] = {0, 0, 0, 0, 0};
    for (int which = 0; which < 2; ++which) {
      const double* Vs = which == 0 ? V0 : V1;
      const double c = which == 0 ? c0 : c1;
      if (!Vs) continue;
      double v[M5];
      for (int i = 0; i < M5; ++i) {
        double s = 0.0;
        for (int b = 0; b < NP; ++b) s += T.Phi[g * NP + b] * Vs[vo + b * M5 + i];
        v[i] = s;
      }
      double rho, vel[3], pr;
      prim_of_v<3>(v, gamma, rho, vel, pr);
      double uu[M5];
      cons_and_flux<3>(rho, vel, pr, gamma, uu, (double(*)[3]) nullptr);
      for (int i = 0; i < M5; ++i) acc[i] += c * uu[i];
    }
    for (int i = 0; i < M5; ++i) u[g * M5 + i] = acc[i] * T.W[g] * detJ;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NP * M5; t += blockDim.x) {
    const int a = t / M5, i = t % M5;
    double s = 0.0;
    for (int g = 0; g < NG; ++g) s += T.Phi[g * NP + a] * u[g * M5 + i];
    hist[vo + t] = s;
  }
}

// w_e = S_e x_e, x_e gathered through the element's trace map (one warp per row)
__global__ void k_pm_elem_matvec(PMixDev p, const double* S, const double* x, double* w, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  extern __shared__ double xs[];
  const int64_t e = blockIdx.x;
  const int nt = (int)(p.toff[e + 1] - p.toff[e]);
  const int* tg = p.tgidx + e * NF4 * p.nfn_max;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    int f = 0, rem = t / M5;  // local node index of unknown t, face by face
    while (rem >= p.fnn[e * NF4 + f]) {
      rem -= p.fnn[e * NF4 + f];
      ++f;
    }
    xs[t] = x[(int64_t)tg[f * p.nfn_max + rem] * M5 + t % M5];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* Se = S + p.soff[e];
  for (int r = wid; r < nt; r += nw) {
    double s = 0.0;
    for (int c = lane; c < nt; c += 32) s += Se[(int64_t)r * nt + c] * xs[c];
    s = wsum(s);
    if (lane == 0) w[p.toff[e] + r] = s;
  }
}

// out[t][i] = scale * sum over the sides of the face of ge[toff[e_s] + loc_s + i]
__global__ void k_pm_gather(PMixDev p, int64_t ntn, const double* ge, double scale, double* out, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  const int64_t n = ntn * M5;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = t / M5;
    const int i = (int)(t % M5);
    double s = 0.0;
    for (int side = 0; side < 2; ++side) {
      const int e = p.occ_e[2 * node + side];
      if (e < 0) continue;
      s += ge[p.toff[e] + p.occ_l[2 * node + side] + i];
    }
    out[t] = scale * s;
  }
}

// dV_e = -y_e - X_e P_e dVhat
__global__ void k_pm_recover(PMixDev p, const double* recov, const double* dvh, double* dV) {
  extern __shared__ double xs[];
  const int64_t e = blockIdx.x;
  const int nt = (int)(p.toff[e + 1] - p.toff[e]);
  const int nv = (int)(p.voff[e + 1] - p.voff[e]);
  const int* tg = p.tgidx + e * NF4 * p.nfn_max;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    int f = 0, rem = t / M5;
    while (rem >= p.fnn[e * NF4 + f]) {
      rem -= p.fnn[e * NF4 + f];
      ++f;
    }
    xs[t] = dvh[(int64_t)tg[f * p.nfn_max + rem] * M5 + t % M5];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* X = recov + p.roff[e];
  const double* y = X + (int64_t)nv * nt;
  for (int r = wid; r < nv; r += nw) {
    double s = 0.0;
    for (int c = lane; c < nt; c += 32) s += X[(int64_t)r * nt + c] * xs[c];
    s = wsum(s);
    if (lane == 0) dV[p.voff[e] + r] = -y[r] - s;
  }
}

// sum over elements of |R_v,e|^2 (R_v,e: the first nv_e entries of element e's R block)
__global__ void k_pm_sumsq_rv(PMixDev p, int64_t E, const double* R, double* out) {
  double s = 0.0;
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    const int nv = (int)(p.voff[e + 1] - p.voff[e]);
    const double* r = R + p.Roff[e];
    for (int t = threadIdx.x; t < nv; t += blockDim.x) s += r[t] * r[t];
  }
  s = bsum(s);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

// |sum_e P_e^T R_t,e|^2
__global__ void k_pm_sumsq_rt(PMixDev p, int64_t ntn, const double* R, double* out) {
  double s = 0.0;
  const int64_t n = ntn * M5;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = t / M5;
    const int i = (int)(t % M5);
    double v = 0.0;
    for (int side = 0; side < 2; ++side) {
      const int e = p.occ_e[2 * node + side];
      if (e < 0) continue;
      const int64_t nv = p.voff[e + 1] - p.voff[e];
      v += R[p.Roff[e] + nv + p.occ_l[2 * node + side] + i];
    }
    s += v * v;
  }
  s = bsum(s);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

// face-block Jacobi: K_FF = sum over the sides of S_e restricted to the face's unknowns (the
// face's own size B = Nf(q_F) m <= 75), LU with partial pivoting, inverse stored transposed at
// pc + pcoff[F] (pc[F][j][i] = K_FF^{-1}[i][j])
constexpr int kMaxB = 80;
__global__ void k_pm_face_factor(PMixDev p, const double* S, double* pc) {
  extern __shared__ double A[];  // [B][B], then the inverse [B][B]
  __shared__ int s_p;
  __shared__ int s_piv[kMaxB];
  const int64_t F = blockIdx.x;
  const int64_t t0 = p.fnoff[F];
  const int B = (int)(p.fnoff[F + 1] - t0) * M5;
  for (int t = threadIdx.x; t < B * B; t += blockDim.x) {
    const int r = t / B, c = t % B;
    double s = 0.0;
    for (int side = 0; side < 2; ++side) {
      const int e = p.occ_e[2 * (t0 + r / M5) + side];
      if (e < 0) continue;
      const int nt = (int)(p.toff[e + 1] - p.toff[e]);
      const int lr = p.occ_l[2 * (t0 + r / M5) + side] + r % M5;
      const int lc = p.occ_l[2 * (t0 + c / M5) + side] + c % M5;
      s += S[p.soff[e] + (int64_t)lr * nt + lc];
    }
    A[t] = s;
  }
  __syncthreads();
  for (int k = 0; k < B; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int r = k + threadIdx.x; r < B; r += 32) {
        const double v = fabs(A[r * B + k]);
        if (v > best) {
          best = v;
          bi = r;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
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
    const int pr = s_p;
    if (pr != k)
      for (int j = threadIdx.x; j < B; j += blockDim.x) {
        const double t = A[k * B + j];
        A[k * B + j] = A[pr * B + j];
        A[pr * B + j] = t;
      }
    __syncthreads();
    const double d = A[k * B + k];
    const double inv = d != 0.0 ? 1.0 / d : 0.0;
    for (int r = k + 1 + threadIdx.x; r < B; r += blockDim.x) A[r * B + k] *= inv;
    __syncthreads();
    const int rem = B - k - 1;
    for (int t = threadIdx.x; t < rem * rem; t += blockDim.x) {
      const int r = k + 1 + t / rem, c = k + 1 + t % rem;
      A[r * B + c] -= A[r * B + k] * A[k * B + c];
    }
    __syncthreads();
  }
  double* X = A + B * B;
  for (int t = threadIdx.x; t < B; t += blockDim.x) {  // column t of the inverse
    for (int i = 0; i < B; ++i) X[i * B + t] = i == t ? 1.0 : 0.0;
    for (int k = 0; k < B; ++k) {
      const int pk = s_piv[k];
      if (pk != k) {
        const double tmp = X[k * B + t];
        X[k * B + t] = X[pk * B + t];
        X[pk * B + t] = tmp;
      }
    }
    for (int k = 0; k < B; ++k) {
      const double xk = X[k * B + t];
      for (int r = k + 1; r < B; ++r) X[r * B + t] -= A[r * B + k] * xk;
    }
    for (int k = B - 1; k >= 0; --k) {
      const double d = A[k * B + k];
      const double xk = d != 0.0 ? X[k * B + t] / d : 0.0;
      X[k * B + t] = xk;
      for (int r = 0; r < k; ++r) X[r * B + t] -= A[r * B + k] * xk;
    }
  }
  __syncthreads();
  double* out = pc + p.pcoff[F];
  for (int t = threadIdx.x; t < B * B; t += blockDim.x) {
    const int j = t / B, i = t % B;
    out[t] = X[i * B + j];
  }
}

// z_F = K_FF^{-1} r_F, one warp per face (B <= 80: lanes take rows i, i + 32, i + 64)
__global__ void k_pm_face_apply(PMixDev p, int64_t F, const double* pc, const double* r, double* z, const int* skip) {
  if (skip && *skip) return;  // a finished Krylov cycle: nothing to do
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t Fi = (int64_t)blockIdx.x * nw + wid;
  if (Fi >= F) return;
  const int64_t b0 = p.fnoff[Fi] * M5;
  const int B = (int)(p.fnoff[Fi + 1] * M5 - b0);
  const double* A = pc + p.pcoff[Fi];
  double a[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < B; ++j) {
    const double rj = r[b0 + j];
    for (int k = 0; k < 3; ++k) {
      const int i = lane + 32 * k;
      if (i < B) a[k] += A[j * B + i] * rj;
    }
  }
  for (int k = 0; k < 3; ++k) {
    const int i = lane + 32 * k;
    if (i < B) z[b0 + i] = a[k];
  }
}

// K[gr][gc] += S_e[r][c] over every element (dense assembly for the direct solver)
__global__ void k_pm_dense_scatter(PMixDev p, const double* S, int64_t E, int64_t n, double* K) {
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    const int nt = (int)(p.toff[e + 1] - p.toff[e]);
    const int* tg = p.tgidx + e * NF4 * p.nfn_max;
    for (int t = threadIdx.x; t < nt * nt; t += blockDim.x) {
      const int r = t / nt, c = t % nt;
      auto glob = [&](int u) {
        int f = 0, rem = u / M5;
        while (rem >= p.fnn[e * NF4 + f]) {
          rem -= p.fnn[e * NF4 + f];
          ++f;
        }
        return (int64_t)tg[f * p.nfn_max + rem] * M5 + u % M5;
      };
      atomicAdd(K + glob(r) * n + glob(c), S[p.soff[e] + t]);
    }
  }
}

}  // namespace

PMixDev pmix_dev(const hdg_ctx* c) {
  const PMix& pm = *c->pm;
  PMixDev d{};
  d.voff = pm.d_voff;
  d.toff = pm.d_toff;
  d.soff = pm.d_soff;
  d.roff = pm.d_roff;
  d.Roff = pm.d_Roff;
  d.tgidx = pm.d_tgidx;
  d.fnn = pm.d_fnn;
  d.cls = pm.d_cls;
  d.occ_e = pm.d_occ_e;
  d.occ_l = pm.d_occ_l;
  d.fnoff = pm.d_fnoff;
  d.pcoff = pm.d_pcoff;
  d.nfn_max = pm.nfn_max;
  for (int k = 0; k < kPClasses; ++k) d.tab[k] = pm.tab[k];
  return d;
}

int pm_history(hdg_ctx* c, const double* V0, const double* V1, double c0, double c1, double* hist, cudaStream_t s) {
  const size_t sm = sizeof(double) * 125 * M5;  // the largest volume rule (p = 4)
  k_pm_history<<<(unsigned)c->E, 128, sm, s>>>(pmix_dev(c), c->d_geo, V0, V1, c0, c1, c->ph.gamma, hist);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int pm_gather(hdg_ctx* c, const double* ge, double scale, double* out, cudaStream_t s, const int* skip) {
  k_pm_gather<<<nblk(c->ntrace), kThreads, 0, s>>>(pmix_dev(c), c->n_tnodes, ge, scale, out, skip);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int pm_elem_matvec(hdg_ctx* c, const double* S, const double* x, double* w, cudaStream_t s, const int* skip) {
  k_pm_elem_matvec<<<(unsigned)c->E, 256, sizeof(double) * c->pm->nt_max, s>>>(pmix_dev(c), S, x, w, skip);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int pm_recover(hdg_ctx* c, const double* recov, const double* dvh, double* dV, cudaStream_t s) {
  k_pm_recover<<<(unsigned)c->E, 256, sizeof(double) * c->pm->nt_max, s>>>(pmix_dev(c), recov, dvh, dV);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int pm_sumsq(hdg_ctx* c, const double* R, double* red, cudaStream_t s) {
  k_pm_sumsq_rv<<<nblk(c->E, 1) < 4096 ? nblk(c->E, 1) : 4096, kThreads, 0, s>>>(pmix_dev(c), c->E, R, red);
  k_pm_sumsq_rt<<<nblk(c->ntrace), kThreads, 0, s>>>(pmix_dev(c), c->n_tnodes, R, red + 1);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int pm_face_factor(hdg_ctx* c, const double* S, double* pc, cudaStream_t s) {
  const int B = c->pm->nfn_max * M5;
  const size_t sm = 2 * sizeof(double) * B * B;
  if (!c->pm->attr_face) {
    HDG_CK(cudaFuncSetAttribute(k_pm_face_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    c->pm->attr_face = true;
  }
  k_pm_face_factor<<<(unsigned)c->F, 128, sm, s>>>(pmix_dev(c), S, pc);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int pm_face_apply(hdg_ctx* c, const double* pc, const double* r, double* z, cudaStream_t s, const int* skip) {
  const int wpb = 8;
  k_pm_face_apply<<<(unsigned)((c->F + wpb - 1) / wpb), 32 * wpb, 0, s>>>(pmix_dev(c), c->F, pc, r, z, skip);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

int pm_dense_scatter(hdg_ctx* c, const double* S, int64_t n, double* K, cudaStream_t s) {
  k_pm_dense_scatter<<<(unsigned)std::min<int64_t>(c->E, 4096), 256, 0, s>>>(pmix_dev(c), S, c->E, n, K);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

}  // namespace hdg
