// Boundary faces: the term <b_h(vhat, v), mu> of Eqs. hDG2 / hDG_NS2 (the paper leaves b_h
// open, Sec. 3.2). The element assembly treats every face alike and leaves, for a face with
// one side, the rows of an interior face in R_t, C and D; k_boundary_patch overwrites those
// rows with the boundary term (the R_v rows keep fhat + ghat with the face's trace):
//   HDG_BC_STATE  b_h = vhat - v_b: R_t = <vhat - v_b, mu>, D = <mu, mu'> I on the face's own
//                 columns (0 elsewhere), C = 0;
//   HDG_BC_SLIP   b_h = fhat(vhat, v; n) + fhat(vhat, R v; -n), R reflecting the momentum
//                 components in the wall plane (Euler): its derivatives with respect to vhat
//                 and v by dual numbers, D on the face's own columns, C over the element's v.
// One CTA per boundary face of the chunk; the threads of the face points evaluate b_h and its
// derivatives, then all threads form the integrals against the trace and element bases.
// EDG on a bounded mesh imposes the state strongly instead, since a boundary node of its
// continuous trace is shared with interior faces: k_dirichlet_patch clears the R_t, C and D rows
// of every occurrence of such a node in an element's local trace and gives one occurrence per
// node the row of vhat - v_b (D = I on its own columns, R_t = vhat - v_b), so the assembled
// equation of the node is vhat = v_b.
#include <algorithm>

#include "assemble_fp64.cuh"
#include "ctx.hpp"

namespace hdg {

namespace {

// the mirror image of a state in the plane with unit normal n: w -> w - 2 (w . n) n
template <int D, class T>
HDG_DEVI void reflect_state(const T* v, const double* n, T* out) {
  T wn = v[1] * n[0];
#pragma unroll
  for (int j = 1; j < D; ++j) wn = wn + v[1 + j] * n[j];
  out[0] = v[0];
#pragma unroll
  for (int j = 0; j < D; ++j) out[1 + j] = v[1 + j] - (2.0 * n[j]) * wn;
  out[D + 1] = v[D + 1];
}

// fhat(vhat, v; n) of Eq. numericalFlux, sigma at v* = vhat: lambda_max A0 (Eq. sLxF) or, with
// SYM, |A_n| A0 (Eq. symStab)
template <int D, bool SYM, class T>
HDG_DEVI void euler_numflux(const T* vh, const T* v, const double* n, double gamma, T* out) {
  constexpr int M = D + 2;
  T rh, velh[D], prh, uh[M], Fh[M][D];
  prim_of_v<D>(vh, gamma, rh, velh, prh);
  cons_and_flux<D>(rh, velh, prh, gamma, uh, Fh);
  T rv, velv[D], pv, Fv[M][D];
  prim_of_v<D>(v, gamma, rv, velv, pv);
  cons_and_flux<D>(rv, velv, pv, gamma, (T*)nullptr, Fv);
  T dv[M], du[M], sdu[M];
#pragma unroll
  for (int i = 0; i < M; ++i) dv[i] = v[i] - vh[i];
  du_of_v<D>(vh, dv, gamma, du);
  if constexpr (SYM) {
    abs_flux_jac_apply<D>(rh, velh, prh, n, gamma, du, sdu);
  } else {
    const T lam = lambda_max<D>(rh, velh, prh, n, gamma);
#pragma unroll
    for (int i = 0; i < M; ++i) sdu[i] = lam * du[i];
  }
#pragma unroll
  for (int i = 0; i < M; ++i) {
    T s = (Fh[i][0] + Fv[i][0]) * n[0];
#pragma unroll
    for (int j = 1; j < D; ++j) s = s + (Fh[i][j] + Fv[i][j]) * n[j];
    out[i] = 0.5 * s + 0.5 * sdu[i];
  }
}

// W b_h of the slip wall at one face point with its derivatives W db/dvhat (dH) and W db/dv (dV)
template <int D, bool SYM>
HDG_DEVI void slip_terms(const double* vh, const double* v, const double* n, double gamma, double W, double* b,
                         double (*dH)[D + 2], double (*dV)[D + 2]) {
  constexpr int M = D + 2;
  double nm[D];
  for (int j = 0; j < D; ++j) nm[j] = -n[j];
  for (int pass = 0; pass < 2; ++pass) {  // 0: seeds on vhat, 1: seeds on v
    Dual<M> xh[M], xv[M], xr[M], f1[M], f2[M];
    for (int l = 0; l < M; ++l) {
      xh[l] = dconst<M>(vh[l]);
      xv[l] = dconst<M>(v[l]);
      if (pass == 0)
        xh[l].d[l] = 1.0;
      else
        xv[l].d[l] = 1.0;
    }
    reflect_state<D>(xv, n, xr);
    euler_numflux<D, SYM>(xh, xv, n, gamma, f1);
    euler_numflux<D, SYM>(xh, xr, nm, gamma, f2);
    for (int i = 0; i < M; ++i) {
      if (pass == 0) b[i] = W * (f1[i].v + f2[i].v);
      for (int l = 0; l < M; ++l) (pass == 0 ? dH : dV)[i][l] = W * (f1[i].d[l] + f2[i].d[l]);
    }
  }
}

template <class C, class OutT, bool SYM>
__global__ void __launch_bounds__(128) k_boundary_patch(AssembleArgs a, DevTables T, PhysParams ph, const int* bface,
                                                        const int* bkind, const double* Vb) {
  constexpr int D = C::D, M = C::M, NP = C::NP, NFN = C::NFN, NF = C::NF, NGF = C::NGF, NV = C::NV, NT = C::NT;
  __shared__ double z[NP][M];       // element state at its nodes
  __shared__ double zh[NFN][M];     // the face's trace, local face-node order
  __shared__ double zb[NFN][M];     // the boundary state there (BC_STATE)
  __shared__ double sb[NGF][M];     // W b_h at the face points
  __shared__ double sH[NGF][M][M];  // W db_h/dvhat
  __shared__ double sV[NGF][M][M];  // W db_h/dv
  __shared__ double nrm[D + 1];     // outward normal, surface Jacobian
  const int entry = bface[blockIdx.x];
  const int64_t e = entry / NF;
  const int f = entry % NF;
  if (skip_element(a, e)) return;
  const int kind = bkind[blockIdx.x];
  const int64_t le = e - a.e0;
  for (int t = threadIdx.x; t < NP * M; t += blockDim.x) z[t / M][t % M] = a.V[e * NP * M + t];
  for (int t = threadIdx.x; t < NFN * M; t += blockDim.x) {
    const int c = t / M, i = t % M;
    const int64_t node = a.tgidx[(e * NF + f) * NFN + c];
    zh[c][i] = a.Vhat[node * M + i];
    zb[c][i] = kind == HDG_BC_STATE ? Vb[node * M + i] : 0.0;
  }
  for (int t = threadIdx.x; t < D + 1; t += blockDim.x) nrm[t] = a.geo[e * C::GEO + D * D + 1 + f * (D + 1) + t];
  __syncthreads();
  if (threadIdx.x < NGF) {
    const int g = threadIdx.x;
    const double* phif = T.PhiF + (f * NGF + g) * NP;
    const double W = T.WF[g] * nrm[D];
    double v[M], vh[M], vb[M];
    for (int i = 0; i < M; ++i) {
      double s = 0.0, sh = 0.0, sbv = 0.0;
      for (int b = 0; b < NP; ++b) s += phif[b] * z[b][i];
      for (int c = 0; c < NFN; ++c) {
        const double psi = phif[T.fnodes[f * NFN + c]];
        sh += psi * zh[c][i];
        sbv += psi * zb[c][i];
      }
      v[i] = s;
      vh[i] = sh;
      vb[i] = sbv;
    }
    if (kind == HDG_BC_STATE) {
      for (int i = 0; i < M; ++i) {
        sb[g][i] = W * (vh[i] - vb[i]);
        for (int l = 0; l < M; ++l) {
          sH[g][i][l] = i == l ? W : 0.0;
          sV[g][i][l] = 0.0;
        }
      }
    } else {
      if constexpr (!C::VISC) slip_terms<D, SYM>(vh, v, nrm, ph.gamma, W, sb[g], sH[g], sV[g]);
    }
  }
  __syncthreads();
  const double* PF = T.PhiF + f * NGF * NP;
  auto psi = [&](int g, int c) { return PF[g * NP + T.fnodes[f * NFN + c]]; };
  constexpr int RB = NFN * M;  // rows of the face
  double* Rt = a.R + e * (int64_t)(NV + NT) + NV + f * RB;
  for (int t = threadIdx.x; t < RB; t += blockDim.x) {
    const int c = t / M, i = t % M;
    double s = 0.0;
    for (int g = 0; g < NGF; ++g) s += psi(g, c) * sb[g][i];
    Rt[t] = s;
  }
  OutT* Cr = reinterpret_cast<OutT*>(a.Cp) + (le * NT + f * RB) * (int64_t)NV;
  for (int t = threadIdx.x; t < RB * NV; t += blockDim.x) {
    const int r = t / NV, col = t % NV;
    const int c = r / M, i = r % M, b = col / M, l = col % M;
    double s = 0.0;
    if (kind != HDG_BC_STATE)
      for (int g = 0; g < NGF; ++g) s += psi(g, c) * sV[g][i][l] * PF[g * NP + b];
    put(Cr, t, s);
  }
  OutT* Dr = reinterpret_cast<OutT*>(a.S + e * (int64_t)NT * NT) + (int64_t)f * RB * NT;
  for (int t = threadIdx.x; t < RB * NT; t += blockDim.x) {
    const int r = t / NT, col = t % NT;
    const int c = r / M, i = r % M;
    double s = 0.0;
    if (col / RB == f) {
      const int cc = (col % RB) / M, l = col % M;
      for (int g = 0; g < NGF; ++g) s += psi(g, c) * psi(g, cc) * sH[g][i][l];
    }
    put(Dr, t, s);
  }
}

// One CTA per occurrence dir[k] = (e NF + f) NFN + c of a strongly imposed node in the chunk;
// first[k] != 0 for the one occurrence of each node that carries its equation.
template <class C, class OutT>
__global__ void __launch_bounds__(128) k_dirichlet_patch(AssembleArgs a, const int* dir, const int* first,
                                                         const double* Vb) {
  constexpr int M = C::M, NFN = C::NFN, NF = C::NF, NV = C::NV, NT = C::NT;
  const int entry = dir[blockIdx.x];
  const int64_t e = entry / (NF * NFN);
  const int r0 = (entry % (NF * NFN)) * M;  // the node's first row in the local trace order
  if (skip_element(a, e)) return;
  const int64_t le = e - a.e0;
  double* Rt = a.R + e * (int64_t)(NV + NT) + NV;
  OutT* Cr = reinterpret_cast<OutT*>(a.Cp) + (le * NT + r0) * (int64_t)NV;
  OutT* Dr = reinterpret_cast<OutT*>(a.S + e * (int64_t)NT * NT) + (int64_t)r0 * NT;
  for (int t = threadIdx.x; t < M * NV; t += blockDim.x) put(Cr, t, 0.0);
  for (int t = threadIdx.x; t < M * NT; t += blockDim.x) put(Dr, t, 0.0);
  for (int t = threadIdx.x; t < M; t += blockDim.x) Rt[r0 + t] = 0.0;
  __syncthreads();
  if (first[blockIdx.x] && threadIdx.x < M) {
    const int i = threadIdx.x;
    const int64_t node = a.tgidx[entry];
    put(Dr, i * NT + r0 + i, 1.0);
    Rt[r0 + i] = a.Vhat[node * M + i] - Vb[node * M + i];
  }
}

template <class C, class OutT>
int run_dirichlet(hdg_ctx* ctx, const AssembleArgs& a, cudaStream_t s) {
  const std::vector<int>& dir = ctx->h_dir;
  const int per = ctx->NF * ctx->NFN;
  const int64_t lo = std::lower_bound(dir.begin(), dir.end(), (int)(a.e0 * per)) - dir.begin();
  const int64_t hi = std::lower_bound(dir.begin(), dir.end(), (int)((a.e0 + a.ne) * per)) - dir.begin();
  if (hi <= lo) return HDG_OK;
  k_dirichlet_patch<C, OutT><<<(unsigned)(hi - lo), 128, 0, s>>>(a, ctx->d_dir + lo, ctx->d_dir_first + lo, ctx->d_vb);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

template <class C, class OutT>
int run_patch(hdg_ctx* ctx, const AssembleArgs& a, int64_t lo, int64_t cnt, cudaStream_t s) {
  LaunchScope ls(ctx, HDG_KERNEL_ASSEMBLE, s);
  const int* bf = ctx->d_bface + lo;
  const int* bk = ctx->d_bkind + lo;
  if (cnt > 0) {
    bool sym = false;
    if constexpr (!C::VISC) sym = ctx->ph.stab == 1;
    if (sym) {
      if constexpr (!C::VISC) k_boundary_patch<C, OutT, true><<<(unsigned)cnt, 128, 0, s>>>(a, ctx->T, ctx->ph, bf, bk, ctx->d_vb);
    } else {
      k_boundary_patch<C, OutT, false><<<(unsigned)cnt, 128, 0, s>>>(a, ctx->T, ctx->ph, bf, bk, ctx->d_vb);
    }
    HDG_CK(cudaGetLastError());
  }
  // after the boundary term: the strongly imposed nodes of EDG overwrite their rows
  return ctx->h_dir.empty() ? HDG_OK : run_dirichlet<C, OutT>(ctx, a, s);
}

}  // namespace

#define HDG_PATCH_CASE(D, P, VISC)                                                      \
  if (ctx->dim == D && ctx->p == P && ctx->K == P + 1 && ctx->visc == VISC)            \
    return precision == HDG_PREC_MIXED ? run_patch<Cfg<D, P, P + 1, VISC>, df2>(ctx, a, lo, cnt, s) \
                                       : run_patch<Cfg<D, P, P + 1, VISC>, double>(ctx, a, lo, cnt, s);

int boundary_patch(hdg_ctx* ctx, const AssembleArgs& a, int precision, cudaStream_t s) {
  if (ctx->h_bface.empty()) return HDG_OK;
  if (ctx->has_state_bc && !ctx->vb_set) {
    set_error("assemble_condense: the boundary state of the HDG_BC_STATE faces is not set");
    return HDG_ERR_INVALID_ARG;
  }
  const std::vector<int>& bf = ctx->h_bface;
  const int64_t lo = std::lower_bound(bf.begin(), bf.end(), (int)(a.e0 * ctx->NF)) - bf.begin();
  const int64_t hi = std::lower_bound(bf.begin(), bf.end(), (int)((a.e0 + a.ne) * ctx->NF)) - bf.begin();
  const int64_t cnt = hi - lo;
  if (cnt <= 0 && ctx->h_dir.empty()) return HDG_OK;
  HDG_PATCH_CASE(2, 1, false)
  HDG_PATCH_CASE(2, 2, false)
  HDG_PATCH_CASE(2, 3, false)
  HDG_PATCH_CASE(2, 4, false)
  HDG_PATCH_CASE(2, 1, true)
  HDG_PATCH_CASE(2, 2, true)
  HDG_PATCH_CASE(2, 3, true)
  HDG_PATCH_CASE(2, 4, true)
  HDG_PATCH_CASE(3, 1, true)
  HDG_PATCH_CASE(3, 2, true)
  HDG_PATCH_CASE(3, 3, true)
  set_error("boundary_patch: configuration not compiled in");
  return HDG_ERR_UNSUPPORTED;
}

}  // namespace hdg
