// Mixed-degree assemble + condense (FP64): every element of a mesh whose elements differ in
// degree, in ONE persistent launch over a work queue ordered by element class.
//
// The paper uses one degree k everywhere; elements of different degree in one mesh are this
// library's extension (a mesh with p_per_elem). Element e has degree pk = p_e; the trace on a face
// has the larger degree of its two sides, q_F = max(p_L, p_R); the element's trace degree pt is
// the largest of its faces' degrees. An element class is the pair (pk, pt), pt >= pk; 3D
// Navier-Stokes has ten classes (pk, pt in 1..4).
//
// Per element the kernel runs the steps of the uniform FP64 form (assemble_fp64.cuh) with the
// trace of every face expressed in the nodal space of degree pt:
//   1. gather vhat at the face's own nodes (degree q_f) and prolong it to the degree-pt nodes,
//      vhat_pt = I_f vhat_q (exact: P_q is contained in P_pt);
//   2. pointwise fluxes and exact pointwise Jacobians (dual numbers) at the volume points (rule
//      with pk + 1 points per direction) and face points (pt + 1), into per-CTA scratch;
//   3. the quadrature contractions into A', B', C', D' and the residuals R_v, R_t (q eliminated
//      exactly through Eq. hDG_NS0, the lift taken in the degree-pt trace space);
//   4. the blocks in the element's own trace space: B_q = B' P, C_q = P^T C', D_q = P^T D' P,
//      R_t,q = P^T R_t, P = block-diag(I_f) (the test functions of degree q_f are combinations
//      of the degree-pt ones with the same coefficients);
//   5. LU of A' (in shared memory when it fits, else in the CTA's global-memory scratch),
//      X = A'^{-1} [B_q | R_v], S = D_q - C_q X, g = R_t,q - C_q y.
// Outputs are packed per element at the offsets of the mesh layout (hdg_mesh_copy_layout):
// S [nt_e][nt_e], g [nt_e], recov [nv_e nt_e + nv_e] (X then y), R [nv_e + nt_e], with
// nt_e = sum_f Nf(q_f) m the element's own trace unknowns in [face][face node][component] order.
//
// The launch is persistent: one CTA of 256 threads per SM; thread 0 takes the next queue entry
// with an atomic counter, the queue lists the elements largest class first (longest work first),
// and one code path serves every class, reading the class's sizes and tables at run time. A 3D
// mesh of the single degree 4, which has no uniform kernels, runs here as the class (4, 4).
#include <algorithm>
#include <cstring>
#include <vector>

#include "assemble_fp64.cuh"
#include "ctx.hpp"
#include "pclass.hpp"

namespace hdg {

namespace {

// Sizes of one class (pk, pt), 3D Navier-Stokes: computed on the host, read by the kernel at run
// time (one code path serves every class, so the launch compiles once).
constexpr int D3 = 3, M5 = 5, NF4 = 4, GEO3 = D3 * D3 + 1 + NF4 * (D3 + 1);
constexpr int NR3 = D3 + 1, NRF3 = D3 + 2;  // value (+ gradient) right operators, volume and face
constexpr int PT_VOL = M5 + D3 * M5 + M5 * M5 + D3 * M5 * M5 + D3 * M5 * M5 * D3;
constexpr int PT_FACE = M5 + 2 * M5 * M5 + M5 * M5 * D3;
constexpr int kLuSmemMax = 12000;     // A' (doubles) factored in shared memory up to this size

// gt: volume points per contraction tile; cb: right-hand-side columns per block of the
// triangular solves (both chosen per class by the autotuner, pclass_autotune)
inline PDims pclass_dims(int pk, int pt, int gt = 32, int cb = 32) {
  PDims d{};
  d.pk = pk;
  d.pt = pt;
  d.NP = (pk + 1) * (pk + 2) * (pk + 3) / 6;
  d.NFK = (pk + 1) * (pk + 2) / 2;
  d.NFN = (pt + 1) * (pt + 2) / 2;
  d.NG = (pk + 1) * (pk + 1) * (pk + 1);
  d.NGF = (pt + 1) * (pt + 1);
  d.NV = d.NP * M5;
  d.NT = NF4 * d.NFN * M5;
  d.NZ = d.NP + NF4 * d.NFN;
  d.GT = d.NG < gt ? d.NG : gt;
  d.CB = cb;
  const int RB = NR3 * d.GT * d.NZ, RBF = NRF3 * d.NGF * d.NZ;
  const int ZS = d.NP * d.GT * NR3, ZSF = (d.NFK + d.NFN) * d.NGF * NRF3;
  d.RBMAX = RB > RBF ? RB : RBF;
  d.ASM = d.RBMAX + (ZS > ZSF ? ZS : ZSF);
  d.lu_smem = d.NV * d.NV <= kLuSmemMax ? 1 : 0;
  d.CND = (d.lu_smem ? d.NV * d.NV : 0) + d.NV * cb;
  d.KEEP = d.NZ * M5 + GEO3 + NF4 * d.NFN * M5 + d.NV + d.NT;
  d.SMEM = d.KEEP + (d.ASM > d.CND ? d.ASM : d.CND) + (d.NV + 1) / 2 + 2;  // + pivots (int)
  d.SLOT = (int64_t)d.NG * PT_VOL + (int64_t)NF4 * d.NGF * PT_FACE + (int64_t)d.NV * d.NV +
           3 * (int64_t)d.NV * d.NT + 2 * (int64_t)d.NT * d.NT;
  return d;
}

constexpr int kThreads = 256;

struct PArgs {
  const double* V;       // element e's [NP_e][M] at V + voff[e]
  const double* Vhat;    // [trace nodes][M]
  const double* hist;    // like V, or null
  double mass_coef;
  const int64_t* voff;   // [E + 1]
  const int64_t* toff;   // [E + 1] trace unknowns nt_e (g)
  const int64_t* soff;   // [E + 1] nt_e^2 (S)
  const int64_t* roff;   // [E + 1] nv_e nt_e + nv_e (recov)
  const int64_t* Roff;   // [E + 1] nv_e + nt_e (R)
  const int* tgidx;      // [E][NF][nfn_max] trace node of each local face node (-1 beyond)
  const int8_t* fdeg;    // [E][NF] degree of each face of the element
  const int8_t* cls;     // [E] class index
  const double* geo;     // [E][GEO]
  const int* queue;      // [E] elements, largest class first
  int64_t E;
  int nfn_max;
  int64_t slot_doubles;
  int* counter;          // work counter (zeroed before the launch)
  double* scratch;       // [grid][slot_doubles]
  double* S;
  double* g;
  double* recov;
  double* R;
  int* status;
  PClassDev tab[kPClasses];
};

HDG_DEVI int nfn3(int q) { return (q + 1) * (q + 2) / 2; }

// ----------------------------------------------------------------------------------- step 2
// One thread per quadrature point: fluxes and exact pointwise Jacobians by dual numbers,
// pre-contracted with the weights and Jinv (the per-point tensors of k_pointwise, FP64).
__device__ void pc_pointwise(const PArgs& a, const PClassDev& T, const PhysParams& ph, const double (*z)[M5],
                             const double (*dz)[M5], const double* G, double* ptv, double* ptf, int64_t e) {
  constexpr int D = D3, M = M5, NF = NF4;
  const int NP = T.d.NP, NFN = T.d.NFN, NG = T.d.NG, NGF = T.d.NGF;
  const double* Jinv = G;
  const double detJ = G[D * D];
  const int tid = threadIdx.x;
  bool bad = false;
  // q at a point from its element-gradient part gr[i][r] and the lifts of the face jumps
  auto lifted_q = [&](const double (*gr)[D], const double (*lift)[NF], double (*q)[D]) {
    for (int i = 0; i < M; ++i)
      for (int k = 0; k < D; ++k) {
        double s = 0.0;
        for (int r = 0; r < D; ++r) s += Jinv[r * D + k] * gr[i][r];
        for (int f = 0; f < NF; ++f) {
          const double* Gf = G + D * D + 1 + f * (D + 1);
          s += Gf[k] * (Gf[D] / detJ) * lift[i][f];
        }
        q[i][k] = s;
      }
  };
  if (tid < NG) {
    const int g = tid;
    const double W = T.W[g] * detJ;
    double v[M], gr[M][D], lift[M][NF], q[M][D];
    for (int i = 0; i < M; ++i) {
      double s = 0.0;
      for (int b = 0; b < NP; ++b) s += T.Phi[g * NP + b] * z[b][i];
      v[i] = s;
      for (int r = 0; r < D; ++r) {
        double t = 0.0;
        for (int b = 0; b < NP; ++b) t += T.dPhi[(r * NG + g) * NP + b] * z[b][i];
        gr[i][r] = t;
      }
      for (int f = 0; f < NF; ++f) {
        double l = 0.0;
        for (int c = 0; c < NFN; ++c) l += T.PL[(f * NG + g) * NFN + c] * dz[f * NFN + c][i];
        lift[i][f] = l;
      }
    }
    lifted_q(gr, lift, q);
    bad = !(v[M - 1] < 0.0);
    Dual<M> vd[M];
    for (int l = 0; l < M; ++l) {
      vd[l] = dconst<M>(v[l]);
      vd[l].d[l] = 1.0;
    }
    Dual<M> rho, vel[D], p, u[M], F[M][D];
    prim_of_v<D>(vd, ph.gamma, rho, vel, p);
    cons_and_flux<D>(rho, vel, p, ph.gamma, u, F);
    bad = bad || !(rho.v > 0.0) || !(p.v > 0.0);
    {
      Dual<M> Gv[M][D];
      visc_flux<D>(vd, q, ph, Gv);
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < D; ++j) F[i][j] = F[i][j] + Gv[i][j];
    }
    double* MU = ptv + g * PT_VOL;
    double* FR = MU + M;
    double* T0 = FR + D * M;
    double* T1 = T0 + M * M;
    double* T2 = T1 + D * M * M;
    for (int i = 0; i < M; ++i) {
      MU[i] = W * a.mass_coef * u[i].v;
      for (int l = 0; l < M; ++l) T0[i * M + l] = W * a.mass_coef * u[i].d[l];
    }
    for (int r = 0; r < D; ++r)
      for (int i = 0; i < M; ++i) {
        double s = 0.0;
        for (int j = 0; j < D; ++j) s += Jinv[r * D + j] * F[i][j].v;
        FR[r * M + i] = -W * s;
        for (int l = 0; l < M; ++l) {
          double t = 0.0;
          for (int j = 0; j < D; ++j) t += Jinv[r * D + j] * F[i][j].d[l];
          T1[(r * M + i) * M + l] = -W * t;
        }
      }
    const ViscFactors<D> vf = visc_factors<D>(v);
    const PhysParams pv = visc_params_at(ph, v[M - 1]);
#pragma unroll 1
    for (int r = 0; r < D; ++r)
      visc_jac_dir<D>(vf, Jinv + r * D, pv,
                      [&](int i, int l, int k, double val) { T2[((r * M + i) * M + l) * D + k] = -W * val; });
  } else if (tid < NG + NF * NGF) {
    const int f = (tid - NG) / NGF;
    const int gf = (tid - NG) % NGF;
    const double* Gf = G + D * D + 1 + f * (D + 1);
    const double* n = Gf;
    const double Wf = T.WF[gf] * Gf[D];
    const double* phif = T.PhiF + (f * NGF + gf) * NP;
    const double* psif = T.PsiF + (f * NGF + gf) * NFN;
    double v[M], vh[M], gr[M][D], lift[M][NF], q[M][D];
    for (int i = 0; i < M; ++i) {
      double s = 0.0, sh = 0.0;
      for (int b = 0; b < NP; ++b) s += phif[b] * z[b][i];
      for (int c = 0; c < NFN; ++c) sh += psif[c] * z[NP + f * NFN + c][i];
      v[i] = s;
      vh[i] = sh;
      for (int r = 0; r < D; ++r) {
        double t = 0.0;
        for (int b = 0; b < NP; ++b) t += T.dPhiF[((f * D + r) * NGF + gf) * NP + b] * z[b][i];
        gr[i][r] = t;
      }
      for (int fl = 0; fl < NF; ++fl) {
        double l = 0.0;
        for (int c = 0; c < NFN; ++c) l += T.PLF[((f * NF + fl) * NGF + gf) * NFN + c] * dz[fl * NFN + c][i];
        lift[i][fl] = l;
      }
    }
    lifted_q(gr, lift, q);
    bad = !(v[M - 1] < 0.0) || !(vh[M - 1] < 0.0);
    // derivatives with respect to vhat: F(vhat).n, sigma(vhat) (v - vhat), G(vhat, q).n
    Dual<M> vhd[M], dvd[M];
    for (int l = 0; l < M; ++l) {
      vhd[l] = dconst<M>(vh[l]);
      vhd[l].d[l] = 1.0;
      dvd[l] = v[l] - vhd[l];
    }
    Dual<M> rh, velh[D], prh, uh[M], Fh[M][D], duh[M];
    prim_of_v<D>(vhd, ph.gamma, rh, velh, prh);
    cons_and_flux<D>(rh, velh, prh, ph.gamma, uh, Fh);
    bad = bad || !(rh.v > 0.0) || !(prh.v > 0.0);
    du_of_v<D>(vhd, dvd, ph.gamma, duh);
    // sigma(vhat) (v - vhat) and the matrix sigma(vhat) = d(sigma (v - vhat))/dv: sigma_SLF =
    // lambda_max A0 (Eq. sLxF) or sigma_S = |A_n| A0 (Eq. symStab), as physics selects
    Dual<M> sdu[M];
    double sig[M][M];
    if (ph.stab == 1) {
      abs_flux_jac_apply<D>(rh, velh, prh, n, ph.gamma, duh, sdu);
      double vv[D];
      for (int j = 0; j < D; ++j) vv[j] = velh[j].v;
      for (int l = 0; l < M; ++l) {
        double x[M], y[M];
        for (int k = 0; k < M; ++k) x[k] = uh[k].d[l];
        abs_flux_jac_apply<D>(rh.v, vv, prh.v, n, ph.gamma, x, y);
        for (int i = 0; i < M; ++i) sig[i][l] = y[i];
      }
    } else {
      const Dual<M> lam = lambda_max<D>(rh, velh, prh, n, ph.gamma);
      for (int i = 0; i < M; ++i) {
        sdu[i] = lam * duh[i];
        for (int l = 0; l < M; ++l) sig[i][l] = lam.v * uh[i].d[l];
      }
    }
    Dual<M> hA[M];
    for (int i = 0; i < M; ++i) {
      Dual<M> s = Fh[i][0] * n[0];
      for (int j = 1; j < D; ++j) s = s + Fh[i][j] * n[j];
      hA[i] = 0.5 * s + 0.5 * sdu[i];
    }
    if (ph.gflux != 1) {  // ghat = G(vhat, q) . n (Eq. numericalFluxNS_2)
      Dual<M> Gh[M][D];
      visc_flux<D>(vhd, q, ph, Gh);
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < D; ++j) hA[i] = hA[i] + Gh[i][j] * n[j];
    }
    // derivatives with respect to v: F(v).n; the sigma term gives sigma(vhat)
    Dual<M> vd[M];
    for (int l = 0; l < M; ++l) {
      vd[l] = dconst<M>(v[l]);
      vd[l].d[l] = 1.0;
    }
    Dual<M> rv, velv[D], pv, Fv[M][D];
    prim_of_v<D>(vd, ph.gamma, rv, velv, pv);
    cons_and_flux<D>(rv, velv, pv, ph.gamma, (Dual<M>*)nullptr, Fv);
    bad = bad || !(rv.v > 0.0) || !(pv.v > 0.0);
    Dual<M> gn[M];  // ghat = G(v, q) . n (Eq. numericalFluxNS_1)
    for (int i = 0; i < M; ++i) gn[i] = vd[0] * 0.0;
    if (ph.gflux == 1) {
      Dual<M> Gv[M][D];
      visc_flux<D>(vd, q, ph, Gv);
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < D; ++j) gn[i] = gn[i] + Gv[i][j] * n[j];
    }
    double* HF = ptf + (f * NGF + gf) * PT_FACE;
    double* U0 = HF + M;
    double* U1 = U0 + M * M;
    double* U2 = U1 + M * M;
    for (int i = 0; i < M; ++i) {
      Dual<M> s = Fv[i][0] * n[0];
      for (int j = 1; j < D; ++j) s = s + Fv[i][j] * n[j];
      HF[i] = Wf * (hA[i].v + 0.5 * s.v + gn[i].v);
      for (int l = 0; l < M; ++l) {
        U0[i * M + l] = Wf * (0.5 * s.d[l] + 0.5 * sig[i][l] + gn[i].d[l]);
        U1[i * M + l] = Wf * hA[i].d[l];
      }
    }
    const double* vs = ph.gflux == 1 ? v : vh;
    const ViscFactors<D> vf = visc_factors<D>(vs);
    visc_jac_dir<D>(vf, n, visc_params_at(ph, vs[M - 1]),
                    [&](int i, int l, int k, double val) { U2[(i * M + l) * D + k] = Wf * val; });
  }
  if (bad) atomicOr(a.status + e, HDG_STATUS_NONPHYSICAL);
}

// ----------------------------------------------------------------------------------- step 3
// Quadrature contractions into A' [NV][NV], B' [NV][NT], C' [NT][NV], D' [NT][NT] and R_v, R_t
// (degree-pt trace layout); the same sums as k_assemble.
__device__ void pc_assemble(const PClassDev& T, const double* G, const double* ptv, const double* ptf,
                            const double* hist_e, double* Ap, double* Bp, double* Cp, double* Dp, double* Rv,
                            double* Rt, double* work) {
  constexpr int D = D3, M = M5, NF = NF4, NR = NR3, NRF = NRF3;
  const int NP = T.d.NP, NFN = T.d.NFN, NFK = T.d.NFK, NG = T.d.NG, NGF = T.d.NGF, NZ = T.d.NZ;
  const int NV = T.d.NV, NT = T.d.NT, GT = T.d.GT;
  double* Rb = work;
  double* Zs = work + T.d.RBMAX;
  const int tid = threadIdx.x, nth = blockDim.x;
  const double* Jinv = G;
  const double detJ = G[D * D];
  for (int t = tid; t < NV; t += nth) {  // R_v, volume part
    const int an = t / M, i = t % M;
    double s = hist_e ? -hist_e[t] : 0.0;
    for (int g = 0; g < NG; ++g) {
      const double* P = ptv + g * PT_VOL;
      s += T.Phi[g * NP + an] * P[i];
      for (int r = 0; r < D; ++r) s += T.dPhi[(r * NG + g) * NP + an] * P[M + r * M + i];
    }
    Rv[t] = s;
  }
  // volume contractions
  for (int g0 = 0; g0 < NG; g0 += GT) {
    const int ng = (NG - g0) < GT ? (NG - g0) : GT;
    __syncthreads();
    for (int t = tid; t < NR * GT * NZ; t += nth) {
      const int beta = t / (GT * NZ), gg = (t / NZ) % GT, j = t % NZ;
      double val = 0.0;
      if (gg < ng) {
        const int g = g0 + gg;
        if (beta == 0) {
          val = j < NP ? T.Phi[g * NP + j] : 0.0;
        } else {
          const int k = beta - 1;
          if (j < NP) {
            for (int r = 0; r < D; ++r) val += Jinv[r * D + k] * T.dPhi[(r * NG + g) * NP + j];
            for (int f = 0; f < NF; ++f) {
              const double* Gf = G + D * D + 1 + f * (D + 1);
              val -= Gf[k] * (Gf[D] / detJ) * T.PLV[(f * NG + g) * NP + j];
            }
          } else {
            const int f = (j - NP) / NFN, c = (j - NP) % NFN;
            const double* Gf = G + D * D + 1 + f * (D + 1);
            val = Gf[k] * (Gf[D] / detJ) * T.PL[(f * NG + g) * NFN + c];
          }
        }
      }
      Rb[t] = val;
    }
    for (int il = 0; il < M * M; ++il) {
      const int i = il / M, l = il % M;
      __syncthreads();
      for (int t = tid; t < NP * GT * NR; t += nth) {
        const int an = t / (GT * NR), gg = (t / NR) % GT, beta = t % NR;
        double val = 0.0;
        if (gg < ng) {
          const int g = g0 + gg;
          const double* P = ptv + g * PT_VOL;
          const double* T0 = P + M + D * M;
          const double* T1 = T0 + M * M;
          const double* T2 = T1 + D * M * M;
          if (beta == 0) {
            val = T.Phi[g * NP + an] * T0[i * M + l];
            for (int r = 0; r < D; ++r) val += T.dPhi[(r * NG + g) * NP + an] * T1[(r * M + i) * M + l];
          } else {
            const int k = beta - 1;
            for (int r = 0; r < D; ++r) val += T.dPhi[(r * NG + g) * NP + an] * T2[((r * M + i) * M + l) * D + k];
          }
        }
        Zs[t] = val;
      }
      __syncthreads();
      for (int t = tid; t < NP * NZ; t += nth) {
        const int an = t / NZ, j = t % NZ;
        const int b0 = j < NP ? 0 : 1;
        double acc = 0.0;
        for (int gg = 0; gg < ng; ++gg)
          for (int beta = b0; beta < NR; ++beta) acc += Zs[(an * GT + gg) * NR + beta] * Rb[(beta * GT + gg) * NZ + j];
        const int row = an * M + i;
        double* dst = j < NP ? Ap + row * NV + j * M + l : Bp + row * NT + (j - NP) * M + l;
        *dst = (g0 == 0) ? acc : *dst + acc;
      }
    }
  }
  // face contractions: test functions phi_b (b on face f: rows of A', B') and psi_c (C', D')
  const int NROW = NFK + NFN;
  for (int f = 0; f < NF; ++f) {
    __syncthreads();
    for (int t = tid; t < NRF * NGF * NZ; t += nth) {
      const int beta = t / (NGF * NZ), gf = (t / NZ) % NGF, j = t % NZ;
      double val = 0.0;
      if (beta == 0) {
        val = j < NP ? T.PhiF[(f * NGF + gf) * NP + j] : 0.0;
      } else if (beta == 1) {
        if (j >= NP && (j - NP) / NFN == f) val = T.PsiF[(f * NGF + gf) * NFN + (j - NP) % NFN];
      } else {
        const int k = beta - 2;
        if (j < NP) {
          for (int r = 0; r < D; ++r) val += Jinv[r * D + k] * T.dPhiF[((f * D + r) * NGF + gf) * NP + j];
          for (int fl = 0; fl < NF; ++fl) {
            const double* Gl = G + D * D + 1 + fl * (D + 1);
            val -= Gl[k] * (Gl[D] / detJ) * T.PLFV[((f * NF + fl) * NGF + gf) * NP + j];
          }
        } else {
          const int fl = (j - NP) / NFN, c = (j - NP) % NFN;
          const double* Gl = G + D * D + 1 + fl * (D + 1);
          val = Gl[k] * (Gl[D] / detJ) * T.PLF[((f * NF + fl) * NGF + gf) * NFN + c];
        }
      }
      Rb[t] = val;
    }
    __syncthreads();
    for (int t = tid; t < NROW * M; t += nth) {  // residuals, face part
      const int row = t / M, i = t % M;
      double s = 0.0;
      if (row < NFK) {
        const int b = T.fnodesK[f * NFK + row];
        for (int gf = 0; gf < NGF; ++gf) s += T.PhiF[(f * NGF + gf) * NP + b] * ptf[(f * NGF + gf) * PT_FACE + i];
        Rv[b * M + i] += s;
      } else {
        const int c = row - NFK;
        for (int gf = 0; gf < NGF; ++gf) s += T.PsiF[(f * NGF + gf) * NFN + c] * ptf[(f * NGF + gf) * PT_FACE + i];
        Rt[(f * NFN + c) * M + i] = s;
      }
    }
    for (int il = 0; il < M * M; ++il) {
      const int i = il / M, l = il % M;
      __syncthreads();
      for (int t = tid; t < NROW * NGF * NRF; t += nth) {
        const int row = t / (NGF * NRF), gf = (t / NRF) % NGF, beta = t % NRF;
        const double* P = ptf + (f * NGF + gf) * PT_FACE;
        const double* U0 = P + M;
        const double* U1 = U0 + M * M;
        const double* U2 = U1 + M * M;
        const double test = row < NFK ? T.PhiF[(f * NGF + gf) * NP + T.fnodesK[f * NFK + row]]
                                      : T.PsiF[(f * NGF + gf) * NFN + (row - NFK)];
        const double u = beta == 0 ? U0[i * M + l] : beta == 1 ? U1[i * M + l] : U2[(i * M + l) * D + (beta - 2)];
        Zs[t] = test * u;
      }
      __syncthreads();
      for (int t = tid; t < NROW * NZ; t += nth) {
        const int row = t / NZ, j = t % NZ;
        double acc = 0.0;
        for (int gf = 0; gf < NGF; ++gf)
          for (int beta = 0; beta < NRF; ++beta) acc += Zs[(row * NGF + gf) * NRF + beta] * Rb[(beta * NGF + gf) * NZ + j];
        if (row < NFK) {
          const int rv = T.fnodesK[f * NFK + row] * M + i;
          if (j < NP)
            Ap[rv * NV + j * M + l] += acc;
          else
            Bp[rv * NT + (j - NP) * M + l] += acc;
        } else {
          const int rt = (f * NFN + (row - NFK)) * M + i;
          if (j < NP)
            Cp[rt * NV + j * M + l] = acc;
          else
            Dp[rt * NT + (j - NP) * M + l] = acc;
        }
      }
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------------- step 4
// Degree-pt local trace index (f, c, i) and the element's own one (f, c', i): P maps the second to
// the first, P[(f,c,i)][(f,c',i)] = I_f[c][c'] (identity when q_f = pt).
struct ProjMap {
  int nfn;
  int qoff[NF4 + 1];  // first own-space unknown of face f
  int nq[NF4];        // own-space nodes of face f
  const double* I[NF4];
  HDG_DEVI double p(int f, int c, int cq) const { return I[f] ? I[f][c * nfn + cq] : (c == cq ? 1.0 : 0.0); }
  HDG_DEVI void own(int tq, int& f, int& cq, int& i) const {
    f = 0;
    while (tq >= qoff[f + 1]) ++f;
    cq = (tq - qoff[f]) / M5;
    i = (tq - qoff[f]) % M5;
  }
};

// ----------------------------------------------------------------------------------- step 5
// LU with partial pivoting of the NV x NV matrix LU (shared or global memory), row interchanges in
// piv; a zero pivot sets the element's SINGULAR bit.
__device__ void pc_factor(double* LU, int NV, int* piv, int* s_misc, int64_t e, const PArgs& a) {
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tid == 0) s_misc[1] = 0;
  __syncthreads();
  for (int k = 0; k < NV; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int r = k + tid; r < NV; r += 32) {
        const double v = fabs(LU[r * NV + k]);
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
      if (tid == 0) {
        s_misc[0] = bi;
        piv[k] = bi;
        if (!(best > 0.0)) s_misc[1] = 1;
      }
    }
    __syncthreads();
    const int pr = s_misc[0];
    if (pr != k)
      for (int j = tid; j < NV; j += nth) {
        const double t = LU[k * NV + j];
        LU[k * NV + j] = LU[pr * NV + j];
        LU[pr * NV + j] = t;
      }
    __syncthreads();
    const double d = LU[k * NV + k];
    const double inv = d != 0.0 ? 1.0 / d : 0.0;
    for (int r = k + 1 + tid; r < NV; r += nth) LU[r * NV + k] *= inv;
    __syncthreads();
    const int rem = NV - k - 1;
    for (int t = tid; t < rem * rem; t += nth) {
      const int r = k + 1 + t / rem, c = k + 1 + t % rem;
      LU[r * NV + c] -= LU[r * NV + k] * LU[k * NV + c];
    }
    __syncthreads();
  }
  if (tid == 0 && s_misc[1]) atomicOr(a.status + e, HDG_STATUS_SINGULAR);
}

// X = A'^{-1} [B_q | R_v] in place (B_q in X, row stride nt), y = A'^{-1} R_v.
__device__ void pc_solve(const double* LU, int NV, int CB, const int* piv, double* Xs, double* X, double* y,
                         const double* Rv, int nt) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int c0 = 0; c0 < nt + 1; c0 += CB) {
    const int nc = (nt + 1 - c0) < CB ? (nt + 1 - c0) : CB;
    __syncthreads();
    for (int t = tid; t < NV * CB; t += nth) {
      const int r = t / CB, c = t % CB, col = c0 + c;
      Xs[t] = c < nc ? (col < nt ? X[r * nt + col] : Rv[r]) : 0.0;
    }
    __syncthreads();
    for (int t = tid; t < CB; t += nth)
      for (int k = 0; k < NV; ++k) {
        const int p = piv[k];
        if (p != k) {
          const double tmp = Xs[k * CB + t];
          Xs[k * CB + t] = Xs[p * CB + t];
          Xs[p * CB + t] = tmp;
        }
      }
    __syncthreads();
    for (int k = 0; k < NV; ++k) {
      for (int t = tid; t < (NV - k - 1) * CB; t += nth) {
        const int r = k + 1 + t / CB, c = t % CB;
        Xs[r * CB + c] -= LU[r * NV + k] * Xs[k * CB + c];
      }
      __syncthreads();
    }
    for (int k = NV - 1; k >= 0; --k) {
      for (int c = tid; c < CB; c += nth) Xs[k * CB + c] /= LU[k * NV + k];
      __syncthreads();
      for (int t = tid; t < k * CB; t += nth) {
        const int r = t / CB, c = t % CB;
        Xs[r * CB + c] -= LU[r * NV + k] * Xs[k * CB + c];
      }
      __syncthreads();
    }
    for (int t = tid; t < NV * CB; t += nth) {
      const int r = t / CB, c = t % CB, col = c0 + c;
      if (c < nc) {
        if (col < nt)
          X[r * nt + col] = Xs[t];
        else
          y[r] = Xs[t];
      }
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------------- one element
__device__ void pc_element(const PArgs& a, const PClassDev& T, const PhysParams& ph, int64_t e, double* sm,
                           double* slot) {
  constexpr int M = M5, NF = NF4;
  const int NP = T.d.NP, NFN = T.d.NFN, NV = T.d.NV, NT = T.d.NT, NZ = T.d.NZ;
  const int tid = threadIdx.x, nth = blockDim.x;
  double(*z)[M] = reinterpret_cast<double(*)[M]>(sm);
  double* G = sm + NZ * M;
  double(*dz)[M] = reinterpret_cast<double(*)[M]>(G + GEO3);
  double* Rv = G + GEO3 + NF * NFN * M;
  double* Rt = Rv + NV;
  double* work = Rt + NT;
  int* piv = reinterpret_cast<int*>(work + (T.d.ASM > T.d.CND ? T.d.ASM : T.d.CND));
  int* s_misc = piv + NV + 1;
  double* ptv = slot;
  double* ptf = ptv + (int64_t)T.d.NG * PT_VOL;
  double* Ap = ptf + (int64_t)NF * T.d.NGF * PT_FACE;
  double* Bp = Ap + (int64_t)NV * NV;
  double* Cp = Bp + (int64_t)NV * NT;
  double* Dp = Cp + (int64_t)NT * NV;
  double* T1 = Dp + (int64_t)NT * NT;
  double* Cq = T1 + (int64_t)NT * NT;
  ProjMap P;
  P.nfn = NFN;
  P.qoff[0] = 0;
  for (int f = 0; f < NF; ++f) {
    const int q = a.fdeg[e * NF + f];
    P.nq[f] = nfn3(q);
    P.I[f] = q == T.d.pt ? nullptr : T.IPro + ((size_t)(q - 1) * NF + f) * NFN * NFN;
    P.qoff[f + 1] = P.qoff[f] + P.nq[f] * M;
  }
  const int ntq = P.qoff[NF];
  // 1. element state; the trace at the degree-pt nodes
  const double* Ve = a.V + a.voff[e];
  for (int t = tid; t < NP * M; t += nth) z[t / M][t % M] = Ve[t];
  for (int t = tid; t < NF * NFN * M; t += nth) {
    const int f = t / (NFN * M), c = (t / M) % NFN, i = t % M;
    const int* tg = a.tgidx + (e * NF + f) * a.nfn_max;
    double val;
    if (!P.I[f]) {
      val = a.Vhat[(int64_t)tg[c] * M + i];
    } else {
      val = 0.0;
      for (int cq = 0; cq < P.nq[f]; ++cq) val += P.I[f][c * NFN + cq] * a.Vhat[(int64_t)tg[cq] * M + i];
    }
    z[NP + f * NFN + c][i] = val;
  }
  for (int t = tid; t < GEO3; t += nth) G[t] = a.geo[e * GEO3 + t];
  __syncthreads();
  for (int t = tid; t < NF * NFN * M; t += nth) {
    const int fc = t / M, i = t % M;
    double s = 0.0;
    for (int b = 0; b < NP; ++b) s += T.PhiN[fc * NP + b] * z[b][i];
    dz[fc][i] = z[NP + fc][i] - s;
  }
  __syncthreads();
  // 2. pointwise
  pc_pointwise(a, T, ph, z, dz, G, ptv, ptf, e);
  __syncthreads();
  // 3. contractions
  pc_assemble(T, G, ptv, ptf, a.hist ? a.hist + a.voff[e] : nullptr, Ap, Bp, Cp, Dp, Rv, Rt, work);
  // 4. the element's own trace space: B_q (into X), D_q (into S), C_q, R_t,q
  double* X = a.recov + a.roff[e];
  double* y = X + (int64_t)NV * ntq;
  double* S = a.S + a.soff[e];
  double* Re = a.R + a.Roff[e];
  double* ge = a.g + a.toff[e];
  for (int t = tid; t < NV * ntq; t += nth) {  // B_q = B' P
    const int r = t / ntq, tq = t % ntq;
    int f, cq, i;
    P.own(tq, f, cq, i);
    double s = 0.0;
    for (int c = 0; c < NFN; ++c) s += Bp[r * NT + (f * NFN + c) * M + i] * P.p(f, c, cq);
    X[t] = s;
  }
  for (int t = tid; t < ntq * NV; t += nth) {  // C_q = P^T C'
    const int tq = t / NV, col = t % NV;
    int f, cq, i;
    P.own(tq, f, cq, i);
    double s = 0.0;
    for (int c = 0; c < NFN; ++c) s += P.p(f, c, cq) * Cp[((f * NFN + c) * M + i) * NV + col];
    Cq[t] = s;
  }
  for (int t = tid; t < NT * ntq; t += nth) {  // T1 = D' P
    const int r = t / ntq, uq = t % ntq;
    int f, dq, l;
    P.own(uq, f, dq, l);
    double s = 0.0;
    for (int d = 0; d < NFN; ++d) s += Dp[r * NT + (f * NFN + d) * M + l] * P.p(f, d, dq);
    T1[t] = s;
  }
  for (int t = tid; t < NV; t += nth) Re[t] = Rv[t];
  for (int t = tid; t < ntq; t += nth) {  // R_t,q = P^T R_t
    int f, cq, i;
    P.own(t, f, cq, i);
    double s = 0.0;
    for (int c = 0; c < NFN; ++c) s += P.p(f, c, cq) * Rt[(f * NFN + c) * M + i];
    Re[NV + t] = s;
  }
  __syncthreads();
  for (int t = tid; t < ntq * ntq; t += nth) {  // D_q = P^T T1
    const int tq = t / ntq, uq = t % ntq;
    int f, cq, i;
    P.own(tq, f, cq, i);
    double s = 0.0;
    for (int c = 0; c < NFN; ++c) s += P.p(f, c, cq) * T1[((f * NFN + c) * M + i) * ntq + uq];
    S[t] = s;
  }
  // 5. factorisation and condensation
  double* LU = T.d.lu_smem ? work : Ap;
  double* Xs = T.d.lu_smem ? work + NV * NV : work;
  if (T.d.lu_smem)
    for (int t = tid; t < NV * NV; t += nth) LU[t] = Ap[t];
  __syncthreads();
  pc_factor(LU, NV, piv, s_misc, e, a);
  pc_solve(LU, NV, T.d.CB, piv, Xs, X, y, Re, ntq);
  for (int t = tid; t < ntq * ntq; t += nth) {  // S = D_q - C_q X
    const int r = t / ntq, c = t % ntq;
    double s = S[t];
    const double* Cr = Cq + r * NV;
    for (int k = 0; k < NV; ++k) s -= Cr[k] * X[k * ntq + c];
    S[t] = s;
  }
  for (int r = tid; r < ntq; r += nth) {  // g = R_t,q - C_q y
    double s = Re[NV + r];
    const double* Cr = Cq + r * NV;
    for (int k = 0; k < NV; ++k) s -= Cr[k] * y[k];
    ge[r] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1) k_pclass_fused(PArgs a, PhysParams ph) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_idx;
  double* slot = a.scratch + (int64_t)blockIdx.x * a.slot_doubles;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(a.counter, 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= a.E) break;
    const int64_t e = a.queue[idx];
    pc_element(a, a.tab[a.cls[e]], ph, e, sm, slot);
  }
}

}  // namespace

int pclass_index(int pk, int pt) {
  if (pk < 1 || pt < pk || pt > 4) return -1;
  static const int base[5] = {0, 0, 4, 7, 9};
  return base[pk] + (pt - pk);
}


namespace {


// One launch of the fused kernel over `count` queue entries starting at `queue`.
int launch_fused(hdg_ctx* c, const PArgs& base, const int* queue, int64_t count, cudaStream_t s) {
  PMix& pm = *c->pm;
  PArgs a = base;
  a.queue = queue;
  a.E = count;
  for (int k = 0; k < kPClasses; ++k) a.tab[k] = pm.tab[k];
  HDG_CK(cudaMemsetAsync(pm.d_counter, 0, sizeof(int), s));
  const int grid = c->num_sms > 0 ? c->num_sms : 152;
  k_pclass_fused<<<grid, kThreads, pm.smem_bytes, s>>>(a, c->ph);
  HDG_CK(cudaGetLastError());
  return HDG_OK;
}

// Tile shapes per class: for every class present, every (GT, CB) in {16, 32, 64}^2 that fits the
// shared memory is timed on up to two waves of that class's elements (CUDA events, one warm-up
// launch each) and the fastest kept. The sample writes its elements' outputs, which the full
// launch that follows writes again.
int pclass_autotune(hdg_ctx* c, const PArgs& base, cudaStream_t s) {
  PMix& pm = *c->pm;
  const int grid = c->num_sms > 0 ? c->num_sms : 152;
  int* d_sample = nullptr;
  HDG_CK(cudaMalloc(&d_sample, sizeof(int) * 2 * grid));
  cudaEvent_t ev0, ev1;
  HDG_CK(cudaEventCreate(&ev0));
  HDG_CK(cudaEventCreate(&ev1));
  int rc = HDG_OK;
  const int cand[3] = {16, 32, 64};
  for (int k = 0; k < kPClasses && rc == HDG_OK; ++k) {
    if (pm.class_count[k] == 0) continue;
    std::vector<int> sample;
    for (int e : pm.h_queue)
      if (pm.h_cls[e] == k && (int)sample.size() < 2 * grid) sample.push_back(e);
    if (cudaMemcpyAsync(d_sample, sample.data(), sizeof(int) * sample.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "pclass_autotune: sample upload");
      break;
    }
    const PDims keep = pm.tab[k].d;
    PDims best = keep;
    float best_ms = -1.0f;
    for (int gt : cand)
      for (int cb : cand) {
        const PDims d = pclass_dims(keep.pk, keep.pt, gt, cb);
        if (sizeof(double) * (size_t)d.SMEM > pm.smem_limit) continue;
        if (gt > cand[0] && keep.NG <= gt / 2) continue;  // the smaller tile already held every point
        pm.tab[k].d = d;
        const size_t smem_keep = pm.smem_bytes;
        pm.smem_bytes = std::max(pm.smem_bytes, sizeof(double) * (size_t)d.SMEM);
        float ms = 0.0f;
        if ((rc = launch_fused(c, base, d_sample, (int64_t)sample.size(), s)) ||
            (rc = cudaEventRecord(ev0, s) == cudaSuccess ? HDG_OK : HDG_ERR_CUDA) ||
            (rc = launch_fused(c, base, d_sample, (int64_t)sample.size(), s)) ||
            (rc = cudaEventRecord(ev1, s) == cudaSuccess ? HDG_OK : HDG_ERR_CUDA) ||
            (rc = cudaEventSynchronize(ev1) == cudaSuccess ? HDG_OK : HDG_ERR_CUDA) ||
            (rc = cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess ? HDG_OK : HDG_ERR_CUDA)) {
          pm.smem_bytes = smem_keep;
          break;
        }
        pm.smem_bytes = smem_keep;
        if (best_ms < 0.0f || ms < best_ms) {
          best_ms = ms;
          best = d;
        }
      }
    pm.tab[k].d = best;
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaFree(d_sample);
  if (rc) return rc == HDG_ERR_CUDA ? cuda_fail(cudaGetLastError(), "pclass_autotune") : rc;
  pm.smem_bytes = 0;
  pm.slot_doubles = 0;
  for (int k = 0; k < kPClasses; ++k)
    if (pm.class_count[k] > 0) {
      pm.smem_bytes = std::max(pm.smem_bytes, sizeof(double) * (size_t)pm.tab[k].d.SMEM);
      pm.slot_doubles = std::max(pm.slot_doubles, pm.tab[k].d.SLOT);
    }
  pm.tuned = true;
  return HDG_OK;
}

}  // namespace

int assemble_condense_pclass(hdg_ctx* c, const double* V, const double* Vhat, const double* hist, double mass_coef,
                             double* S, double* g, double* recov, double* R, int32_t* status, cudaStream_t s) {
  PMix& pm = *c->pm;
  const int grid = c->num_sms > 0 ? c->num_sms : 152;
  const size_t need = sizeof(double) * (size_t)grid * pm.slot_doubles;
  if (c->scr_bytes < need) {
    if (c->d_scr) cudaFree(c->d_scr);
    c->d_scr = nullptr;
    c->scr_bytes = 0;
    HDG_CK(cudaMalloc(&c->d_scr, need));
    c->scr_bytes = need;
  }
  if (!pm.attr_set) {  // per context, hence per device: all the dynamic shared memory a CTA may have
    int optin = 0;
    cudaFuncAttributes fa{};
    HDG_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    HDG_CK(cudaFuncGetAttributes(&fa, k_pclass_fused));
    pm.smem_limit = (size_t)optin - fa.sharedSizeBytes;
    if (pm.smem_bytes > pm.smem_limit) {
      set_error("assemble_condense: the element classes need more shared memory than the device has");
      return HDG_ERR_UNSUPPORTED;
    }
    HDG_CK(cudaFuncSetAttribute(k_pclass_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pm.smem_limit));
    pm.attr_set = true;
  }
  PArgs a{};
  a.V = V;
  a.Vhat = Vhat;
  a.hist = hist;
  a.mass_coef = mass_coef;
  a.voff = pm.d_voff;
  a.toff = pm.d_toff;
  a.soff = pm.d_soff;
  a.roff = pm.d_roff;
  a.Roff = pm.d_Roff;
  a.tgidx = pm.d_tgidx;
  a.fdeg = pm.d_fdeg;
  a.cls = pm.d_cls;
  a.geo = c->d_geo;
  a.queue = pm.d_queue;
  a.E = c->E;
  a.nfn_max = pm.nfn_max;
  a.slot_doubles = pm.slot_doubles;
  a.counter = pm.d_counter;
  a.scratch = c->d_scr;
  a.S = S;
  a.g = g;
  a.recov = recov;
  a.R = R;
  a.status = status;
  if (!pm.tuned && c->E >= 4 * (int64_t)grid) {
    if (int rc = pclass_autotune(c, a, s)) return rc;
  }
  LaunchScope ls(c, HDG_KERNEL_PCLASS, s);
  return launch_fused(c, a, pm.d_queue, c->E, s);
}

namespace {

template <class T>
int up(T** dst, const std::vector<T>& src) {
  HDG_CK(cudaMalloc(dst, sizeof(T) * std::max<size_t>(1, src.size())));
  if (!src.empty()) HDG_CK(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return HDG_OK;
}

}  // namespace

int pclass_setup(hdg_ctx* c) {
  const Mesh& m = c->mesh->m;
  if (m.dim != 3 || !c->visc) {
    set_error("hdg_ctx_create: mixed-degree meshes are built for 3D Navier-Stokes");
    return HDG_ERR_UNSUPPORTED;
  }
  auto* pm = new PMix();
  c->pm = pm;
  const int NF = c->NF;
  const int64_t E = c->E;
  pm->pmin = 99;
  for (int8_t q : m.pe) {
    pm->pmin = std::min<int>(pm->pmin, q);
    pm->pmax = std::max<int>(pm->pmax, q);
  }
  pm->nfn_max = m.ref.Nf;
  pm->n_tnodes = m.fnoff.back();
  // class tables, one buffer
  std::vector<double> tab;
  std::vector<int> itab;
  size_t off[kPClasses][13], ioff[kPClasses];
  bool have[kPClasses] = {};
  for (int pk = 1; pk <= 4; ++pk)
    for (int pt = pk; pt <= 4; ++pt) {
      const int k = pclass_index(pk, pt);
      if (pt > pm->pmax || pk < pm->pmin) continue;
      const ClassTables T = make_class_tables(3, pk, pt);
      const std::vector<double>* parts[13] = {&T.W,  &T.Phi, &T.dPhi, &T.WF,  &T.PhiF, &T.dPhiF, &T.PsiF,
                                              &T.PhiN, &T.PL, &T.PLF,  &T.PLV, &T.PLFV, &T.IPro};
      for (int i = 0; i < 13; ++i) {
        off[k][i] = tab.size();
        tab.insert(tab.end(), parts[i]->begin(), parts[i]->end());
      }
      ioff[k] = itab.size();
      itab.insert(itab.end(), T.fnodesK.begin(), T.fnodesK.end());
      have[k] = true;
      pm->tab[k].d = pclass_dims(pk, pt);
    }
  // classes and trace map
  auto nfn = [](int q) { return (q + 1) * (q + 2) / 2; };
  std::vector<int8_t> fdeg(E * NF), cls(E);
  std::vector<int> tg(E * NF * pm->nfn_max, -1);
  for (int64_t e = 0; e < E; ++e) {
    for (int f = 0; f < NF; ++f) {
      const int64_t F = m.face_of[e * NF + f];
      const int q = m.fdeg[F];
      fdeg[e * NF + f] = (int8_t)q;
      for (int cc = 0; cc < nfn(q); ++cc)
        tg[(e * NF + f) * pm->nfn_max + cc] = (int)(m.fnoff[F] + m.fnode_mix[(e * NF + f) * pm->nfn_max + cc]);
    }
    cls[e] = (int8_t)pclass_index(m.pe[e], m.ptr[e]);
    pm->class_count[cls[e]]++;
  }
  // trace addressing: own face-node counts, the two local occurrences of every trace node,
  // face-block offsets
  std::vector<int> fnn(E * NF), occ_e(2 * m.fnoff.back(), -1), occ_l(2 * m.fnoff.back(), -1);
  std::vector<int64_t> pcoff(c->F + 1, 0);
  for (int64_t e = 0; e < E; ++e) {
    int qoff = 0;
    for (int f = 0; f < NF; ++f) {
      const int64_t F = m.face_of[e * NF + f];
      const int nq = nfn(m.fdeg[F]);
      fnn[e * NF + f] = nq;
      const int side = m.face_side[2 * F] == (int32_t)(e * NF + f) ? 0 : 1;
      for (int cl = 0; cl < nq; ++cl) {
        const int64_t t = m.fnoff[F] + m.fnode_mix[(e * NF + f) * pm->nfn_max + cl];
        occ_e[2 * t + side] = (int)e;
        occ_l[2 * t + side] = qoff + cl * 5;
      }
      qoff += nq * 5;
    }
    pm->nt_max = std::max(pm->nt_max, qoff);
  }
  for (int64_t F = 0; F < c->F; ++F) {
    const int64_t B = (m.fnoff[F + 1] - m.fnoff[F]) * 5;
    pcoff[F + 1] = pcoff[F] + B * B;
  }
  pm->pc_len = pcoff.back();
  // queue: largest class first (interior size, then trace degree), element order within a class
  std::vector<int> queue(E);
  for (int64_t e = 0; e < E; ++e) queue[e] = (int)e;
  std::stable_sort(queue.begin(), queue.end(), [&](int x, int y) {
    const int kx = m.pe[x] * 8 + m.ptr[x], ky = m.pe[y] * 8 + m.ptr[y];
    return kx > ky;
  });
  pm->h_queue = queue;
  pm->h_cls = cls;
  int rc = HDG_OK;
  if ((rc = up(&pm->d_tab, tab)) || (rc = up(&pm->d_itab, itab)) || (rc = up(&pm->d_voff, m.voff)) ||
      (rc = up(&pm->d_toff, m.toff)) || (rc = up(&pm->d_soff, m.soff)) || (rc = up(&pm->d_roff, m.roff)) ||
      (rc = up(&pm->d_Roff, m.Roff)) || (rc = up(&pm->d_tgidx, tg)) || (rc = up(&pm->d_fdeg, fdeg)) ||
      (rc = up(&pm->d_cls, cls)) || (rc = up(&pm->d_queue, queue)) || (rc = up(&pm->d_fnn, fnn)) ||
      (rc = up(&pm->d_occ_e, occ_e)) || (rc = up(&pm->d_occ_l, occ_l)) || (rc = up(&pm->d_fnoff, m.fnoff)) ||
      (rc = up(&pm->d_pcoff, pcoff)))
    return rc;
  HDG_CK(cudaMalloc(&pm->d_counter, sizeof(int)));
  for (int k = 0; k < kPClasses; ++k) {
    if (!have[k]) continue;
    const double* b = pm->d_tab;
    PClassDev& d = pm->tab[k];
    d.W = b + off[k][0];
    d.Phi = b + off[k][1];
    d.dPhi = b + off[k][2];
    d.WF = b + off[k][3];
    d.PhiF = b + off[k][4];
    d.dPhiF = b + off[k][5];
    d.PsiF = b + off[k][6];
    d.PhiN = b + off[k][7];
    d.PL = b + off[k][8];
    d.PLF = b + off[k][9];
    d.PLV = b + off[k][10];
    d.PLFV = b + off[k][11];
    d.IPro = b + off[k][12];
    d.fnodesK = pm->d_itab + ioff[k];
  }
  for (int k = 0; k < kPClasses; ++k)
    if (pm->class_count[k] > 0) {
      pm->smem_bytes = std::max(pm->smem_bytes, sizeof(double) * (size_t)pm->tab[k].d.SMEM);
      pm->slot_doubles = std::max(pm->slot_doubles, pm->tab[k].d.SLOT);
    }
  if (!c->num_sms) HDG_CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  return HDG_OK;
}

void pclass_free(PMix* pm) {
  if (!pm) return;
  void* bufs[] = {pm->d_voff, pm->d_toff,  pm->d_soff,    pm->d_roff, pm->d_Roff,  pm->d_tgidx,
                  pm->d_fdeg, pm->d_cls,   pm->d_queue,   pm->d_counter, pm->d_tab, pm->d_itab,
                  pm->d_fnn,  pm->d_occ_e, pm->d_occ_l,   pm->d_fnoff, pm->d_pcoff};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete pm;
}

}  // namespace hdg
