// Plain FP64 assemble + condense (the reference GPU form of the hot path).
//
// Per element K the Newton linearisation of the local equations (Eq. hDG_NS1 / hDG1,
// with q eliminated exactly through Eq. hDG_NS0, which is linear in (q, v, vhat)) and
// of the element's share of the trace equation (Eq. hDG_NS2 / hDG2) is assembled as
//   A' = dR_v/dV, B' = dR_v/dVhat, C' = dR_t/dV, D' = dR_t/dVhat
// and condensed: X = A'^{-1} B', y = A'^{-1} R_v, S = D' - C' X, g = R_t - C' y.
// This equals the block elimination of the full [q; v] interior system in the order
// q first (the q-q block is the element mass matrix times the identity).
//
// Unknowns are grouped per state component into NZ "nodal" values z = [V (NP); Vhat
// (NF x NFN)]. At each quadrature point the value of v is Phi z and the lifted
// gradient is q_k = R_k z with
//   R_k(g, b)     = sum_r Jinv[r][k] dPhi_r(g, b) - sum_{f: b on f} n_fk s_f PL_f(g, c_f(b))
//   R_k(g, (f,c)) = n_fk s_f PL_f(g, c),  s_f = |F| / |K| (face / element Jacobians),
// PL_f = Phi Mref^{-1} E_f the lift of face f. Three kernels per chunk of elements:
//   k_pointwise  one thread per quadrature point: fluxes and exact pointwise Jacobians
//                by forward-mode dual numbers, pre-contracted with weights and Jinv;
//   k_assemble   one CTA per element: quadrature contractions into A', B', C', D', R;
//   k_condense   one CTA per element: LU with partial pivoting of A' in shared memory,
//                triangular solves for X and y, Schur products for S and g.
#pragma once
#include "dfloat.cuh"
#include "hdg_device.cuh"

namespace hdg {

struct AssembleArgs {
  const double* V;      // [E][NP][M]
  const double* Vhat;   // [F][NFN][M]
  const int* tgidx;     // [E][NF][NFN] global face-node index
  const double* geo;    // [E][GEO]
  const double* hist;   // [E][NP][M] or null
  double mass_coef;
  int64_t e0, ne;       // element chunk
  // scratch (chunk-local)
  double* ptv;          // [ne][NG][PT_VOL]
  double* ptf;          // [ne][NF][NGF][PT_FACE]
  double* Ap;           // [ne][NV][NV]
  double* Cp;           // [ne][NT][NV]
  uint4* oz;            // [ne][...] exact-slice operands of the mixed condensation
  float* prep;          // [ne][...] inverse, FP32 copy and scales for the mixed condensation
  uint2* rb;            // [ne][...] operator slices of the mixed assembly
  // outputs (global element index)
  double* S;            // [E][NT][NT]   (D' on entry to condense)
  double* g;            // [E][NT]
  double* recov;        // [E][NV*NT + NV]  X then y (B' on entry to condense)
  double* R;            // [E][NV + NT] raw residuals R_v, R_t (always written)
  int* status;          // [E]
  // With only_flag != 0 a CTA whose element has none of these status bits returns at once:
  // the FP64 kernels then recompute just the blocks the mixed form flagged, and k_condense
  // replaces the flag by HDG_STATUS_FP64 (the block is now the FP64 form's).
  int only_flag;
  float refine_tol;     // mixed condensation: tolerance of the refinement status bit
  int stall_first_copy; // test hook of k_condense_t5: its first operand copy is never issued
};

enum { HDG_STATUS_NONPHYSICAL = 1, HDG_STATUS_SINGULAR = 2, HDG_STATUS_REFINE = 4, HDG_STATUS_FP64 = 8,
       HDG_STATUS_TIMEOUT = 16 };

// true if the CTA of element e has nothing to do in a flagged-only pass
HDG_DEVI bool skip_element(const AssembleArgs& a, int64_t e) {
  return a.only_flag != 0 && (__ldg(a.status + e) & a.only_flag) == 0;
}

template <class C>
HDG_DEVI void load_element(const AssembleArgs& a, int64_t e, double (*z)[C::M], double* G) {
  constexpr int M = C::M;
  for (int t = threadIdx.x; t < C::NP * M; t += blockDim.x) z[t / M][t % M] = a.V[e * C::NV + t];
  for (int t = threadIdx.x; t < C::NF * C::NFN * M; t += blockDim.x) {
    int fc = t / M, i = t % M;
    int gi = a.tgidx[e * (C::NF * C::NFN) + fc];
    z[C::NP + fc][i] = a.Vhat[(int64_t)gi * M + i];
  }
  for (int t = threadIdx.x; t < C::GEO; t += blockDim.x) G[t] = a.geo[e * C::GEO + t];
}

// v_h and, for Navier-Stokes, the gradient q_h of Eq. hDG_NS0 solved element by element (the
// gradient of v_h plus the lifting of the face jumps vhat - v) at volume quadrature point g of the
// element staged in shared memory (z: nodal values, dz: jumps at the face nodes, G: geometry).
template <class C>
HDG_DEVI void volume_point_state(int g, const DevTables& T, const double (*z)[C::M], const double (*dz)[C::M],
                                 const double* G, double* v, double (*q)[C::D]) {
  constexpr int D = C::D, M = C::M, NP = C::NP, NFN = C::NFN, NF = C::NF, NG = C::NG;
  const double* Jinv = G;
  const double detJ = G[D * D];
  for (int i = 0; i < M; ++i) {
    double s = 0.0;
    for (int b = 0; b < NP; ++b) s += T.Phi[g * NP + b] * z[b][i];
    v[i] = s;
  }
  if (C::VISC) {
    for (int i = 0; i < M; ++i) {
      double gr[D], lift[NF];
      for (int r = 0; r < D; ++r) {
        double s = 0.0;
        for (int b = 0; b < NP; ++b) s += T.dPhi[(r * NG + g) * NP + b] * z[b][i];
        gr[r] = s;
      }
      for (int f = 0; f < NF; ++f) {  // the same for every direction k
        double l = 0.0;
        for (int c = 0; c < NFN; ++c) l += T.PL[(f * NG + g) * NFN + c] * dz[f * NFN + c][i];
        lift[f] = l;
      }
      for (int k = 0; k < D; ++k) {
        double s = 0.0;
        for (int r = 0; r < D; ++r) s += Jinv[r * D + k] * gr[r];
        for (int f = 0; f < NF; ++f) {
          const double* Gf = G + D * D + 1 + f * (D + 1);
          s += Gf[k] * (Gf[D] / detJ) * lift[f];
        }
        q[i][k] = s;
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// k_pointwise
// ------------------------------------------------------------------------------------
HDG_DEVI void put(double* p, int i, double v) { p[i] = v; }
HDG_DEVI void put(df2* p, int i, double v) { p[i] = df_from(v); }

// The values of sigma(vhat) = d(sigma (v - vhat))/dv at one face point, [row][column]:
// lambda_max A0 (Eq. sLxF) from the wave speed and u(vhat)'s derivatives, or |A_n| A0 (Eq. symStab)
// as a table.
template <int M, bool SYM>
struct SigmaValues {
  double lam;
  const Dual<M>* uh;
  HDG_DEVI double operator()(int i, int l) const { return lam * uh[i].d[l]; }
};
template <int M>
struct SigmaValues<M, true> {
  double s[M][M];
  HDG_DEVI double operator()(int i, int l) const { return s[i][l]; }
};

// OutT = double (FP64 form) or df2 (mixed form: per-point tensors as double-floats);
// SYM: sigma_S of Eq. symStab instead of sigma_SLF (launch through launch_pointwise).
template <class C, class OutT = double, bool SYM = false>
__global__ void __launch_bounds__(128) k_pointwise(AssembleArgs a, DevTables T, PhysParams ph) {
  constexpr int D = C::D, M = C::M, NP = C::NP, NFN = C::NFN, NF = C::NF, NG = C::NG, NGF = C::NGF;
  __shared__ double z[C::NZ][M];
  __shared__ double G[C::GEO];
  __shared__ double dz[NF * NFN][M];  // vhat - v at the face nodes (the lifting's jumps)
  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  if (skip_element(a, e)) return;
  load_element<C>(a, e, z, G);
  __syncthreads();
  if (C::VISC)
    for (int t = threadIdx.x; t < NF * NFN * M; t += blockDim.x) {
      const int fc = t / M, i = t % M;
      dz[fc][i] = z[NP + fc][i] - z[T.fnodes[fc]][i];
    }
  __syncthreads();
  const double* Jinv = G;
  const double detJ = G[D * D];
  const int tid = threadIdx.x;
  bool bad = false;
  if (tid < NG) {
    const int g = tid;
    const double W = T.W[g] * detJ;
    double v[M];
    double q[M][D];
    volume_point_state<C>(g, T, z, dz, G, v, q);
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
    if (C::VISC) {
      Dual<M> Gv[M][D];
      visc_flux<D>(vd, q, ph, Gv);
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < D; ++j) F[i][j] = F[i][j] + Gv[i][j];
    }
    OutT* out = reinterpret_cast<OutT*>(a.ptv) + (le * NG + g) * C::PT_VOL;
    OutT* MU = out;
    OutT* FR = MU + M;
    OutT* T0 = FR + D * M;
    OutT* T1 = T0 + M * M;
    OutT* T2 = T1 + D * M * M;
    for (int i = 0; i < M; ++i) {
      put(MU, i, W * a.mass_coef * u[i].v);
      for (int l = 0; l < M; ++l) put(T0, i * M + l, W * a.mass_coef * u[i].d[l]);
    }
    for (int r = 0; r < D; ++r)
      for (int i = 0; i < M; ++i) {
        double s = 0.0;
        for (int j = 0; j < D; ++j) s += Jinv[r * D + j] * F[i][j].v;
        put(FR, r * M + i, -W * s);
        for (int l = 0; l < M; ++l) {
          double t = 0.0;
          for (int j = 0; j < D; ++j) t += Jinv[r * D + j] * F[i][j].d[l];
          put(T1, (r * M + i) * M + l, -W * t);
        }
      }
    if (C::VISC) {
      // dG/dq contracted with the rows of Jinv (G is linear in q)
      const ViscFactors<D> vf = visc_factors<D>(v);
      const PhysParams pv = visc_params_at(ph, v[M - 1]);
#pragma unroll 1
      for (int r = 0; r < D; ++r)
        visc_jac_dir<D>(vf, Jinv + r * D, pv, [&](int i, int l, int k, double val) {
          put(T2, ((r * M + i) * M + l) * D + k, -W * val);
        });
    }
  } else if (tid < NG + NF * NGF) {
    const int f = (tid - NG) / NGF;
    const int gf = (tid - NG) % NGF;
    const double* Gf = G + D * D + 1 + f * (D + 1);
    const double* n = Gf;
    const double Wf = T.WF[gf] * Gf[D];
    const double* phif = T.PhiF + (f * NGF + gf) * NP;
    double v[M], vh[M];
    for (int i = 0; i < M; ++i) {
      double s = 0.0, sh = 0.0;
      for (int b = 0; b < NP; ++b) s += phif[b] * z[b][i];
      for (int c = 0; c < NFN; ++c) sh += phif[T.fnodes[f * NFN + c]] * z[NP + f * NFN + c][i];
      v[i] = s;
      vh[i] = sh;
    }
    double q[M][D];
    if (C::VISC) {
      for (int i = 0; i < M; ++i) {
        double gr[D], lift[NF];
        for (int r = 0; r < D; ++r) {
          double s = 0.0;
          for (int b = 0; b < NP; ++b) s += T.dPhiF[((f * D + r) * NGF + gf) * NP + b] * z[b][i];
          gr[r] = s;
        }
        for (int fl = 0; fl < NF; ++fl) {  // the same for every direction k
          double l = 0.0;
          for (int c = 0; c < NFN; ++c) l += T.PLF[((f * NF + fl) * NGF + gf) * NFN + c] * dz[fl * NFN + c][i];
          lift[fl] = l;
        }
        for (int k = 0; k < D; ++k) {
          double s = 0.0;
          for (int r = 0; r < D; ++r) s += Jinv[r * D + k] * gr[r];
          for (int fl = 0; fl < NF; ++fl) {
            const double* Gl = G + D * D + 1 + fl * (D + 1);
            s += Gl[k] * (Gl[D] / detJ) * lift[fl];
          }
          q[i][k] = s;
        }
      }
    }
    bad = !(v[M - 1] < 0.0) || !(vh[M - 1] < 0.0);
    // pass A: derivatives with respect to vhat
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
    du_of_v<D>(vhd, dvd, ph.gamma, duh);  // A0(vhat) (v - vhat)
    Dual<M> sdu[M];                        // sigma(vhat) (v - vhat)
    SigmaValues<M, SYM> sig;
    if constexpr (SYM) {  // sigma_S = |A_n| A0 (Eq. symStab)
      abs_flux_jac_apply<D>(rh, velh, prh, n, ph.gamma, duh, sdu);
      double vv[D];
      for (int j = 0; j < D; ++j) vv[j] = velh[j].v;
      for (int l = 0; l < M; ++l) {
        double x[M], y[M];
        for (int k = 0; k < M; ++k) x[k] = uh[k].d[l];
        abs_flux_jac_apply<D>(rh.v, vv, prh.v, n, ph.gamma, x, y);
        for (int i = 0; i < M; ++i) sig.s[i][l] = y[i];
      }
    } else {  // sigma_SLF = lambda_max A0 (Eq. sLxF)
      const Dual<M> lam = lambda_max<D>(rh, velh, prh, n, ph.gamma);
      for (int i = 0; i < M; ++i) sdu[i] = lam * duh[i];
      sig.lam = lam.v;
      sig.uh = uh;
    }
    Dual<M> hA[M];
    for (int i = 0; i < M; ++i) {
      Dual<M> s = Fh[i][0] * n[0];
      for (int j = 1; j < D; ++j) s = s + Fh[i][j] * n[j];
      hA[i] = 0.5 * s + 0.5 * sdu[i];
    }
    if (C::VISC && ph.gflux != 1) {  // ghat = G(vhat, q) . n (Eq. numericalFluxNS_2)
      Dual<M> Gh[M][D];
      visc_flux<D>(vhd, q, ph, Gh);
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < D; ++j) hA[i] = hA[i] + Gh[i][j] * n[j];
    }
    // pass B: derivatives with respect to v (F(v).n; the sigma term gives sigma(vhat))
    Dual<M> vd[M];
    for (int l = 0; l < M; ++l) {
      vd[l] = dconst<M>(v[l]);
      vd[l].d[l] = 1.0;
    }
    Dual<M> rv, velv[D], pv, Fv[M][D];
    prim_of_v<D>(vd, ph.gamma, rv, velv, pv);
    cons_and_flux<D>(rv, velv, pv, ph.gamma, (Dual<M>*)nullptr, Fv);
    bad = bad || !(rv.v > 0.0) || !(pv.v > 0.0);
    OutT* out = reinterpret_cast<OutT*>(a.ptf) + ((le * NF + f) * NGF + gf) * C::PT_FACE;
    OutT* HF = out;
    OutT* U0 = HF + M;
    OutT* U1 = U0 + M * M;
    OutT* U2 = U1 + M * M;
    Dual<M> gn[M];  // ghat = G(v, q) . n (Eq. numericalFluxNS_1): value and d/dv
    for (int i = 0; i < M; ++i) gn[i] = vd[0] * 0.0;
    if (C::VISC && ph.gflux == 1) {
      Dual<M> Gv[M][D];
      visc_flux<D>(vd, q, ph, Gv);
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < D; ++j) gn[i] = gn[i] + Gv[i][j] * n[j];
    }
    for (int i = 0; i < M; ++i) {
      Dual<M> s = Fv[i][0] * n[0];
      for (int j = 1; j < D; ++j) s = s + Fv[i][j] * n[j];
      put(HF, i, Wf * (hA[i].v + 0.5 * s.v + gn[i].v));
      for (int l = 0; l < M; ++l) {
        put(U0, i * M + l, Wf * (0.5 * s.d[l] + 0.5 * sig(i, l) + gn[i].d[l]));
        put(U1, i * M + l, Wf * hA[i].d[l]);
      }
    }
    if (C::VISC) {  // dG/dq contracted with the normal, at the state the viscous flux uses
      const double* vs = ph.gflux == 1 ? v : vh;
      const ViscFactors<D> vf = visc_factors<D>(vs);
      visc_jac_dir<D>(vf, n, visc_params_at(ph, vs[M - 1]),
                      [&](int i, int l, int k, double val) { put(U2, (i * M + l) * D + k, Wf * val); });
    }
  }
  if (bad) atomicOr(a.status + e, HDG_STATUS_NONPHYSICAL);
}

// k_pointwise with the stabilization matrix the physics selects
template <class C, class OutT = double>
void launch_pointwise(const AssembleArgs& a, const DevTables& T, const PhysParams& ph, cudaStream_t s) {
  const int threads = ((C::NG + C::NF * C::NGF + 31) / 32) * 32;
  if (ph.stab == 1)
    k_pointwise<C, OutT, true><<<(unsigned)a.ne, threads, 0, s>>>(a, T, ph);
  else
    k_pointwise<C, OutT, false><<<(unsigned)a.ne, threads, 0, s>>>(a, T, ph);
}

// ------------------------------------------------------------------------------------
// k_assemble
// ------------------------------------------------------------------------------------
template <class C>
struct AsmSmem {
  static constexpr int GT = C::NG < 64 ? C::NG : 64;  // volume points per tile
  static constexpr int RB = C::NR * GT * C::NZ;
  static constexpr int RBF = C::NRF * C::NGF * C::NZ;
  static constexpr int RBMAX = RB > RBF ? RB : RBF;
  static constexpr int ZS = C::NP * GT * C::NR;
  static constexpr int ZSF = C::NFN * C::NGF * C::NRF;
  static constexpr int ZSMAX = ZS > ZSF ? ZS : ZSF;
  static constexpr size_t bytes =
      sizeof(double) * (RBMAX + ZSMAX + C::NZ * C::M + C::GEO + C::NV + C::NT);
};

template <class C>
__global__ void __launch_bounds__(256) k_assemble(AssembleArgs a, DevTables T) {
  constexpr int D = C::D, M = C::M, NP = C::NP, NFN = C::NFN, NF = C::NF, NG = C::NG, NGF = C::NGF;
  constexpr int NZ = C::NZ, NV = C::NV, NT = C::NT, NR = C::NR, NRF = C::NRF;
  using SM = AsmSmem<C>;
  constexpr int GT = SM::GT;
  extern __shared__ double smem[];
  double* Rb = smem;
  double* Zs = Rb + SM::RBMAX;
  double(*z)[M] = reinterpret_cast<double(*)[M]>(Zs + SM::ZSMAX);
  double* G = Zs + SM::ZSMAX + NZ * M;
  double* Rv = G + C::GEO;
  double* Rt = Rv + NV;
  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  if (skip_element(a, e)) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  load_element<C>(a, e, z, G);
  __syncthreads();
  const double* Jinv = G;
  const double detJ = G[D * D];
  double* Ap = a.Ap + le * NV * NV;
  double* Cp = a.Cp + le * NT * NV;
  double* Bp = a.recov + e * (int64_t)(NV * NT + NV);
  double* Dp = a.S + e * (int64_t)NT * NT;
  const double* ptv = a.ptv + le * NG * C::PT_VOL;
  const double* ptf = a.ptf + le * NF * NGF * C::PT_FACE;

  // residual R_v, volume part
  for (int t = tid; t < NV; t += nth) {
    int an = t / M, i = t % M;
    double s = a.hist ? -a.hist[e * NV + t] : 0.0;
    for (int g = 0; g < NG; ++g) {
      const double* P = ptv + g * C::PT_VOL;
      s += T.Phi[g * NP + an] * P[i];
      for (int r = 0; r < D; ++r) s += T.dPhi[(r * NG + g) * NP + an] * P[M + r * M + i];
    }
    Rv[t] = s;
  }

  // ---------------- volume contractions ----------------
  for (int g0 = 0; g0 < NG; g0 += GT) {
    const int ng = (NG - g0) < GT ? (NG - g0) : GT;
    __syncthreads();
    // right operators Rb[beta][gg][j]
    for (int t = tid; t < NR * GT * NZ; t += nth) {
      int beta = t / (GT * NZ), gg = (t / NZ) % GT, j = t % NZ;
      double val = 0.0;
      if (gg < ng) {
        int g = g0 + gg;
        if (beta == 0) {
          val = j < NP ? T.Phi[g * NP + j] : 0.0;
        } else {
          int k = beta - 1;
          if (j < NP) {
            for (int r = 0; r < D; ++r) val += Jinv[r * D + k] * T.dPhi[(r * NG + g) * NP + j];
            for (int f = 0; f < NF; ++f) {
              int c = T.nodepos[f * NP + j];
              if (c >= 0) {
                const double* Gf = G + D * D + 1 + f * (D + 1);
                val -= Gf[k] * (Gf[D] / detJ) * T.PL[(f * NG + g) * NFN + c];
              }
            }
          } else {
            int f = (j - NP) / NFN, c = (j - NP) % NFN;
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
      // Zs[a][gg][beta] = sum_alpha L_alpha(g, a) C^{il}_{alpha beta}(g)
      for (int t = tid; t < NP * GT * NR; t += nth) {
        int an = t / (GT * NR), gg = (t / NR) % GT, beta = t % NR;
        double val = 0.0;
        if (gg < ng) {
          int g = g0 + gg;
          const double* P = ptv + g * C::PT_VOL;
          const double* T0 = P + M + D * M;
          const double* T1 = T0 + M * M;
          const double* T2 = T1 + D * M * M;
          if (beta == 0) {
            val = T.Phi[g * NP + an] * T0[i * M + l];
            for (int r = 0; r < D; ++r) val += T.dPhi[(r * NG + g) * NP + an] * T1[(r * M + i) * M + l];
          } else {
            int k = beta - 1;
            for (int r = 0; r < D; ++r)
              val += T.dPhi[(r * NG + g) * NP + an] * T2[((r * M + i) * M + l) * D + k];
          }
        }
        Zs[t] = val;
      }
      __syncthreads();
      for (int t = tid; t < NP * NZ; t += nth) {
        int an = t / NZ, j = t % NZ;
        const int b0 = j < NP ? 0 : 1;
        double acc = 0.0;
        for (int gg = 0; gg < ng; ++gg)
          for (int beta = b0; beta < NR; ++beta) acc += Zs[(an * GT + gg) * NR + beta] * Rb[(beta * GT + gg) * NZ + j];
        int row = an * M + i;
        if (j < NP) {
          double* dst = Ap + row * NV + j * M + l;
          *dst = (g0 == 0) ? acc : *dst + acc;
        } else {
          double* dst = Bp + row * NT + (j - NP) * M + l;
          *dst = (g0 == 0) ? acc : *dst + acc;
        }
      }
    }
  }

  // ---------------- face contractions ----------------
  for (int f = 0; f < NF; ++f) {
    __syncthreads();
    const double* Gf = G + D * D + 1 + f * (D + 1);
    for (int t = tid; t < NRF * NGF * NZ; t += nth) {
      int beta = t / (NGF * NZ), gf = (t / NZ) % NGF, j = t % NZ;
      const double* phif = T.PhiF + (f * NGF + gf) * NP;
      double val = 0.0;
      if (beta == 0) {
        val = j < NP ? phif[j] : 0.0;
      } else if (beta == 1) {
        if (j >= NP && (j - NP) / NFN == f) val = phif[T.fnodes[f * NFN + (j - NP) % NFN]];
      } else {
        int k = beta - 2;
        if (j < NP) {
          for (int r = 0; r < D; ++r) val += Jinv[r * D + k] * T.dPhiF[((f * D + r) * NGF + gf) * NP + j];
          for (int fl = 0; fl < NF; ++fl) {
            int c = T.nodepos[fl * NP + j];
            if (c >= 0) {
              const double* Gl = G + D * D + 1 + fl * (D + 1);
              val -= Gl[k] * (Gl[D] / detJ) * T.PLF[((f * NF + fl) * NGF + gf) * NFN + c];
            }
          }
        } else {
          int fl = (j - NP) / NFN, c = (j - NP) % NFN;
          const double* Gl = G + D * D + 1 + fl * (D + 1);
          val = Gl[k] * (Gl[D] / detJ) * T.PLF[((f * NF + fl) * NGF + gf) * NFN + c];
        }
      }
      Rb[t] = val;
    }
    (void)Gf;
    // residual: face contribution
    __syncthreads();
    for (int t = tid; t < NFN * M; t += nth) {
      int c = t / M, i = t % M;
      double s = 0.0;
      for (int gf = 0; gf < NGF; ++gf) {
        double psi = T.PhiF[(f * NGF + gf) * NP + T.fnodes[f * NFN + c]];
        s += psi * ptf[(f * NGF + gf) * C::PT_FACE + i];
      }
      Rv[T.fnodes[f * NFN + c] * M + i] += s;
      Rt[(f * NFN + c) * M + i] = s;
    }
    for (int il = 0; il < M * M; ++il) {
      const int i = il / M, l = il % M;
      __syncthreads();
      for (int t = tid; t < NFN * NGF * NRF; t += nth) {
        int c = t / (NGF * NRF), gf = (t / NRF) % NGF, beta = t % NRF;
        const double* P = ptf + (f * NGF + gf) * C::PT_FACE;
        const double* U0 = P + M;
        const double* U1 = U0 + M * M;
        const double* U2 = U1 + M * M;
        double psi = T.PhiF[(f * NGF + gf) * NP + T.fnodes[f * NFN + c]];
        double u;
        if (beta == 0)
          u = U0[i * M + l];
        else if (beta == 1)
          u = U1[i * M + l];
        else
          u = U2[(i * M + l) * D + (beta - 2)];
        Zs[t] = psi * u;
      }
      __syncthreads();
      for (int t = tid; t < NFN * NZ; t += nth) {
        int c = t / NZ, j = t % NZ;
        double acc = 0.0;
        for (int gf = 0; gf < NGF; ++gf)
          for (int beta = 0; beta < NRF; ++beta) acc += Zs[(c * NGF + gf) * NRF + beta] * Rb[(beta * NGF + gf) * NZ + j];
        int rowv = T.fnodes[f * NFN + c] * M + i;
        int rowt = (f * NFN + c) * M + i;
        if (j < NP) {
          Ap[rowv * NV + j * M + l] += acc;
          Cp[rowt * NV + j * M + l] = acc;
        } else {
          int tcol = (j - NP) * M + l;
          Bp[rowv * NT + tcol] += acc;
          Dp[rowt * NT + tcol] = acc;
        }
      }
    }
  }
  __syncthreads();
  double* Rout = a.R + e * (int64_t)(NV + NT);
  for (int t = tid; t < NV; t += nth) Rout[t] = Rv[t];
  for (int t = tid; t < NT; t += nth) Rout[NV + t] = Rt[t];
}

// ------------------------------------------------------------------------------------
// k_condense
// ------------------------------------------------------------------------------------
template <class C>
struct CondSmem {
  static constexpr int CB = 64;  // right-hand-side columns per block
  static constexpr size_t bytes = sizeof(double) * (C::NV * C::NV + C::NV * CB) + sizeof(int) * C::NV + 64;
};

template <class C>
__global__ void __launch_bounds__(256) k_condense(AssembleArgs a) {
  constexpr int NV = C::NV, NT = C::NT;
  using SM = CondSmem<C>;
  constexpr int CB = SM::CB;
  extern __shared__ double smem[];
  double* LU = smem;                 // [NV][NV]
  double* Xs = LU + NV * NV;         // [NV][CB]
  int* piv = reinterpret_cast<int*>(Xs + NV * CB);
  __shared__ int s_piv;
  __shared__ int s_bad;
  const int64_t le = blockIdx.x;
  const int64_t e = a.e0 + le;
  if (skip_element(a, e)) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const double* Ap = a.Ap + le * NV * NV;
  const double* Cp = a.Cp + le * NT * NV;
  double* X = a.recov + e * (int64_t)(NV * NT + NV);
  double* y = X + NV * NT;
  double* S = a.S + e * (int64_t)NT * NT;
  const double* R = a.R + e * (int64_t)(NV + NT);
  for (int t = tid; t < NV * NV; t += nth) LU[t] = Ap[t];
  if (tid == 0) s_bad = 0;
  __syncthreads();
  // LU with partial pivoting (row interchanges recorded in piv)
  for (int k = 0; k < NV; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int r = k + tid; r < NV; r += 32) {
        double v = fabs(LU[r * NV + k]);
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
      if (tid == 0) {
        s_piv = bi;
        piv[k] = bi;
        if (!(best > 0.0)) s_bad = 1;
      }
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != k)
      for (int j = tid; j < NV; j += nth) {
        double t = LU[k * NV + j];
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
      int r = k + 1 + t / rem, c = k + 1 + t % rem;
      LU[r * NV + c] -= LU[r * NV + k] * LU[k * NV + c];
    }
    __syncthreads();
  }
  if (tid == 0 && s_bad) atomicOr(a.status + e, HDG_STATUS_SINGULAR);
  // X = A'^{-1} [B' | R_v] in column blocks (B' stored in X)
  for (int c0 = 0; c0 < NT + 1; c0 += CB) {
    const int nc = (NT + 1 - c0) < CB ? (NT + 1 - c0) : CB;
    __syncthreads();
    for (int t = tid; t < NV * CB; t += nth) {
      int r = t / CB, c = t % CB;
      int col = c0 + c;
      double v = 0.0;
      if (c < nc) v = col < NT ? X[r * NT + col] : R[r];
      Xs[t] = v;
    }
    __syncthreads();
    // apply the row interchanges in order
    for (int t = tid; t < CB; t += nth)
      for (int k = 0; k < NV; ++k) {
        int p = piv[k];
        if (p != k) {
          double tmp = Xs[k * CB + t];
          Xs[k * CB + t] = Xs[p * CB + t];
          Xs[p * CB + t] = tmp;
        }
      }
    __syncthreads();
    for (int k = 0; k < NV; ++k) {  // forward, unit lower
      for (int t = tid; t < (NV - k - 1) * CB; t += nth) {
        int r = k + 1 + t / CB, c = t % CB;
        Xs[r * CB + c] -= LU[r * NV + k] * Xs[k * CB + c];
      }
      __syncthreads();
    }
    for (int k = NV - 1; k >= 0; --k) {  // backward, upper
      for (int c = tid; c < CB; c += nth) Xs[k * CB + c] /= LU[k * NV + k];
      __syncthreads();
      for (int t = tid; t < k * CB; t += nth) {
        int r = t / CB, c = t % CB;
        Xs[r * CB + c] -= LU[r * NV + k] * Xs[k * CB + c];
      }
      __syncthreads();
    }
    for (int t = tid; t < NV * CB; t += nth) {
      int r = t / CB, c = t % CB;
      int col = c0 + c;
      if (c < nc) {
        if (col < NT)
          X[r * NT + col] = Xs[t];
        else
          y[r] = Xs[t];
      }
    }
  }
  __syncthreads();
  // S = D' - C' X ; g = R_t - C' y
  for (int t = tid; t < NT * NT; t += nth) {
    int r = t / NT, c = t % NT;
    double s = S[t];
    const double* Cr = Cp + r * NV;
    for (int k = 0; k < NV; ++k) s -= Cr[k] * X[k * NT + c];
    S[t] = s;
  }
  double* g = a.g + e * NT;
  for (int r = tid; r < NT; r += nth) {
    double s = R[NV + r];
    const double* Cr = Cp + r * NV;
    for (int k = 0; k < NV; ++k) s -= Cr[k] * y[k];
    g[r] = s;
  }
  if (a.only_flag != 0 && tid == 0) {  // flagged-only pass: the block is now the FP64 form's
    atomicAnd(a.status + e, ~a.only_flag);
    atomicOr(a.status + e, HDG_STATUS_FP64);
  }
}

// ------------------------------------------------------------------------------------
// k_entropy_terms: the two integrals of Eq. PiS (Sec. 5.6) from (v_h, q_h), one CTA per element:
//   acc[0] += int_K rho s,  s = log(p / rho^gamma) (Sec. 2.3)
//   acc[1] += (1/c_v) int_K (Phi / T + kappa |grad T|^2 / T^2),  Phi = grad V : tau
// ------------------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(128) k_entropy_terms(AssembleArgs a, DevTables T, PhysParams ph, double* acc) {
  constexpr int D = C::D, M = C::M, NP = C::NP, NFN = C::NFN, NF = C::NF, NG = C::NG;
  __shared__ double z[C::NZ][M];
  __shared__ double G[C::GEO];
  __shared__ double dz[NF * NFN][M];
  __shared__ double red[2][4];
  const int64_t e = a.e0 + blockIdx.x;
  load_element<C>(a, e, z, G);
  __syncthreads();
  for (int t = threadIdx.x; t < NF * NFN * M; t += blockDim.x) {
    const int fc = t / M, i = t % M;
    dz[fc][i] = z[NP + fc][i] - z[T.fnodes[fc]][i];
  }
  __syncthreads();
  double rs = 0.0, pr = 0.0;
  for (int g = threadIdx.x; g < NG; g += blockDim.x) {
    const double W = T.W[g] * G[D * D];
    double v[M], q[M][D];
    volume_point_state<C>(g, T, z, dz, G, v, q);
    double rho, vel[D], p;
    prim_of_v<D>(v, ph.gamma, rho, vel, p);
    rs += W * rho * (::log(p) - ph.gamma * ::log(rho));
    if (C::VISC) {
      const double vm = v[M - 1], ivm = 1.0 / vm, Temp = -ivm / ph.cv;
      const double fac = ph.mu_exp != 0.0 ? ::exp(-ph.mu_exp * ::log(ph.cv * (-vm))) : 1.0;
      const double mu = ph.mu * fac, kappa = ph.kappa * fac;
      double gV[D][D], gT2 = 0.0, div = 0.0;
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) gV[i][j] = v[1 + i] * ivm * ivm * q[M - 1][j] - q[1 + i][j] * ivm;
      for (int j = 0; j < D; ++j) {
        const double gt = q[M - 1][j] * ivm * ivm / ph.cv;
        gT2 += gt * gt;
        div += gV[j][j];
      }
      double Phi = 0.0;
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          const double tau = mu * (gV[i][j] + gV[j][i] - (i == j ? (2.0 / 3.0) * div : 0.0));
          Phi += gV[i][j] * tau;
        }
      pr += W * (Phi / Temp + kappa * gT2 / (Temp * Temp)) / ph.cv;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    rs += __shfl_xor_sync(0xffffffffu, rs, off);
    pr += __shfl_xor_sync(0xffffffffu, pr, off);
  }
  const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][warp] = rs;
    red[1][warp] = pr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < nw; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    atomicAdd(acc, s0);
    atomicAdd(acc + 1, s1);
  }
}

}  // namespace hdg
