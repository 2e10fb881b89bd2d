// Device-side building blocks: compile-time element sizes, forward-mode dual
// numbers, and the pointwise physics of the entropy-variable formulation.
//
// Physics (paper Sec. 2): m = d + 2 conserved variables u = (rho, rho V, rho E),
// inviscid flux F (Eq. flux), viscous flux G (Eqs. viscFlux, closuresNS) and the
// entropy variables v = dH/du for H = -rho s (Sec. 2.3). The inverse map u(v) is not
// printed; from v(u):  s = gamma - v_1 + |w|^2 / (2 v_m),
//   log rho = (log(gamma-1) - log(-v_m) - s) / (gamma-1),
//   p = rho (gamma-1) / (-v_m),  V = -w / v_m,  w = (v_2..v_{d+1}).
// Nondimensionalisation: c_v = 1/(gamma (gamma-1) M^2), mu = 1/Re,
// kappa = gamma c_v mu / Pr, beta = 0.
#pragma once
#include <cstdint>

#define HDG_DEVI __device__ __forceinline__

namespace hdg {

constexpr int cbinom(int n, int k) { return k == 0 ? 1 : (n * cbinom(n - 1, k - 1)) / k; }
constexpr int cipow(int b, int e) { return e == 0 ? 1 : b * cipow(b, e - 1); }

template <int D_, int P_, int K_, bool VISC_>
struct Cfg {
  static constexpr int D = D_, P = P_, K = K_;
  static constexpr bool VISC = VISC_;
  static constexpr int M = D + 2;
  static constexpr int NP = cbinom(P + D, D);
  static constexpr int NFN = cbinom(P + D - 1, D - 1);
  static constexpr int NF = D + 1;
  static constexpr int NG = cipow(K, D);
  static constexpr int NGF = cipow(K, D - 1);
  static constexpr int NV = NP * M;            // interior unknowns (v) per element
  static constexpr int NT = NF * NFN * M;      // trace unknowns per element
  static constexpr int NZ = NP + NF * NFN;     // nodal unknowns per component
  static constexpr int GEO = D * D + 1 + NF * (D + 1);
  static constexpr int NR = VISC ? D + 1 : 1;  // volume right operators: value (+ grad)
  static constexpr int NRF = VISC ? D + 2 : 2; // face right operators: v, vhat (+ grad)
  // per-point tensors written by the pointwise kernel
  static constexpr int PT_VOL = M + D * M + M * M + D * M * M + (VISC ? D * M * M * D : 0);
  static constexpr int PT_FACE = M + 2 * M * M + (VISC ? M * M * D : 0);
};

struct PhysParams {
  double gamma, cv, mu, kappa;
  double mu_exp;  // power law mu = mu (T / T_inf)^mu_exp, kappa likewise (T_inf = 1); 0: constant
  int gflux;      // viscous numerical flux: 2 = G(vhat, q) . n, 1 = G(v, q) . n
  int stab;       // stabilization matrix: 0 = lambda_max A0 (Eq. sLxF), 1 = |A_n| A0 (Eq. symStab)
};

// Constant reference tables (device pointers into one buffer).
struct DevTables {
  const double* W;      // [NG]
  const double* Phi;    // [NG][NP]
  const double* dPhi;   // [D][NG][NP]
  const double* PL;     // [NF][NG][NFN]
  const double* WF;     // [NGF]
  const double* PhiF;   // [NF][NGF][NP]
  const double* dPhiF;  // [NF][D][NGF][NP]
  const double* PLF;    // [NF][NF][NGF][NFN]
  const int* fnodes;    // [NF][NFN]
  const int* nodepos;   // [NF][NP] position of node a on face f, -1 if off the face
};

// ---------------------------------------------------------------------------------
// Forward-mode dual numbers with N derivative directions.
// ---------------------------------------------------------------------------------
template <int N>
struct Dual {
  double v;
  double d[N];
};

template <int N>
HDG_DEVI Dual<N> dconst(double a) {
  Dual<N> r;
  r.v = a;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = 0.0;
  return r;
}
template <int N>
HDG_DEVI Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
HDG_DEVI Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
HDG_DEVI Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N>
HDG_DEVI Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N>
HDG_DEVI Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N>
HDG_DEVI Dual<N> operator+(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v += b;
  return r;
}
template <int N>
HDG_DEVI Dual<N> operator+(double b, const Dual<N>& a) {
  return a + b;
}
template <int N>
HDG_DEVI Dual<N> operator-(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v -= b;
  return r;
}
template <int N>
HDG_DEVI Dual<N> operator-(double b, const Dual<N>& a) {
  Dual<N> r = -a;
  r.v += b;
  return r;
}
template <int N>
HDG_DEVI Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N>
HDG_DEVI Dual<N> operator*(double b, const Dual<N>& a) {
  return a * b;
}
template <int N>
HDG_DEVI Dual<N> operator/(const Dual<N>& a, double b) {
  return a * (1.0 / b);
}
template <int N>
HDG_DEVI Dual<N> operator/(double a, const Dual<N>& b) {
  Dual<N> r;
  double ib = 1.0 / b.v;
  r.v = a * ib;
  double s = -r.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = s * b.d[i];
  return r;
}
template <int N>
HDG_DEVI Dual<N> log(const Dual<N>& a) {
  Dual<N> r;
  r.v = ::log(a.v);
  double s = 1.0 / a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s;
  return r;
}
template <int N>
HDG_DEVI Dual<N> exp(const Dual<N>& a) {
  Dual<N> r;
  r.v = ::exp(a.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * r.v;
  return r;
}
template <int N>
HDG_DEVI Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r;
  r.v = ::sqrt(a.v);
  double s = 0.5 / r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s;
  return r;
}
// |x| with d|x|/dx = sign(x), sign(0) = 0
template <int N>
HDG_DEVI Dual<N> absk(const Dual<N>& a) {
  double s = (a.v > 0.0) ? 1.0 : ((a.v < 0.0) ? -1.0 : 0.0);
  return a * s;
}
HDG_DEVI double absk(double a) { return a > 0.0 ? a : -a; }
HDG_DEVI double valof(double a) { return a; }
template <int N>
HDG_DEVI double valof(const Dual<N>& a) {
  return a.v;
}

// ---------------------------------------------------------------------------------
// Pointwise physics, generic in the scalar type (double or Dual<N>).
// ---------------------------------------------------------------------------------
template <int D, class T>
HDG_DEVI void prim_of_v(const T* v, double gamma, T& rho, T* vel, T& p) {
  using ::log;
  using ::exp;
  const double g1 = gamma - 1.0;
  const T& vm = v[D + 1];
  T ww = v[1] * v[1];
#pragma unroll
  for (int i = 1; i < D; ++i) ww = ww + v[1 + i] * v[1 + i];
  T s = (gamma - v[0]) + ww / (2.0 * vm);
  T lnrho = (::log(g1) - log(-vm) - s) * (1.0 / g1);
  rho = exp(lnrho);
  T ivm = 1.0 / vm;
  p = -(rho * g1) * ivm;
#pragma unroll
  for (int i = 0; i < D; ++i) vel[i] = -(v[1 + i] * ivm);
}

// u(v) and the inviscid flux F(v) [M][D] from primitives.
template <int D, class T>
HDG_DEVI void cons_and_flux(const T& rho, const T* vel, const T& p, double gamma, T* u, T (*F)[D]) {
  T vv = vel[0] * vel[0];
#pragma unroll
  for (int i = 1; i < D; ++i) vv = vv + vel[i] * vel[i];
  T rhoE = p * (1.0 / (gamma - 1.0)) + 0.5 * (rho * vv);
  if (u) {
    u[0] = rho;
#pragma unroll
    for (int i = 0; i < D; ++i) u[1 + i] = rho * vel[i];
    u[D + 1] = rhoE;
  }
  if (F) {
    T H = rhoE + p;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      T mj = rho * vel[j];
      F[0][j] = mj;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        F[1 + i][j] = mj * vel[i];
        if (i == j) F[1 + i][j] = F[1 + i][j] + p;
      }
      F[D + 1][j] = vel[j] * H;
    }
  }
}

// Directional derivative du = A0(v) dv of u(v) (chain rule on the inverse map).
template <int D, class T>
HDG_DEVI void du_of_v(const T* v, const T* dv, double gamma, T* du) {
  const double g1 = gamma - 1.0;
  T rho, vel[D], p;
  prim_of_v<D>(v, gamma, rho, vel, p);
  const T& vm = v[D + 1];
  const T& dvm = dv[D + 1];
  T ivm = 1.0 / vm;
  T wdw = v[1] * dv[1];
  T ww = v[1] * v[1];
#pragma unroll
  for (int i = 1; i < D; ++i) {
    wdw = wdw + v[1 + i] * dv[1 + i];
    ww = ww + v[1 + i] * v[1 + i];
  }
  T ds = wdw * ivm - dv[0] - 0.5 * (ww * dvm) * (ivm * ivm);
  T dlnrho = (-(dvm * ivm) - ds) * (1.0 / g1);
  T drho = rho * dlnrho;
  T dvel[D];
#pragma unroll
  for (int i = 0; i < D; ++i) dvel[i] = (v[1 + i] * dvm) * (ivm * ivm) - dv[1 + i] * ivm;
  T dp = p * (dlnrho - dvm * ivm);
  du[0] = drho;
  T vv = vel[0] * vel[0];
  T vdv = vel[0] * dvel[0];
#pragma unroll
  for (int i = 1; i < D; ++i) {
    vv = vv + vel[i] * vel[i];
    vdv = vdv + vel[i] * dvel[i];
  }
#pragma unroll
  for (int i = 0; i < D; ++i) du[1 + i] = drho * vel[i] + rho * dvel[i];
  du[D + 1] = dp * (1.0 / g1) + 0.5 * (drho * vv) + rho * vdv;
}

// Viscous flux G(v, q) [M][D] (Eq. viscFlux) with q ~ grad v, through
// grad V_i = -grad w_i / v_m + w_i grad v_m / v_m^2 and grad T = grad v_m / (c_v v_m^2).
template <int D, class T, class TQ>
HDG_DEVI void visc_flux(const T* v, const TQ (*q)[D], const PhysParams& ph, T (*G)[D]) {
  using ::exp;
  using ::log;
  const T& vm = v[D + 1];
  T ivm = 1.0 / vm;
  T ivm2 = ivm * ivm;
  // (T / T_inf)^omega with T = 1 / (c_v (-v_m)): scales mu and kappa (Pr fixed)
  const T fac = ph.mu_exp != 0.0 ? exp(-ph.mu_exp * log(ph.cv * (-vm))) : vm * 0.0 + 1.0;
  T vel[D];
#pragma unroll
  for (int i = 0; i < D; ++i) vel[i] = -(v[1 + i] * ivm);
  T gV[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) gV[i][j] = (v[1 + i] * ivm2) * q[D + 1][j] - q[1 + i][j] * ivm;
  T div = gV[0][0];
#pragma unroll
  for (int i = 1; i < D; ++i) div = div + gV[i][i];
  T tau[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      T t = gV[i][j] + gV[j][i];
      if (i == j) t = t - (2.0 / 3.0) * div;
      tau[i][j] = (ph.mu * fac) * t;
    }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    G[0][j] = vm * 0.0;
    T e = vel[0] * tau[0][j];
#pragma unroll
    for (int i = 1; i < D; ++i) e = e + vel[i] * tau[i][j];
    T gradT = ((ph.kappa / ph.cv) * fac) * (q[D + 1][j] * ivm2);
#pragma unroll
    for (int i = 0; i < D; ++i) G[1 + i][j] = -tau[i][j];
    G[D + 1][j] = -(e + gradT);
  }
}

// Physical parameters with mu and kappa at the temperature of state v (power law; constant
// viscosity returns ph unchanged): the coefficients of dG/dq, which is linear in them.
HDG_DEVI PhysParams visc_params_at(const PhysParams& ph, double vm) {
  PhysParams p = ph;
  if (ph.mu_exp != 0.0) {
    const double fac = ::exp(-ph.mu_exp * ::log(ph.cv * (-vm)));
    p.mu *= fac;
    p.kappa *= fac;
  }
  return p;
}

// The state-dependent factors of the viscous flux, shared by every gradient direction.
template <int D>
struct ViscFactors {
  double ivm, ivm2, vel[D], A[D];  // 1/v_m, 1/v_m^2, V_i = -w_i/v_m, w_i/v_m^2
};
template <int D>
HDG_DEVI ViscFactors<D> visc_factors(const double* v) {
  ViscFactors<D> f;
  f.ivm = 1.0 / v[D + 1];
  f.ivm2 = f.ivm * f.ivm;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    f.vel[i] = -(v[1 + i] * f.ivm);
    f.A[i] = v[1 + i] * f.ivm2;
  }
  return f;
}

// sum_j c_j dG_ij/dq_lk for one vector c: the viscous flux (Eq. viscFlux) is linear in q, and
// differentiating it by hand gives, with V_a = -w_a/v_m, A_a = w_a/v_m^2 and the Kronecker
// delta d,
//   momentum i = 1+a, l = 1+b:    mu/v_m (d_ab c_k + d_ak c_b - 2/3 d_bk c_a)
//   momentum i = 1+a, l = m-1:   -mu (A_a c_k + d_ak c.A - 2/3 A_k c_a)
//   energy   i = m-1, l = 1+b:    mu/v_m (V_b c_k + V_k c_b - 2/3 d_bk c.V)
//   energy   i = m-1, l = m-1:   -mu (V.A c_k + V_k c.A - 2/3 A_k c.V) - kappa/(c_v v_m^2) c_k
// and zero for i = 0 or l = 0. emit(i, l, k, value) receives every entry; the deltas are
// branches on unrolled indices, so no arithmetic is spent on the vanishing terms.
template <int D, class Emit>
HDG_DEVI void visc_jac_dir(const ViscFactors<D>& f, const double* c, const PhysParams& ph, Emit emit) {
  constexpr int M = D + 2;
  constexpr double t3 = 2.0 / 3.0;
  double cA = c[0] * f.A[0], cV = c[0] * f.vel[0], VA = f.vel[0] * f.A[0];
#pragma unroll
  for (int j = 1; j < D; ++j) {
    cA += c[j] * f.A[j];
    cV += c[j] * f.vel[j];
    VA += f.vel[j] * f.A[j];
  }
  const double mi = ph.mu * f.ivm, kc = (ph.kappa / ph.cv) * f.ivm2;
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int l = 0; l < M; ++l) emit(0, l, k, 0.0);
#pragma unroll
    for (int i = 1; i < M; ++i) emit(i, 0, k, 0.0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
#pragma unroll
      for (int b = 0; b < D; ++b) {
        double s = 0.0;
        bool any = false;
        if (a == b) {
          s = c[k];
          any = true;
        }
        if (a == k) {
          s = any ? s + c[b] : c[b];
          any = true;
        }
        if (b == k) {
          s = any ? s - t3 * c[a] : -t3 * c[a];
          any = true;
        }
        emit(1 + a, 1 + b, k, any ? mi * s : 0.0);
      }
      double s = f.A[a] * c[k] - t3 * f.A[k] * c[a];
      if (a == k) s += cA;
      emit(1 + a, M - 1, k, -ph.mu * s);
    }
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double s = f.vel[b] * c[k] + f.vel[k] * c[b];
      if (b == k) s -= t3 * cV;
      emit(M - 1, 1 + b, k, mi * s);
    }
    emit(M - 1, M - 1, k, -ph.mu * (VA * c[k] + f.vel[k] * cA - t3 * f.A[k] * cV) - kc * c[k]);
  }
}

// Largest-magnitude eigenvalue of A_n: |V.n| + c (Eq. sLxF).
template <int D, class T>
HDG_DEVI T lambda_max(const T& rho, const T* vel, const T& p, const double* n, double gamma) {
  using ::sqrt;
  T vn = vel[0] * n[0];
#pragma unroll
  for (int i = 1; i < D; ++i) vn = vn + vel[i] * n[i];
  return absk(vn) + sqrt(gamma * p / rho);
}

// (B x)_i for B = A_n - V_n I, A_n = (dF/du) . n the Euler flux Jacobian in conservation
// variables along n; with k = |V|^2 / 2, H = gamma p / ((gamma - 1) rho) + k:
//   mass      x_V . n - V_n x_0
//   momentum  ((gamma-1) k n_i - V_i V_n) x_0 + V_i (n . x_V) - (gamma-1) n_i (V . x_V) + (gamma-1) n_i x_E
//   energy    V_n ((gamma-1) k - H) x_0 + H (n . x_V) - (gamma-1) V_n (V . x_V) + (gamma - 1) V_n x_E
template <int D, class T, class X, class Y>
HDG_DEVI void flux_jac_shifted(const T* vel, const T& vn, const T& k, const T& H, const double* n, double gamma,
                               const X* x, Y* y) {
  const double g1 = gamma - 1.0;
  Y nx = x[1] * n[0], Vx = x[1] * vel[0];
#pragma unroll
  for (int j = 1; j < D; ++j) {
    nx = nx + x[1 + j] * n[j];
    Vx = Vx + x[1 + j] * vel[j];
  }
  y[0] = nx - vn * x[0];
#pragma unroll
  for (int i = 0; i < D; ++i)
    y[1 + i] = (g1 * n[i] * k - vel[i] * vn) * x[0] + vel[i] * nx + g1 * n[i] * (x[D + 1] - Vx);
  y[D + 1] = vn * (g1 * k - H) * x[0] + H * nx + g1 * vn * (x[D + 1] - Vx);
}

// y = |A_n| x (the absolute value of Sec. 4.1, sigma_S = |A_n| A0 of Eq. symStab): the
// eigenvalues of A_n are V_n - c, V_n (d-fold), V_n + c, and interpolating |.| on them gives
//   |A_n| = |V_n| I + a B + b B^2,  B = A_n - V_n I,
//   a = (|V_n + c| - |V_n - c|) / (2 c),  b = (|V_n - c| + |V_n + c| - 2 |V_n|) / (2 c^2).
template <int D, class T, class X, class Y>
HDG_DEVI void abs_flux_jac_apply(const T& rho, const T* vel, const T& p, const double* n, double gamma, const X* x,
                                 Y* y) {
  using ::sqrt;
  constexpr int M = D + 2;
  T vn = vel[0] * n[0], k = vel[0] * vel[0];
#pragma unroll
  for (int i = 1; i < D; ++i) {
    vn = vn + vel[i] * n[i];
    k = k + vel[i] * vel[i];
  }
  k = 0.5 * k;
  const T c2 = gamma * p / rho;
  const T c = sqrt(c2);
  const T H = c2 / (gamma - 1.0) + k;
  const T am = absk(vn - c), a0 = absk(vn), ap = absk(vn + c);
  const T ca = (ap - am) / (2.0 * c), cb = (am + ap - 2.0 * a0) / (2.0 * c2);
  Y b1[M], b2[M];
  flux_jac_shifted<D>(vel, vn, k, H, n, gamma, x, b1);
  flux_jac_shifted<D>(vel, vn, k, H, n, gamma, b1, b2);
#pragma unroll
  for (int i = 0; i < M; ++i) y[i] = a0 * x[i] + ca * b1[i] + cb * b2[i];
}

}  // namespace hdg
