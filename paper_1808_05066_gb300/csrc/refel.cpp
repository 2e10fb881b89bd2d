// Reference simplex: quadrature, Lagrange basis and the constant tables of the
// element kernels. See refel.hpp for the conventions.
#include "refel.hpp"

#include <cmath>
#include <stdexcept>

namespace hdg {

namespace {

// Jacobi polynomial P_n^{(a,b)}(x) by its three-term recurrence.
double jacobi_p(int n, double a, double b, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
  for (int k = 2; k <= n; ++k) {
    double c = 2.0 * k + a + b;
    double num = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b) * p1 - 2.0 * (k + a - 1.0) * (k + b - 1.0) * c * p0;
    double den = 2.0 * k * (k + a + b) * (c - 2.0);
    p0 = p1;
    p1 = num / den;
  }
  return p1;
}

double jacobi_dp(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  return 0.5 * (n + a + b + 1.0) * jacobi_p(n - 1, a + 1.0, b + 1.0, x);
}

// Solve A X = B in place (A n x n, B n x m), Gaussian elimination with partial pivoting.
void dense_solve(std::vector<double> A, std::vector<double>& B, int n, int m) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[piv * n + k])) piv = i;
    if (A[piv * n + k] == 0.0) throw std::runtime_error("singular reference matrix");
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
      for (int j = 0; j < m; ++j) std::swap(B[k * m + j], B[piv * m + j]);
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      if (l == 0.0) continue;
      for (int j = k; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
      for (int j = 0; j < m; ++j) B[i * m + j] -= l * B[k * m + j];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    for (int j = 0; j < m; ++j) {
      double s = B[k * m + j];
      for (int i = k + 1; i < n; ++i) s -= A[k * n + i] * B[i * m + j];
      B[k * m + j] = s / A[k * n + k];
    }
  }
}

}  // namespace

void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  // roots by Newton iteration with deflation of the roots already found
  for (int k = 0; k < n; ++k) {
    double r = -std::cos((2.0 * k + 1.0) * pi / (2.0 * n));
    if (k > 0) r = 0.5 * (r + x[k - 1]);
    for (int it = 0; it < 200; ++it) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += 1.0 / (r - x[j]);
      double f = jacobi_p(n, a, b, r);
      double df = jacobi_dp(n, a, b, r);
      double delta = f / (df - s * f);
      r -= delta;
      if (std::fabs(delta) < 1e-17) break;
    }
    x[k] = r;
  }
  double c = std::pow(2.0, a + b + 1.0) * std::exp(std::lgamma(n + a + 1.0) + std::lgamma(n + b + 1.0) -
                                                   std::lgamma(n + a + b + 1.0) - std::lgamma(n + 1.0));
  for (int k = 0; k < n; ++k) {
    double d = jacobi_dp(n, a, b, x[k]);
    w[k] = c / ((1.0 - x[k] * x[k]) * d * d);
  }
}

Rule simplex_rule(int dim, int k) {
  Rule R;
  R.dim = dim;
  std::vector<double> a, wa, b, wb, c, wc;
  gauss_jacobi(k, 0.0, 0.0, a, wa);
  if (dim == 1) {
    for (int i = 0; i < k; ++i) {
      R.x.push_back(0.5 * (1.0 + a[i]));
      R.w.push_back(0.5 * wa[i]);
    }
  } else if (dim == 2) {
    gauss_jacobi(k, 1.0, 0.0, b, wb);
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) {
        double s = 0.5 * (1.0 + b[j]);
        double r = 0.5 * (1.0 + a[i]) * (1.0 - s);
        R.x.push_back(r);
        R.x.push_back(s);
        R.w.push_back(wa[i] * wb[j] / 8.0);
      }
  } else if (dim == 3) {
    gauss_jacobi(k, 1.0, 0.0, b, wb);
    gauss_jacobi(k, 2.0, 0.0, c, wc);
    for (int l = 0; l < k; ++l)
      for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
          double t = 0.5 * (1.0 + c[l]);
          double s = 0.5 * (1.0 + b[j]) * (1.0 - t);
          double r = 0.5 * (1.0 + a[i]) * (1.0 - s - t);
          R.x.push_back(r);
          R.x.push_back(s);
          R.x.push_back(t);
          R.w.push_back(wa[i] * wb[j] * wc[l] / 64.0);
        }
  } else {
    throw std::runtime_error("simplex_rule: dim");
  }
  R.n = (int)R.w.size();
  return R;
}

// Silvester factor R_k(t) = prod_{j<k} (p t - j) / (j + 1) and its derivative.
static void silvester(int k, int p, double t, double& val, double& der) {
  val = 1.0;
  der = 0.0;
  for (int j = 0; j < k; ++j) {
    double f = (p * t - j) / (j + 1.0);
    double df = p / (j + 1.0);
    der = der * f + val * df;
    val *= f;
  }
}

void RefElement::eval(const double* x, int npts, double* phi, double* dphi) const {
  const int nb = dim + 1;
  for (int q = 0; q < npts; ++q) {
    double lam[4];
    lam[0] = 1.0;
    for (int r = 0; r < dim; ++r) {
      lam[r + 1] = x[q * dim + r];
      lam[0] -= lam[r + 1];
    }
    for (int a = 0; a < Np; ++a) {
      int alpha[4];
      alpha[0] = p;
      for (int r = 0; r < dim; ++r) {
        alpha[r + 1] = idx[a * dim + r];
        alpha[0] -= alpha[r + 1];
      }
      double val[4], der[4];
      for (int i = 0; i < nb; ++i) silvester(alpha[i], p, lam[i], val[i], der[i]);
      double prod = 1.0;
      for (int i = 0; i < nb; ++i) prod *= val[i];
      phi[q * Np + a] = prod;
      if (dphi) {
        double dl[4];  // d phi / d lambda_i
        for (int i = 0; i < nb; ++i) {
          double g = der[i];
          for (int j = 0; j < nb; ++j)
            if (j != i) g *= val[j];
          dl[i] = g;
        }
        for (int r = 0; r < dim; ++r) dphi[(q * Np + a) * dim + r] = dl[r + 1] - dl[0];
      }
    }
  }
}

RefElement make_refel(int dim, int p, int K) {
  RefElement R;
  R.dim = dim;
  R.p = p;
  R.K = K;
  if (dim == 2) {
    for (int j = 0; j <= p; ++j)
      for (int i = 0; i <= p - j; ++i) {
        R.idx.push_back(i);
        R.idx.push_back(j);
      }
  } else {
    for (int k = 0; k <= p; ++k)
      for (int j = 0; j <= p - k; ++j)
        for (int i = 0; i <= p - k - j; ++i) {
          R.idx.push_back(i);
          R.idx.push_back(j);
          R.idx.push_back(k);
        }
  }
  R.Np = (int)R.idx.size() / dim;
  R.nF = dim + 1;
  R.face_nodes.resize(R.nF);
  for (int f = 0; f < R.nF; ++f)
    for (int a = 0; a < R.Np; ++a) {
      int s = 0;
      for (int r = 0; r < dim; ++r) s += R.idx[a * dim + r];
      bool on = (f == 0) ? (s == p) : (R.idx[a * dim + f - 1] == 0);
      if (on) R.face_nodes[f].push_back(a);
    }
  R.Nf = (int)R.face_nodes[0].size();
  R.vol = simplex_rule(dim, K);
  R.face = simplex_rule(dim - 1, K);
  R.NG = R.vol.n;
  R.NGF = R.face.n;
  R.fqp.resize(R.nF);
  for (int f = 0; f < R.nF; ++f) {
    // reference vertices except f, increasing
    double Y[4][3] = {};
    int nv = 0;
    for (int v = 0; v <= dim; ++v) {
      if (v == f) continue;
      for (int r = 0; r < dim; ++r) Y[nv][r] = (v > 0 && r == v - 1) ? 1.0 : 0.0;
      ++nv;
    }
    for (int q = 0; q < R.NGF; ++q)
      for (int r = 0; r < dim; ++r) {
        double xr = Y[0][r];
        for (int i = 1; i < dim; ++i) xr += R.face.x[q * (dim - 1) + i - 1] * (Y[i][r] - Y[0][r]);
        R.fqp[f].push_back(xr);
      }
  }
  return R;
}

RefTables make_tables(const RefElement& r) {
  RefTables T;
  T.dim = r.dim;
  T.p = r.p;
  T.K = r.K;
  T.Np = r.Np;
  T.Nf = r.Nf;
  T.nF = r.nF;
  T.NG = r.NG;
  T.NGF = r.NGF;
  const int d = r.dim, Np = r.Np, Nf = r.Nf, nF = r.nF, NG = r.NG, NGF = r.NGF;
  T.W = r.vol.w;
  T.WF = r.face.w;
  std::vector<double> dtmp(NG * Np * d);
  T.Phi.resize(NG * Np);
  r.eval(r.vol.x.data(), NG, T.Phi.data(), dtmp.data());
  T.dPhi.resize(d * NG * Np);
  for (int g = 0; g < NG; ++g)
    for (int a = 0; a < Np; ++a)
      for (int s = 0; s < d; ++s) T.dPhi[(s * NG + g) * Np + a] = dtmp[(g * Np + a) * d + s];
  T.PhiF.resize(nF * NGF * Np);
  T.dPhiF.resize(nF * d * NGF * Np);
  std::vector<double> dft(NGF * Np * d);
  for (int f = 0; f < nF; ++f) {
    r.eval(r.fqp[f].data(), NGF, &T.PhiF[f * NGF * Np], dft.data());
    for (int g = 0; g < NGF; ++g)
      for (int a = 0; a < Np; ++a)
        for (int s = 0; s < d; ++s) T.dPhiF[((f * d + s) * NGF + g) * Np + a] = dft[(g * Np + a) * d + s];
  }
  T.fnodes.resize(nF * Nf);
  for (int f = 0; f < nF; ++f)
    for (int c = 0; c < Nf; ++c) T.fnodes[f * Nf + c] = r.face_nodes[f][c];
  // reference mass matrix and face lifts L_f = Mref^{-1} E_f
  T.Mref.assign(Np * Np, 0.0);
  for (int g = 0; g < NG; ++g)
    for (int a = 0; a < Np; ++a)
      for (int b = 0; b < Np; ++b) T.Mref[a * Np + b] += T.W[g] * T.Phi[g * Np + a] * T.Phi[g * Np + b];
  std::vector<double> L(nF * Np * Nf);
  for (int f = 0; f < nF; ++f) {
    std::vector<double> E(Np * Nf, 0.0);
    for (int q = 0; q < NGF; ++q)
      for (int a = 0; a < Np; ++a)
        for (int c = 0; c < Nf; ++c)
          E[a * Nf + c] += T.WF[q] * T.PhiF[(f * NGF + q) * Np + a] * T.PhiF[(f * NGF + q) * Np + r.face_nodes[f][c]];
    dense_solve(T.Mref, E, Np, Nf);
    for (int i = 0; i < Np * Nf; ++i) L[f * Np * Nf + i] = E[i];
  }
  T.PL.assign(nF * NG * Nf, 0.0);
  for (int f = 0; f < nF; ++f)
    for (int g = 0; g < NG; ++g)
      for (int c = 0; c < Nf; ++c) {
        double s = 0.0;
        for (int b = 0; b < Np; ++b) s += T.Phi[g * Np + b] * L[(f * Np + b) * Nf + c];
        T.PL[(f * NG + g) * Nf + c] = s;
      }
  T.PLF.assign(nF * nF * NGF * Nf, 0.0);
  for (int f = 0; f < nF; ++f)
    for (int fl = 0; fl < nF; ++fl)
      for (int g = 0; g < NGF; ++g)
        for (int c = 0; c < Nf; ++c) {
          double s = 0.0;
          for (int b = 0; b < Np; ++b) s += T.PhiF[(f * NGF + g) * Np + b] * L[(fl * Np + b) * Nf + c];
          T.PLF[((f * nF + fl) * NGF + g) * Nf + c] = s;
        }
  return T;
}

ClassTables make_class_tables(int dim, int pk, int pt) {
  const RefElement rk = make_refel(dim, pk, pk + 1), rt = make_refel(dim, pt, pt + 1);
  ClassTables T;
  T.dim = dim;
  T.pk = pk;
  T.pt = pt;
  T.Np = rk.Np;
  T.Nfk = rk.Nf;
  T.Nft = rt.Nf;
  T.nF = rk.nF;
  T.NG = rk.NG;
  T.NGF = rt.NGF;
  const int d = dim, Np = rk.Np, Nft = rt.Nf, nF = rk.nF, NG = rk.NG, NGF = rt.NGF;
  T.W = rk.vol.w;
  T.WF = rt.face.w;
  std::vector<double> dtmp(NG * Np * d);
  T.Phi.resize(NG * Np);
  rk.eval(rk.vol.x.data(), NG, T.Phi.data(), dtmp.data());
  T.dPhi.resize(d * NG * Np);
  for (int g = 0; g < NG; ++g)
    for (int a = 0; a < Np; ++a)
      for (int s = 0; s < d; ++s) T.dPhi[(s * NG + g) * Np + a] = dtmp[(g * Np + a) * d + s];
  T.PhiF.resize(nF * NGF * Np);
  T.dPhiF.resize(nF * d * NGF * Np);
  T.PsiF.resize(nF * NGF * Nft);
  std::vector<double> dft(NGF * Np * d), pt_all(NGF * rt.Np);
  for (int f = 0; f < nF; ++f) {
    rk.eval(rt.fqp[f].data(), NGF, &T.PhiF[f * NGF * Np], dft.data());
    for (int g = 0; g < NGF; ++g)
      for (int a = 0; a < Np; ++a)
        for (int s = 0; s < d; ++s) T.dPhiF[((f * d + s) * NGF + g) * Np + a] = dft[(g * Np + a) * d + s];
    rt.eval(rt.fqp[f].data(), NGF, pt_all.data(), nullptr);
    for (int g = 0; g < NGF; ++g)
      for (int c = 0; c < Nft; ++c) T.PsiF[(f * NGF + g) * Nft + c] = pt_all[g * rt.Np + rt.face_nodes[f][c]];
  }
  // reference coordinates of the degree-pt nodes
  auto node_x = [&](const RefElement& r, int a, double* x) {
    for (int s = 0; s < d; ++s) x[s] = (double)r.idx[a * d + s] / (double)r.p;
  };
  T.PhiN.resize(nF * Nft * Np);
  {
    std::vector<double> x(d);
    for (int f = 0; f < nF; ++f)
      for (int c = 0; c < Nft; ++c) {
        node_x(rt, rt.face_nodes[f][c], x.data());
        rk.eval(x.data(), 1, &T.PhiN[(f * Nft + c) * Np], nullptr);
      }
  }
  T.fnodesK.resize(nF * rk.Nf);
  for (int f = 0; f < nF; ++f)
    for (int c = 0; c < rk.Nf; ++c) T.fnodesK[f * rk.Nf + c] = rk.face_nodes[f][c];
  // lifts L_f = Mref^{-1} E_f with E_f[a][c] = int_f phi_a psi_c (exact: degree pk + pt <= 2 pt + 1)
  std::vector<double> Mref(Np * Np, 0.0);
  for (int g = 0; g < NG; ++g)
    for (int a = 0; a < Np; ++a)
      for (int b = 0; b < Np; ++b) Mref[a * Np + b] += T.W[g] * T.Phi[g * Np + a] * T.Phi[g * Np + b];
  std::vector<double> L(nF * Np * Nft);
  for (int f = 0; f < nF; ++f) {
    std::vector<double> E(Np * Nft, 0.0);
    for (int q = 0; q < NGF; ++q)
      for (int a = 0; a < Np; ++a)
        for (int c = 0; c < Nft; ++c)
          E[a * Nft + c] += T.WF[q] * T.PhiF[(f * NGF + q) * Np + a] * T.PsiF[(f * NGF + q) * Nft + c];
    dense_solve(Mref, E, Np, Nft);
    for (int i = 0; i < Np * Nft; ++i) L[f * Np * Nft + i] = E[i];
  }
  T.PL.assign(nF * NG * Nft, 0.0);
  for (int f = 0; f < nF; ++f)
    for (int g = 0; g < NG; ++g)
      for (int c = 0; c < Nft; ++c) {
        double s = 0.0;
        for (int b = 0; b < Np; ++b) s += T.Phi[g * Np + b] * L[(f * Np + b) * Nft + c];
        T.PL[(f * NG + g) * Nft + c] = s;
      }
  T.PLF.assign(nF * nF * NGF * Nft, 0.0);
  for (int f = 0; f < nF; ++f)
    for (int fl = 0; fl < nF; ++fl)
      for (int g = 0; g < NGF; ++g)
        for (int c = 0; c < Nft; ++c) {
          double s = 0.0;
          for (int b = 0; b < Np; ++b) s += T.PhiF[(f * NGF + g) * Np + b] * L[(fl * Np + b) * Nft + c];
          T.PLF[((f * nF + fl) * NGF + g) * Nft + c] = s;
        }
  // the lift of the trace of element function b on face fl: sum_c PL(., c) phi_b(x_c)
  T.PLV.assign(nF * NG * Np, 0.0);
  for (int f = 0; f < nF; ++f)
    for (int g = 0; g < NG; ++g)
      for (int b = 0; b < Np; ++b) {
        double s = 0.0;
        for (int c = 0; c < Nft; ++c) s += T.PL[(f * NG + g) * Nft + c] * T.PhiN[(f * Nft + c) * Np + b];
        T.PLV[(f * NG + g) * Np + b] = s;
      }
  T.PLFV.assign(nF * nF * NGF * Np, 0.0);
  for (int f = 0; f < nF; ++f)
    for (int fl = 0; fl < nF; ++fl)
      for (int g = 0; g < NGF; ++g)
        for (int b = 0; b < Np; ++b) {
          double s = 0.0;
          for (int c = 0; c < Nft; ++c)
            s += T.PLF[((f * nF + fl) * NGF + g) * Nft + c] * T.PhiN[(fl * Nft + c) * Np + b];
          T.PLFV[((f * nF + fl) * NGF + g) * Np + b] = s;
        }
  // prolongation of the degree-q trace nodes of face f to its degree-pt nodes:
  // IPro[q-1][f][c][c'] = psi^q_{c'}(x^pt_c) (zero for c' beyond the degree-q face nodes)
  T.IPro.assign((size_t)pt * nF * Nft * Nft, 0.0);
  for (int q = 1; q <= pt; ++q) {
    const RefElement rq = make_refel(dim, q, q + 1);
    std::vector<double> x(d), vals(rq.Np);
    for (int f = 0; f < nF; ++f)
      for (int c = 0; c < Nft; ++c) {
        node_x(rt, rt.face_nodes[f][c], x.data());
        rq.eval(x.data(), 1, vals.data(), nullptr);
        for (int cq = 0; cq < rq.Nf; ++cq)
          T.IPro[(((size_t)(q - 1) * nF + f) * Nft + c) * Nft + cq] = vals[rq.face_nodes[f][cq]];
      }
  }
  return T;
}

}  // namespace hdg
