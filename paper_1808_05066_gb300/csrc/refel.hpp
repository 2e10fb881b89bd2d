// Reference simplex tables for the GPU path (host side).
//
// The paper fixes the spaces (full P_k on the reference simplex, Sec. 3.1.2) but not
// the basis or the quadrature. This library uses:
//   * nodal Lagrange basis on equispaced nodes, lexicographic with i fastest, evaluated
//     by Silvester's barycentric product formula;
//   * collapsed Gauss-Jacobi rules with K points per direction (exact to degree 2K-1);
//     the 1D rules are found by Newton iteration on the Jacobi polynomial;
//   * local face f = the face opposite reference vertex f; face nodes in increasing
//     element-node order; the trace basis on face f is the element basis restricted
//     to that face.
#pragma once
#include <vector>

namespace hdg {

struct Rule {
  std::vector<double> x;  // [n * dim]
  std::vector<double> w;  // [n]
  int n = 0, dim = 0;
};

// n-point Gauss-Jacobi rule on [-1, 1] for the weight (1-x)^a (1+x)^b.
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);
// Rule on the unit simplex {r_i >= 0, sum r_i <= 1}; dim = 1 is [0, 1].
Rule simplex_rule(int dim, int k);

struct RefElement {
  int dim = 0, p = 0, K = 0;
  int Np = 0, Nf = 0, nF = 0, NG = 0, NGF = 0;
  std::vector<int> idx;                 // [Np * dim] lattice multi-indices
  std::vector<std::vector<int>> face_nodes;  // [nF][Nf]
  Rule vol, face;                       // reference rules
  std::vector<std::vector<double>> fqp; // [nF][NGF * dim] face rule mapped into face f

  // Lagrange basis values / reference gradients at points x [npts * dim]
  void eval(const double* x, int npts, double* phi /*[npts*Np]*/, double* dphi /*[npts*Np*dim] or null*/) const;
};

RefElement make_refel(int dim, int p, int K);

// Device tables for one (dim, p, K), all row-major, double precision.
struct RefTables {
  int dim, p, K, Np, Nf, nF, NG, NGF;
  std::vector<double> W;      // [NG]            reference volume weights
  std::vector<double> Phi;    // [NG][Np]
  std::vector<double> dPhi;   // [dim][NG][Np]   reference gradients
  std::vector<double> PL;     // [nF][NG][Nf]    volume values of the face lifts
  std::vector<double> WF;     // [NGF]           reference face weights (parameter simplex)
  std::vector<double> PhiF;   // [nF][NGF][Np]   element basis at face-f points
  std::vector<double> dPhiF;  // [nF][dim][NGF][Np]
  std::vector<double> PLF;    // [nF(face pts)][nF(lift)][NGF][Nf]
  std::vector<double> Mref;   // [Np][Np] reference mass matrix
  std::vector<int> fnodes;    // [nF][Nf] element node of face node c
};

RefTables make_tables(const RefElement& r);

}  // namespace hdg
