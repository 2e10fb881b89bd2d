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

// Tables of one element class of a mixed-degree mesh: element degree pk (volume rule with
// pk + 1 points per direction) and trace degree pt >= pk (face rule with pt + 1 points per
// direction; the trace space on face f is the nodal space of degree pt on that face, in the
// face-node order of the degree-pt reference element). With pt = pk the tables equal
// make_tables(make_refel(dim, pk, pk + 1)) (fnodes aside).
struct ClassTables {
  int dim, pk, pt, Np, Nfk, Nft, nF, NG, NGF;
  std::vector<double> W;      // [NG]
  std::vector<double> Phi;    // [NG][Np]
  std::vector<double> dPhi;   // [dim][NG][Np]
  std::vector<double> WF;     // [NGF]
  std::vector<double> PhiF;   // [nF][NGF][Np]       element basis at face-f points
  std::vector<double> dPhiF;  // [nF][dim][NGF][Np]
  std::vector<double> PsiF;   // [nF][NGF][Nft]      trace basis (degree pt) at face-f points
  std::vector<double> PhiN;   // [nF][Nft][Np]       element basis at the trace nodes of face f
  std::vector<double> PL;     // [nF][NG][Nft]       volume values of the lift of trace function c
  std::vector<double> PLF;    // [nF(points)][nF(lift)][NGF][Nft]
  std::vector<double> PLV;    // [nF][NG][Np]        lift of the trace of element function b
  std::vector<double> PLFV;   // [nF(points)][nF(lift)][NGF][Np]
  std::vector<double> IPro;   // [pt][nF][Nft][Nft]  degree-q trace nodes -> degree-pt nodes (q = 1..pt)
  std::vector<int> fnodesK;   // [nF][Nfk]           element nodes on face f
};

ClassTables make_class_tables(int dim, int pk, int pt);

}  // namespace hdg
