// Periodic simplex meshes (host side): Kuhn split of an n^d Cartesian grid,
// faces, face-node matching and affine element geometry.
//
// Sec. 3.1.1 of the paper defines the mesh T_h, its faces and the skeleton; Sec. 3.4
// assumes about 2 N_v triangles / 6 N_v tetrahedra. The split itself is not given;
// this library uses the Kuhn (Freudenthal) split, the same in every cell, which is
// conforming under periodic identification:
//   2D: cell (i,j), c = j n + i, triangles (00,10,11), (00,11,01); e = 2c + t.
//   3D: cell (i,j,k), c = (k n + j) n + i, for each axis permutation s in lexicographic
//       order the tetrahedron 0, e_s0, e_s0+e_s1, (1,1,1), with vertices 1 and 2
//       swapped when the determinant is negative; e = 6c + t.
// Global faces are numbered in order of first appearance over (element, local face);
// the first element is the owner and its face-node order is the canonical one.
// An axis is periodic (faces on its two sides identified) or bounded: then the faces on
// its sides have one side each (face_side[2F+1] = -1) and carry the boundary type of
// their side (face_bc, HDG_BC_*).
#pragma once
#include <cstdint>
#include <vector>

#include "refel.hpp"

namespace hdg {

struct Mesh {
  int dim = 0, p = 0, K = 0;
  int64_t n[3] = {0, 0, 0};
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int64_t E = 0, nFaces = 0;
  RefElement ref;
  std::vector<int64_t> lat;        // [E][nF][dim] integer vertex lattice coordinates
  std::vector<int32_t> face_of;    // [E][nF]
  std::vector<int32_t> fnode_map;  // [E][nF][Nf] canonical face-node index
  std::vector<int32_t> face_side;  // [F][2] = e * nF + f of the two sides (owner first; -1: boundary)
  int bc[3][2] = {{0, 0}, {0, 0}, {0, 0}};  // per axis, (lo, hi) boundary type; 0 = periodic
  std::vector<int8_t> face_bc;     // [F] boundary type of the face (0: interior)
  int64_t n_boundary = 0;          // faces with one side
  std::vector<double> geo;         // [E][geo_stride]: Jinv (dim*dim, [r][k]), |det J|,
                                   //   per face: normal (dim), face_jac (1)
  int geo_stride = 0;
  std::vector<double> xnode;       // [E][Np][dim] node coordinates
  std::vector<double> xfnode;      // [F][Nf][dim] canonical face-node coordinates (owner)
  // EDG trace space (Sec. 3.4, E^E_h = all faces): one unknown per skeleton node, numbered in
  // order of first appearance over (element, local face, face node); empty for HDG
  int scheme = 0;                  // HDG_SCHEME_*
  int64_t n_edg = 0;
  std::vector<int32_t> edg_index;  // [E][nF][Nf] skeleton node of each local face node
  std::vector<double> xedg;        // [n_edg][dim] node coordinates (first appearance)
  // Mixed degrees (not in the paper, which uses one degree): element e has degree pe[e], the
  // trace on face F the larger degree of its two sides, fdeg[F] = max(p_L, p_R), with the face
  // nodes of the degree-fdeg reference element; trace node of canonical face node c of face F:
  // fnoff[F] + c. Empty for a mesh of one degree (then p is that degree; otherwise the largest).
  std::vector<int8_t> pe;          // [E]
  std::vector<int8_t> fdeg;        // [F]
  std::vector<int8_t> ptr;         // [E] trace degree of the element: the largest of its faces
  std::vector<int64_t> fnoff;      // [F + 1]
  std::vector<int32_t> fnode_mix;  // [E][nF][Nf(p)] canonical face node of each local face node
                                   //   at the face's degree; -1 beyond that face's node count
  // packed per-element layout of a mixed-degree mesh, offsets [E + 1] in doubles: V and hist
  // (np_e m), g (nt_e = sum_f Nf(q_f) m), S (nt_e^2), recov (nv_e nt_e + nv_e), R (nv_e + nt_e)
  std::vector<int64_t> voff, toff, soff, roff, Roff;
  std::vector<double> xnode_mix;   // [sum_e Np_e][dim] element nodes at the element's degree
  std::vector<double> xfnode_mix;  // [trace nodes][dim] face nodes at the face's degree (owner side)
};

// Returns 0 on success; -1 on invalid arguments. bc: per axis (lo, hi) boundary type
// (HDG_BC_*), or null for all periodic; an axis is periodic on both sides or on neither.
int build_mesh(int dim, const int64_t n[3], const double lo[3], const double hi[3], int p, int K, Mesh& m,
               const int32_t* bc = nullptr);
// The continuous numbering of the skeleton nodes of a built mesh (Sec. 3.4): identifies the face
// nodes of all elements by their integer coordinates (modulo the period on periodic axes), in
// order of first appearance over (element, local face, face node). EDG: every face takes part;
// IEDG (interior_only): the nodes of each boundary face are its own, shared with no other face.
void build_edg(Mesh& m, bool interior_only);
// The mixed-degree data of a periodic HDG mesh built with p = the largest degree in pe.
// Returns 0 on success; -1 on invalid degrees.
int build_mixed(Mesh& m, const int8_t* pe);

}  // namespace hdg
