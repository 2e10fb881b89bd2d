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
};

// Returns 0 on success; -1 on invalid arguments. bc: per axis (lo, hi) boundary type
// (HDG_BC_*), or null for all periodic; an axis is periodic on both sides or on neither.
int build_mesh(int dim, const int64_t n[3], const double lo[3], const double hi[3], int p, int K, Mesh& m,
               const int32_t* bc = nullptr);
// The continuous (EDG) numbering of the skeleton nodes of a built mesh: identifies the face
// nodes of all elements by their integer coordinates modulo the period.
void build_edg(Mesh& m);

}  // namespace hdg
