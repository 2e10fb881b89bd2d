// Kuhn-split simplex meshes, periodic or bounded per axis; see mesh.hpp for the numbering rules.
#include "mesh.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>

namespace hdg {

namespace {

using V3 = std::array<int64_t, 3>;

int64_t pmod(int64_t a, int64_t n) {
  int64_t r = a % n;
  return r < 0 ? r + n : r;
}

}  // namespace

int build_mesh(int dim, const int64_t n_[3], const double lo_[3], const double hi_[3], int p, int K, Mesh& m,
               const int32_t* bc) {
  if (dim != 2 && dim != 3) return -1;
  if (p < 1 || p > 6 || K < 1) return -1;
  for (int r = 0; r < dim; ++r)
    if (n_[r] < 1 || !(hi_[r] > lo_[r])) return -1;
  m = Mesh();
  if (bc)
    for (int r = 0; r < dim; ++r) {
      for (int s = 0; s < 2; ++s) {
        if (bc[2 * r + s] < 0 || bc[2 * r + s] > 2) return -1;
        m.bc[r][s] = bc[2 * r + s];
      }
      if ((m.bc[r][0] == 0) != (m.bc[r][1] == 0)) return -1;
    }
  m.dim = dim;
  m.p = p;
  m.K = K;
  for (int r = 0; r < 3; ++r) {
    m.n[r] = r < dim ? n_[r] : 1;
    m.lo[r] = r < dim ? lo_[r] : 0.0;
    m.hi[r] = r < dim ? hi_[r] : 1.0;
  }
  m.ref = make_refel(dim, p, K);
  const RefElement& ref = m.ref;
  const int nF = ref.nF, Nf = ref.Nf, Np = ref.Np;

  // element vertices on the integer lattice
  std::vector<std::array<V3, 4>> verts;
  if (dim == 2) {
    const int tri[2][3][2] = {{{0, 0}, {1, 0}, {1, 1}}, {{0, 0}, {1, 1}, {0, 1}}};
    for (int64_t j = 0; j < m.n[1]; ++j)
      for (int64_t i = 0; i < m.n[0]; ++i)
        for (int t = 0; t < 2; ++t) {
          std::array<V3, 4> vs{};
          for (int v = 0; v < 3; ++v) vs[v] = {i + tri[t][v][0], j + tri[t][v][1], 0};
          verts.push_back(vs);
        }
  } else {
    int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int64_t k = 0; k < m.n[2]; ++k)
      for (int64_t j = 0; j < m.n[1]; ++j)
        for (int64_t i = 0; i < m.n[0]; ++i)
          for (int t = 0; t < 6; ++t) {
            V3 P[4] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 1}};
            P[1][perm[t][0]] = 1;
            P[2] = P[1];
            P[2][perm[t][1]] = 1;
            // orientation: det [P1; P2; P3]
            int64_t det = P[1][0] * (P[2][1] * P[3][2] - P[2][2] * P[3][1]) -
                          P[1][1] * (P[2][0] * P[3][2] - P[2][2] * P[3][0]) +
                          P[1][2] * (P[2][0] * P[3][1] - P[2][1] * P[3][0]);
            if (det < 0) std::swap(P[1], P[2]);
            std::array<V3, 4> vs{};
            for (int v = 0; v < 4; ++v) vs[v] = {i + P[v][0], j + P[v][1], k + P[v][2]};
            verts.push_back(vs);
          }
  }
  m.E = (int64_t)verts.size();
  const int64_t E = m.E;
  m.lat.resize(E * nF * dim);
  for (int64_t e = 0; e < E; ++e)
    for (int v = 0; v < nF; ++v)
      for (int r = 0; r < dim; ++r) m.lat[(e * nF + v) * dim + r] = verts[e][v][r];

  double h[3];
  for (int r = 0; r < 3; ++r) h[r] = (m.hi[r] - m.lo[r]) / (double)m.n[r];

  // faces: key = (smallest vertex mod n, offsets of the other vertices)
  std::map<std::array<int64_t, 9>, int32_t> key2id;
  m.face_of.assign(E * nF, -1);
  std::vector<std::vector<int32_t>> sides;
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < nF; ++f) {
      std::vector<V3> fv;
      for (int v = 0; v < nF; ++v)
        if (v != f) fv.push_back(verts[e][v]);
      std::sort(fv.begin(), fv.end());
      std::array<int64_t, 9> key{};
      for (int r = 0; r < 3; ++r) key[r] = m.bc[r][0] == 0 ? pmod(fv[0][r], m.n[r]) : fv[0][r];
      for (size_t i = 1; i < fv.size(); ++i)
        for (int r = 0; r < 3; ++r) key[3 * i + r] = fv[i][r] - fv[0][r];
      auto it = key2id.find(key);
      int32_t id;
      if (it == key2id.end()) {
        id = (int32_t)sides.size();
        key2id.emplace(key, id);
        sides.emplace_back();
      } else {
        id = it->second;
      }
      sides[id].push_back((int32_t)(e * nF + f));
      m.face_of[e * nF + f] = id;
    }
  m.nFaces = (int64_t)sides.size();
  m.face_side.resize(m.nFaces * 2);
  m.face_bc.assign(m.nFaces, 0);
  for (int64_t F = 0; F < m.nFaces; ++F) {
    if (sides[F].size() == 2) {
      m.face_side[2 * F] = sides[F][0];
      m.face_side[2 * F + 1] = sides[F][1];
      continue;
    }
    if (sides[F].size() != 1) return -2;
    // a face with one side: all its vertices on one side of a bounded axis
    const int64_t e = sides[F][0] / nF;
    const int f = sides[F][0] % nF;
    int kind = -1;
    for (int r = 0; r < dim; ++r) {
      if (m.bc[r][0] == 0) continue;
      for (int s = 0; s < 2; ++s) {
        bool on = true;
        for (int v = 0; v < nF; ++v)
          if (v != f && verts[e][v][r] != (s == 0 ? 0 : m.n[r])) on = false;
        if (on) {
          if (kind >= 0) return -2;
          kind = m.bc[r][s];
        }
      }
    }
    if (kind <= 0) return -2;
    m.face_side[2 * F] = sides[F][0];
    m.face_side[2 * F + 1] = -1;
    m.face_bc[F] = (int8_t)kind;
    ++m.n_boundary;
  }

  // integer node coordinates (units h/p) and face-node matching relative to the
  // face's smallest vertex (periodic copies differ by a translation)
  auto node_int = [&](int64_t e, int a, int r) -> int64_t {
    int64_t x = p * verts[e][0][r];
    for (int s = 0; s < dim; ++s) x += (verts[e][s + 1][r] - verts[e][0][r]) * ref.idx[a * dim + s];
    return x;
  };
  auto face_min = [&](int64_t e, int f) {
    V3 best{};
    bool first = true;
    for (int v = 0; v < nF; ++v) {
      if (v == f) continue;
      if (first || verts[e][v] < best) best = verts[e][v];
      first = false;
    }
    return best;
  };
  m.fnode_map.assign(E * nF * Nf, -1);
  for (int64_t F = 0; F < m.nFaces; ++F) {
    int64_t e0 = m.face_side[2 * F] / nF;
    int f0 = m.face_side[2 * F] % nF;
    V3 A0 = face_min(e0, f0);
    std::map<V3, int> pos;
    for (int c = 0; c < Nf; ++c) {
      int a = ref.face_nodes[f0][c];
      V3 key{};
      for (int r = 0; r < dim; ++r) key[r] = node_int(e0, a, r) - p * A0[r];
      pos[key] = c;
    }
    if ((int)pos.size() != Nf) return -3;
    for (int s = 0; s < 2; ++s) {
      if (m.face_side[2 * F + s] < 0) continue;
      int64_t e = m.face_side[2 * F + s] / nF;
      int f = m.face_side[2 * F + s] % nF;
      V3 A = face_min(e, f);
      for (int c = 0; c < Nf; ++c) {
        int a = ref.face_nodes[f][c];
        V3 key{};
        for (int r = 0; r < dim; ++r) key[r] = node_int(e, a, r) - p * A[r];
        auto it = pos.find(key);
        if (it == pos.end()) return -4;
        m.fnode_map[(e * nF + f) * Nf + c] = it->second;
      }
    }
  }

  // affine geometry
  m.geo_stride = dim * dim + 1 + nF * (dim + 1);
  m.geo.assign(E * m.geo_stride, 0.0);
  m.xnode.assign(E * Np * dim, 0.0);
  const double param_measure = dim == 2 ? 1.0 : 0.5;
  for (int64_t e = 0; e < E; ++e) {
    double X[4][3];
    for (int v = 0; v < nF; ++v)
      for (int r = 0; r < dim; ++r) X[v][r] = m.lo[r] + h[r] * (double)verts[e][v][r];
    double J[3][3];  // columns X_s - X_0
    for (int r = 0; r < dim; ++r)
      for (int s = 0; s < dim; ++s) J[r][s] = X[s + 1][r] - X[0][r];
    double det, Ji[3][3];
    if (dim == 2) {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      Ji[0][0] = J[1][1] / det;
      Ji[0][1] = -J[0][1] / det;
      Ji[1][0] = -J[1][0] / det;
      Ji[1][1] = J[0][0] / det;
    } else {
      det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
            J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
      Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
      Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    }
    double* G = &m.geo[e * m.geo_stride];
    // Jinv stored as [r][k] = d r / d x_k
    for (int r = 0; r < dim; ++r)
      for (int k = 0; k < dim; ++k) G[r * dim + k] = Ji[r][k];
    G[dim * dim] = std::fabs(det);
    for (int f = 0; f < nF; ++f) {
      double Y[3][3];
      int nv = 0;
      for (int v = 0; v < nF; ++v) {
        if (v == f) continue;
        for (int r = 0; r < dim; ++r) Y[nv][r] = X[v][r];
        ++nv;
      }
      double nrm[3] = {0, 0, 0}, area;
      if (dim == 2) {
        double t0 = Y[1][0] - Y[0][0], t1 = Y[1][1] - Y[0][1];
        nrm[0] = t1;
        nrm[1] = -t0;
        area = std::sqrt(t0 * t0 + t1 * t1);
      } else {
        double a[3], b[3];
        for (int r = 0; r < 3; ++r) {
          a[r] = Y[1][r] - Y[0][r];
          b[r] = Y[2][r] - Y[0][r];
        }
        nrm[0] = a[1] * b[2] - a[2] * b[1];
        nrm[1] = a[2] * b[0] - a[0] * b[2];
        nrm[2] = a[0] * b[1] - a[1] * b[0];
        area = 0.5 * std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
      }
      double len = 0.0, dot = 0.0;
      for (int r = 0; r < dim; ++r) len += nrm[r] * nrm[r];
      len = std::sqrt(len);
      for (int r = 0; r < dim; ++r) {
        nrm[r] /= len;
        dot += nrm[r] * (X[f][r] - Y[0][r]);
      }
      if (dot > 0)
        for (int r = 0; r < dim; ++r) nrm[r] = -nrm[r];
      double* Gf = G + dim * dim + 1 + f * (dim + 1);
      for (int r = 0; r < dim; ++r) Gf[r] = nrm[r];
      Gf[dim] = area / param_measure;
    }
    for (int a = 0; a < Np; ++a)
      for (int r = 0; r < dim; ++r) {
        double x = X[0][r];
        for (int s = 0; s < dim; ++s) x += J[r][s] * (double)ref.idx[a * dim + s] / (double)p;
        m.xnode[(e * Np + a) * dim + r] = x;
      }
  }
  m.xfnode.assign(m.nFaces * Nf * dim, 0.0);
  for (int64_t F = 0; F < m.nFaces; ++F) {
    int64_t e0 = m.face_side[2 * F] / nF;
    int f0 = m.face_side[2 * F] % nF;
    for (int c = 0; c < Nf; ++c) {
      int a = ref.face_nodes[f0][c];
      for (int r = 0; r < dim; ++r) m.xfnode[(F * Nf + c) * dim + r] = m.xnode[(e0 * Np + a) * dim + r];
    }
  }
  return 0;
}

void build_edg(Mesh& m, bool interior_only) {
  const RefElement& ref = m.ref;
  const int dim = m.dim, nF = ref.nF, Nf = ref.Nf, Np = ref.Np, p = m.p;
  std::map<V3, int32_t> ids;
  int32_t next = 0;
  m.edg_index.assign(m.E * nF * Nf, -1);
  m.xedg.clear();
  for (int64_t e = 0; e < m.E; ++e)
    for (int f = 0; f < nF; ++f) {
      // IEDG: a face on the boundary keeps its own nodes (only one element visits it)
      const bool own = interior_only && m.face_bc[m.face_of[e * nF + f]] != 0;
      for (int c = 0; c < Nf; ++c) {
        const int a = ref.face_nodes[f][c];
        int32_t id;
        bool fresh = own;
        if (own) {
          id = next++;
        } else {
          V3 key{};
          for (int r = 0; r < dim; ++r) {  // integer coordinates (units h/p), modulo the period if periodic
            const int64_t* L = &m.lat[(e * nF) * dim];
            int64_t x = p * L[r];
            for (int s = 0; s < dim; ++s) x += (L[(s + 1) * dim + r] - L[r]) * ref.idx[a * dim + s];
            key[r] = m.bc[r][0] == 0 ? pmod(x, p * m.n[r]) : x;
          }
          auto it = ids.find(key);
          if (it == ids.end()) {
            id = next++;
            ids.emplace(key, id);
            fresh = true;
          } else {
            id = it->second;
          }
        }
        if (fresh)
          for (int r = 0; r < dim; ++r) m.xedg.push_back(m.xnode[(e * Np + a) * dim + r]);
        m.edg_index[(e * nF + f) * Nf + c] = id;
      }
    }
  m.n_edg = (int64_t)next;
}

int build_mixed(Mesh& m, const int8_t* pe_in) {
  const int dim = m.dim, nF = m.ref.nF, NfMax = m.ref.Nf;
  const int64_t E = m.E, F = m.nFaces;
  m.pe.assign(pe_in, pe_in + E);
  for (int8_t q : m.pe)
    if (q < 1 || q > m.p) return -1;
  m.fdeg.assign(F, 0);
  for (int64_t Fi = 0; Fi < F; ++Fi)
    for (int s = 0; s < 2; ++s) {
      const int32_t ef = m.face_side[2 * Fi + s];
      if (ef >= 0) m.fdeg[Fi] = std::max(m.fdeg[Fi], m.pe[ef / nF]);
    }
  m.ptr.assign(E, 0);
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < nF; ++f) m.ptr[e] = std::max(m.ptr[e], m.fdeg[m.face_of[e * nF + f]]);
  std::vector<RefElement> rq(m.p + 1);
  for (int q = 1; q <= m.p; ++q) rq[q] = make_refel(dim, q, q + 1);
  m.fnoff.assign(F + 1, 0);
  for (int64_t Fi = 0; Fi < F; ++Fi) m.fnoff[Fi + 1] = m.fnoff[Fi] + rq[m.fdeg[Fi]].Nf;
  // lattice vertices of element e (units h)
  auto vtx = [&](int64_t e, int v, int r) { return m.lat[(e * nF + v) * dim + r]; };
  // integer coordinates (units h/q) of node a of the degree-q element e, relative to q A
  auto node_rel = [&](int64_t e, const RefElement& r, int a, const V3& A, V3& out) {
    const int q = r.p;
    for (int s = 0; s < dim; ++s) {
      int64_t x = q * vtx(e, 0, s);
      for (int t = 0; t < dim; ++t) x += (vtx(e, t + 1, s) - vtx(e, 0, s)) * r.idx[a * dim + t];
      out[s] = x - q * A[s];
    }
    for (int s = dim; s < 3; ++s) out[s] = 0;
  };
  auto face_min = [&](int64_t e, int f) {
    V3 best{};
    bool first = true;
    for (int v = 0; v < nF; ++v) {
      if (v == f) continue;
      V3 x{};
      for (int s = 0; s < dim; ++s) x[s] = vtx(e, v, s);
      if (first || x < best) best = x;
      first = false;
    }
    return best;
  };
  m.fnode_mix.assign(E * nF * NfMax, -1);
  for (int64_t Fi = 0; Fi < F; ++Fi) {
    const RefElement& r = rq[m.fdeg[Fi]];
    const int32_t ef0 = m.face_side[2 * Fi];
    const int64_t e0 = ef0 / nF;
    const int f0 = ef0 % nF;
    const V3 A0 = face_min(e0, f0);
    std::map<V3, int> pos;
    for (int c = 0; c < r.Nf; ++c) {
      V3 key{};
      node_rel(e0, r, r.face_nodes[f0][c], A0, key);
      pos[key] = c;
    }
    if ((int)pos.size() != r.Nf) return -3;
    for (int s = 0; s < 2; ++s) {
      const int32_t ef = m.face_side[2 * Fi + s];
      if (ef < 0) continue;
      const int64_t e = ef / nF;
      const int f = ef % nF;
      const V3 A = face_min(e, f);
      for (int c = 0; c < r.Nf; ++c) {
        V3 key{};
        node_rel(e, r, r.face_nodes[f][c], A, key);
        auto it = pos.find(key);
        if (it == pos.end()) return -4;
        m.fnode_mix[(e * nF + f) * NfMax + c] = it->second;
      }
    }
  }
  const int M = dim + 2;
  m.voff.assign(E + 1, 0);
  m.toff.assign(E + 1, 0);
  m.soff.assign(E + 1, 0);
  m.roff.assign(E + 1, 0);
  m.Roff.assign(E + 1, 0);
  for (int64_t e = 0; e < E; ++e) {
    int64_t nt = 0;
    for (int f = 0; f < nF; ++f) nt += (int64_t)rq[m.fdeg[m.face_of[e * nF + f]]].Nf * M;
    const int64_t nv = (int64_t)rq[m.pe[e]].Np * M;
    m.voff[e + 1] = m.voff[e] + nv;
    m.toff[e + 1] = m.toff[e] + nt;
    m.soff[e + 1] = m.soff[e] + nt * nt;
    m.roff[e + 1] = m.roff[e] + nv * nt + nv;
    m.Roff[e + 1] = m.Roff[e] + nv + nt;
  }
  // node coordinates: x = X_0 + J idx / q for the lattice multi-index idx of degree q
  auto node_x = [&](int64_t e, const RefElement& r, int a, double* x) {
    for (int s = 0; s < dim; ++s) {
      const double h = (m.hi[s] - m.lo[s]) / (double)m.n[s];
      double v = m.lo[s] + h * (double)vtx(e, 0, s);
      for (int t = 0; t < dim; ++t) v += h * (double)(vtx(e, t + 1, s) - vtx(e, 0, s)) * r.idx[a * dim + t] / r.p;
      x[s] = v;
    }
  };
  m.xnode_mix.assign(m.voff.back() / M * dim, 0.0);
  for (int64_t e = 0; e < E; ++e) {
    const RefElement& r = rq[m.pe[e]];
    for (int a = 0; a < r.Np; ++a) node_x(e, r, a, &m.xnode_mix[(m.voff[e] / M + a) * dim]);
  }
  m.xfnode_mix.assign(m.fnoff.back() * dim, 0.0);
  for (int64_t Fi = 0; Fi < F; ++Fi) {
    const RefElement& r = rq[m.fdeg[Fi]];
    const int64_t e0 = m.face_side[2 * Fi] / nF;
    const int f0 = m.face_side[2 * Fi] % nF;
    for (int c = 0; c < r.Nf; ++c) node_x(e0, r, r.face_nodes[f0][c], &m.xfnode_mix[(m.fnoff[Fi] + c) * dim]);
  }
  return 0;
}

}  // namespace hdg
