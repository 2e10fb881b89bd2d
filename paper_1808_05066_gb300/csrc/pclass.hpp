// Mixed-degree meshes (elements of different degree in one mesh): the per-class device tables,
// the packed per-element layout and the work queue of the persistent assemble + condense launch
// (pclass.cu). The paper uses one degree; this is the library's extension.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

struct hdg_ctx;

namespace hdg {

constexpr int kPClasses = 10;  // (pk, pt) with 1 <= pk <= pt <= 4 (3D Navier-Stokes)

// sizes of one (pk, pt) class: nodes, points, unknowns, tiles, shared memory and per-CTA scratch
// (doubles) of the fused kernel
struct PDims {
  int pk, pt, NP, NFK, NFN, NG, NGF, NV, NT, NZ, GT, CB, RBMAX, ASM, CND, KEEP, SMEM, lu_smem;
  int64_t SLOT;
};

// device pointers of the tables of one (pk, pt) class (layouts of ClassTables, refel.hpp) and its sizes
struct PClassDev {
  const double *W, *Phi, *dPhi, *WF, *PhiF, *dPhiF, *PsiF, *PhiN, *PL, *PLF, *PLV, *PLFV, *IPro;
  const int* fnodesK;
  PDims d;
};

struct PMix {
  int pmin = 0, pmax = 0, nfn_max = 0;
  int64_t n_tnodes = 0;
  // device copies of the mesh's packed layout offsets (Mesh::voff ..)
  int64_t *d_voff = nullptr, *d_toff = nullptr, *d_soff = nullptr, *d_roff = nullptr, *d_Roff = nullptr;
  int* d_tgidx = nullptr;     // [E][NF][nfn_max] trace node of each local face node, -1 beyond
  int8_t* d_fdeg = nullptr;   // [E][NF]
  int8_t* d_cls = nullptr;    // [E] class index
  int* d_fnn = nullptr;       // [E][NF] own face nodes of each face of the element (Nf(q_f))
  int* d_occ_e = nullptr;     // [trace nodes][2] element of each side of the node's face (-1: none)
  int* d_occ_l = nullptr;     // [trace nodes][2] first unknown of the node in that element's trace vector
  int64_t* d_fnoff = nullptr; // [F + 1] first trace node of each face
  int64_t* d_pcoff = nullptr; // [F + 1] face-block preconditioner offsets (sum of B_F^2)
  int64_t pc_len = 0;         // doubles of the face-block preconditioner
  int nt_max = 0;             // largest element trace vector
  bool attr_face = false;
  int* d_queue = nullptr;     // [E] elements, largest class first
  int* d_counter = nullptr;   // work counter of the persistent launch
  double* d_tab = nullptr;
  int* d_itab = nullptr;
  PClassDev tab[kPClasses] = {};
  int64_t class_count[kPClasses] = {};
  size_t smem_bytes = 0;      // dynamic shared memory of the launch: the largest class present
  size_t smem_limit = 0;      // dynamic shared memory a CTA of the fused kernel may use on the device
  bool tuned = false;         // tile shapes (GT, CB) chosen per class by timing (first call)
  std::vector<int> h_queue;   // host copy of the queue
  std::vector<int8_t> h_cls;  // host copy of the classes
  int64_t slot_doubles = 0;   // per-CTA scratch: the largest class present
  bool attr_set = false;
};

// the device addressing of the packed layout, passed to the trace kernels by value
struct PMixDev {
  const int64_t *voff, *toff, *soff, *roff, *Roff, *fnoff, *pcoff;
  const int *tgidx, *fnn, *occ_e, *occ_l;
  const int8_t* cls;
  int nfn_max;
  PClassDev tab[kPClasses];
};

int pclass_index(int pk, int pt);
// class tables, layout and queue of a mixed-degree mesh; frees with pclass_free
int pclass_setup(hdg_ctx* c);
void pclass_free(PMix* pm);
PMixDev pmix_dev(const hdg_ctx* c);
// trace-space operations of pclass_trace.cu (the packed layout's counterparts of trace.cu); skip:
// a device flag that, when set, makes the launch return at once (a finished Krylov cycle)
int pm_history(hdg_ctx* c, const double* V0, const double* V1, double c0, double c1, double* hist, cudaStream_t s);
int pm_gather(hdg_ctx* c, const double* ge, double scale, double* out, cudaStream_t s, const int* skip = nullptr);
int pm_elem_matvec(hdg_ctx* c, const double* S, const double* x, double* w, cudaStream_t s,
                   const int* skip = nullptr);
int pm_recover(hdg_ctx* c, const double* recov, const double* dvh, double* dV, cudaStream_t s);
int pm_sumsq(hdg_ctx* c, const double* R, double* red, cudaStream_t s);
int pm_face_factor(hdg_ctx* c, const double* S, double* pc, cudaStream_t s);
int pm_face_apply(hdg_ctx* c, const double* pc, const double* r, double* z, cudaStream_t s,
                  const int* skip = nullptr);
int pm_dense_scatter(hdg_ctx* c, const double* S, int64_t n, double* K, cudaStream_t s);
int assemble_condense_pclass(hdg_ctx* c, const double* V, const double* Vhat, const double* hist, double mass_coef,
                             double* S, double* g, double* recov, double* R, int32_t* status, cudaStream_t s);

}  // namespace hdg
