/* C-ABI of the GB300 entropy-variable hybridized DG hot path.
 *
 * The method (Fernandez, Nguyen & Peraire, arXiv:1808.05066) discretises the
 * compressible Euler (Sec. 3.2, Eqs. hDG1-hDG3) and Navier-Stokes equations
 * (Sec. 3.3, Eqs. hDG_NS0-hDG_NS3) in entropy variables v with a hybrid trace vhat.
 * The local equations are eliminated element by element ("static condensation",
 * Sec. 3.2 last paragraph, Sec. 3.3) and only the trace unknowns are globally
 * coupled. This library implements, on simplex meshes of a Cartesian box (periodic or
 * bounded per axis; one degree, or elements of different degree) with the HDG trace space
 * (E^E_h empty) or the continuous EDG / IEDG trace spaces of Sec. 3.4:
 *   - the per-element Newton linearisation and condensation     hdg_assemble_condense
 *   - the global trace solve                                     hdg_trace_solve
 *   - the interior recovery                                      hdg_recover_interior
 *   - a full BDF Newton step around them                         hdg_newton_step
 *   - a DIRK(3,3) step (Sec. 5's integrator)                     hdg_dirk3_step
 * with, by default, the symmetric Lax-Friedrichs stabilisation sigma = lambda_max(vhat)
 * A0(vhat) (Eq. sLxF with v* = vhat, the choice of Sec. 5) in the inviscid flux of
 * Eq. numericalFlux and the viscous flux G(vhat, q) . n of Eq. numericalFluxNS_2; hdg_physics
 * selects sigma_S (Eq. symStab), the viscous flux of Eq. numericalFluxNS_1 and a power-law
 * viscosity (Sec. 5.6). Bounded axes take a given boundary state or a slip wall
 * (hdg_ctx_set_boundary_state), and a source term enters with the time history
 * (hdg_add_source), as in the steady exact-solution examples of Secs. 5.1-5.2.
 *
 * Conventions shared by all calls
 *   - m = d + 2 state components. Entropy variables (v_1, w_1..w_d, v_m), v_m < 0.
 *   - Nondimensionalisation: freestream density, speed and length are 1, so
 *     p_inf = 1/(gamma M^2), c_v = 1/(gamma (gamma-1) M^2), mu = 1/Re,
 *     kappa = gamma c_v mu / Pr, beta = 0.  reynolds == 0 selects Euler.
 *   - Every array argument of a compute call is a DEVICE pointer owned by the caller
 *     (the library never frees it); all are row-major double unless stated.
 *       V     [E][Np][m]        element nodal entropy variables
 *       Vhat  [F][Nf][m]        trace values at the canonical nodes of each face
 *       hist  [E][Np][m]        BDF history (sum_j c_j (u(v^{n-j}), phi_a)_K) plus any source
 *                               term (hdg_add_source), or NULL
 *       S     [E][nt][nt]       condensed trace matrix per element, nt = nF Nf m
 *       g     [E][nt]           condensed right-hand side per element
 *       recov [E][nv*nt + nv]   recovery data X = A^{-1}B (row-major nv x nt) then
 *                               y = A^{-1} R_v, nv = Np m
 *       R     [E][nv + nt]      raw residuals R_v then R_t (element contribution)
 *     Local trace order is [local face][face node][component]; local face f is the
 *     face opposite vertex f; face nodes in increasing element-node order.
 *   - stream is a cudaStream_t (NULL = legacy default stream). Calls enqueue work and
 *     return without synchronising unless they write a host scalar (iterations,
 *     norms), which they document.
 *   - Return value: HDG_OK or an HDG_ERR_* code; hdg_last_error() gives a message
 *     (thread-local, valid until the next call from the same thread).
 */
#ifndef HDG_H_
#define HDG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HDG_OK = 0,
  HDG_ERR_INVALID_ARG = 1,
  HDG_ERR_NONPHYSICAL = 2, /* some element has v_m >= 0 or non-positive rho / p  */
  HDG_ERR_SINGULAR = 3,    /* zero pivot in an element factorisation              */
  HDG_ERR_REFINE = 4,      /* iterative refinement did not reach its tolerance    */
  HDG_ERR_NOT_CONVERGED = 5, /* Newton or the trace solver missed its tolerance          */
  HDG_ERR_TIMEOUT = 6,       /* a bounded wait inside a kernel gave up (HDG_ELEM_TIMEOUT) */
  HDG_ERR_CUDA = 7,
  HDG_ERR_UNSUPPORTED = 8  /* (dim, p, quadrature, physics) not compiled in        */
};

enum { HDG_PREC_FP64 = 0, HDG_PREC_MIXED = 1 };
enum { HDG_SOLVER_AUTO = 0, HDG_SOLVER_GMRES = 1, HDG_SOLVER_DENSE = 2 };
/* trace spaces of Sec. 3.4: E^E_h empty (HDG), all faces (EDG), interior faces (IEDG) */
enum { HDG_SCHEME_HDG = 0, HDG_SCHEME_EDG = 1, HDG_SCHEME_IEDG = 2 };
/* per-element status bits written by hdg_assemble_condense:
 *   NONPHYSICAL  v_m >= 0 or non-positive rho / p at a quadrature point
 *   SINGULAR     zero pivot in the element factorisation
 *   REFINE       mixed form: the iterative refinement of X = A^{-1}[B | R_v] missed its
 *                tolerance (left set only when the FP64 recomputation is switched off)
 *   FP64         mixed form: the block missed the tolerance (or timed out) and was recomputed
 *                by the FP64 kernels (hdg_ctx_set_refinement); S, g, X, y are the FP64 form's
 *   TIMEOUT      mixed form, tcgen05 condensation: a bounded wait for its operands or its
 *                tensor-core products gave up (about a second); the kernel freed its tensor
 *                memory and returned, the context stays usable, and the block's outputs are
 *                invalid unless the FP64 recomputation replaced them (then FP64 is set instead) */
enum { HDG_ELEM_NONPHYSICAL = 1, HDG_ELEM_SINGULAR = 2, HDG_ELEM_REFINE = 4, HDG_ELEM_FP64 = 8,
       HDG_ELEM_TIMEOUT = 16 };

typedef struct hdg_mesh* hdg_mesh_t;
typedef struct hdg_ctx* hdg_ctx_t;

typedef struct {
  double gamma;       /* ratio of specific heats (1.4) */
  double mach;        /* reference Mach number M */
  double reynolds;    /* Re; 0 = inviscid (Euler) */
  double prandtl;     /* Pr */
  double mu_exponent; /* power law mu = (1/Re)(T/T_inf)^omega, kappa likewise (Sec. 5.6 uses 3/4;
                         T_inf = 1 in this nondimensionalisation); 0 = constant viscosity; 0..4 */
  int32_t visc_flux;  /* viscous numerical flux: 0 or 2 = G(vhat, q) . n (Eq. numericalFluxNS_2, the
                         choice of Sec. 5), 1 = G(v, q) . n (Eq. numericalFluxNS_1) */
  int32_t stabilization; /* stabilization matrix of Eq. numericalFlux at v* = vhat: HDG_STAB_SLF
                            (0, lambda_max A0 of Eq. sLxF, the choice of Sec. 5) or HDG_STAB_S (1,
                            |A_n| A0 of Eq. symStab with the absolute value of Sec. 4.1) */
} hdg_physics;

enum { HDG_STAB_SLF = 0, HDG_STAB_S = 1 };

typedef struct {
  int32_t dim, p, quad_points; /* quad_points K per direction: exact to degree 2K-1 */
  int32_t m, Np, Nf, nF, NG, NGF;
  int32_t nv, nt;              /* per-element interior / trace unknowns */
  int32_t geo_stride;
  int64_t n_elem, n_faces, n_trace; /* n_trace = n_trace_nodes * m */
  int32_t scheme;                   /* HDG_SCHEME_* */
  int64_t n_trace_nodes;            /* HDG: n_faces * Nf (a trace per face); EDG / IEDG: skeleton nodes */
  int64_t n_boundary_faces;         /* faces with one side (on the sides of bounded axes) */
  /* Elements of different degree (p_per_elem; the paper uses one degree): mixed != 0, p is the
   * largest degree, Np / Nf / nv / nt are those of degree p (the largest per-element sizes), and
   * the arrays of the compute calls are packed per element; their total lengths in doubles are
   * below (for a mesh of one degree they equal the uniform sizes E Np m, E nt, ...). */
  int32_t mixed, p_min;
  int64_t len_V, len_g, len_S, len_recov, len_R;
} hdg_mesh_info;

/* Boundary types of the sides of the box (the term b_h of Eqs. hDG2 / hDG_NS2, which the paper
 * leaves open, Sec. 3.2):
 *   HDG_BC_PERIODIC  the two sides of the axis are identified (no boundary);
 *   HDG_BC_STATE     b_h = vhat - v_b: the trace takes a given boundary state v_b (the prescribed
 *                    exact solutions of Secs. 5.1-5.2), set by hdg_ctx_set_boundary_state (EDG:
 *                    imposed strongly at the trace nodes of these faces);
 *   HDG_BC_SLIP      b_h = fhat(vhat, v; n) + fhat(vhat, R v; -n), R reflecting the momentum
 *                    components in the wall: the trace residual of an interior face whose other
 *                    side is the element's mirror image (a slip wall; Euler only). */
enum { HDG_BC_PERIODIC = 0, HDG_BC_STATE = 1, HDG_BC_SLIP = 2 };

/* Mesh T_h (Sec. 3.1.1): the n[0] x .. x n[dim-1] grid on the box [lo, hi], periodic or
 * bounded per axis, each cell split into 2 triangles / 6 tetrahedra (Kuhn split, the same in
 * every cell; element e = (cells in x-fastest order) x (2 or 6) + local index).
 *   p_per_elem  host array [E] of per-element degrees (1..4), or NULL for the uniform degree p.
 *               An array whose entries all equal p is the uniform mesh. Elements of different
 *               degree (an extension: the paper uses one degree k) give each face the larger
 *               degree of its two sides, q_F = max(p_L, p_R), with the nodes of the degree-q_F
 *               reference face; the trace unknowns are numbered face by face (face F's canonical
 *               node c is trace node face_node_off[F] + c, hdg_mesh_copy_layout), so Vhat is
 *               [trace nodes][m]. Such meshes are built periodic, HDG, with the default rules
 *               (quad_points 0: element degree + 1 points per direction in the volume, the
 *               element's largest face degree + 1 on its faces); the compute calls then take
 *               the packed per-element layout of hdg_mesh_copy_layout.
 *   p           polynomial degree k of Sec. 3.1.2 (1..4); ignored when p_per_elem is given. 3D p = 4
 *               (Navier-Stokes, FP64 form) runs on the element-class kernels of mixed-degree meshes,
 *               with the uniform layout.
 *   scheme      trace space of Sec. 3.4: HDG_SCHEME_HDG (one trace per face, Vhat [F][Nf][m]) or
 *               HDG_SCHEME_EDG (a continuous trace, one unknown per skeleton node, Vhat [N][m],
 *               nodes numbered in order of first appearance over (element, local face, face
 *               node)); HDG_SCHEME_IEDG continuous on the interior faces, each boundary face with
 *               nodes of its own (shared with no other face), which on periodic meshes (every
 *               face interior) is EDG. The local problem and the condensation are the same for
 *               all three; only the global trace numbering differs (and, on a bounded EDG mesh,
 *               the strongly imposed state of the boundary nodes, see bc).
 *   quad_points K Gauss-Jacobi points per direction, exact to degree 2K-1 (0 selects p+1).
 *   bc          host array [2 dim] of HDG_BC_* per axis (lo side, hi side), or NULL for a fully
 *               periodic mesh; an axis is periodic on both sides or on neither. Bounded meshes
 *               are built for all three schemes; the boundary state of an EDG / IEDG mesh is
 *               given at its trace nodes like Vhat. EDG's boundary nodes are shared with
 *               interior faces, so there the state is imposed strongly (the node's equation is
 *               vhat = v_b) and the slip wall is not built (HDG_ERR_UNSUPPORTED).
 * Host-only work; the mesh owns host arrays only (freed by hdg_mesh_destroy).
 * Errors: HDG_ERR_INVALID_ARG, HDG_ERR_UNSUPPORTED. */
int hdg_mesh_create(int dim, const int64_t n[3], const double lo[3], const double hi[3], const int8_t* p_per_elem,
                    int p, int scheme, int quad_points, const int32_t* bc, hdg_mesh_t* out);
void hdg_mesh_destroy(hdg_mesh_t mesh);
int hdg_mesh_get_info(hdg_mesh_t mesh, hdg_mesh_info* out);
/* Host copies of the topology: face_of [E][nF], fnode_map [E][nF][Nf] (canonical face
 * node of each local face node), face_side [F][2] (e * nF + f; owner first; -1 for the missing
 * side of a boundary face). Any pointer may be NULL. */
int hdg_mesh_copy_topology(hdg_mesh_t mesh, int32_t* face_of, int32_t* fnode_map, int32_t* face_side);
/* Host copy of the boundary type of every face, face_bc [F] (HDG_BC_*; 0 for interior faces). */
int hdg_mesh_copy_face_bc(hdg_mesh_t mesh, int8_t* face_bc);
/* Global trace node of every local face node, tnode [E][nF][Nf] (host): HDG face * Nf + canonical
 * face node; EDG / IEDG the skeleton node. The element's trace unknowns are Vhat[tnode][0..m).
 * Mixed degrees: Nf of the largest degree; face_node_off[F] + canonical node, -1 beyond the
 * nodes of the face's own degree. */
int hdg_mesh_copy_trace_map(hdg_mesh_t mesh, int32_t* tnode);
/* Packed per-element layout (host copies; any pointer may be NULL). Offsets [E + 1] in doubles
 * of element e's block in: V and hist (voff: [Np_e][m]), g (toff: nt_e = sum_f Nf(q_f) m),
 * S (soff: [nt_e][nt_e]), recov (roff: X [nv_e][nt_e] then y [nv_e]), R (Roff: R_v [nv_e] then
 * R_t [nt_e]); elem_p [E] element degrees, face_deg [F] face degrees, face_node_off [F + 1] first
 * trace node of each face. The local trace order is [local face][its own face nodes][component].
 * For a mesh of one degree the offsets are the uniform strides. Host-only. */
int hdg_mesh_copy_layout(hdg_mesh_t mesh, int64_t* voff, int64_t* toff, int64_t* soff, int64_t* roff, int64_t* Roff,
                         int8_t* elem_p, int8_t* face_deg, int64_t* face_node_off);
/* Host copies: element node coordinates xnode [E][Np][dim], trace-node coordinates xfnode
 * [n_trace_nodes][dim] (HDG: canonical face nodes [F][Nf], owner side; EDG: skeleton nodes),
 * geometry geo [E][geo_stride] =
 * (Jinv [dim][dim] with Jinv[r][k] = d r / d x_k, |det J|, per face: unit outward
 * normal [dim], surface Jacobian). Mixed degrees: xnode is packed [sum_e Np_e][dim] (each element's
 * nodes at its own degree), xfnode [trace nodes][dim] (each face's nodes at its degree, owner side).
 * Any pointer may be NULL. */
int hdg_mesh_copy_coords(hdg_mesh_t mesh, double* xnode, double* xfnode, double* geo);

/* Context: mesh tables, reference tables and physics on one CUDA device. Allocates the
 * device tables and (lazily, on first use) the internal scratch of the calls below;
 * everything is freed by hdg_ctx_destroy. The mesh must outlive the context.
 * Errors: HDG_ERR_INVALID_ARG (physics), HDG_ERR_UNSUPPORTED (configuration not compiled; slip
 * walls with viscous physics), HDG_ERR_CUDA. */
int hdg_ctx_create(hdg_mesh_t mesh, const hdg_physics* phys, int device, hdg_ctx_t* out);
void hdg_ctx_destroy(hdg_ctx_t ctx);

/* The boundary state v_b of the HDG_BC_STATE faces: Vb is a device array in the trace layout,
 * [n_faces][Nf][m] (HDG) or [n_trace_nodes][m] (EDG / IEDG), of which only the nodes of state
 * faces are read, copied on `stream` into the context (the caller may free or reuse Vb once
 * the stream passes the copy). Every later assembly reads
 * the copy, so a time-dependent state is set before each step. A mesh with state faces must have
 * its state set before the first assembly (else HDG_ERR_INVALID_ARG there).
 * Errors: HDG_ERR_INVALID_ARG (null), HDG_ERR_CUDA. */
int hdg_ctx_set_boundary_state(hdg_ctx_t ctx, const double* Vb, void* stream);

/* Mixed form only: tolerance of the refinement status bit and what happens to a flagged
 * block. A block is flagged when its last correction, squared over the one before it, is
 * above tol times the largest |X| entry (default tol 1e-10: the error left after the last
 * correction is about that ratio). With fp64_fallback (the default) the flagged elements
 * of each chunk are recomputed by the FP64 kernels on the same stream, without a host
 * synchronisation, and carry HDG_ELEM_FP64 instead of HDG_ELEM_REFINE; without it the bit
 * stays set and hdg_newton_solve / hdg_newton_step return HDG_ERR_REFINE. tol = 0 flags
 * every block whose last correction is not exactly zero. Errors: HDG_ERR_INVALID_ARG for
 * tol outside [0, 1). Drops a graph captured by hdg_assemble_condense_graph. */
int hdg_ctx_set_refinement(hdg_ctx_t ctx, double tol, int fp64_fallback);

/* Trace solver of the Newton iterations of hdg_newton_solve / hdg_newton_step: method as for
 * hdg_trace_solve (default HDG_SOLVER_AUTO), relative tolerance (default 1e-12) and iteration
 * limit (default 600). rtol = 0 selects an inexact Newton method: each trace solve stops at the
 * Eisenstat-Walker forcing term eta_k = 0.9 (|R_k|/|R_{k-1}|)^2 (safeguarded, at most 0.1, never
 * tighter than the nonlinear tolerance still requires); the converged state meets the same
 * Newton tolerance. Errors: HDG_ERR_INVALID_ARG (rtol outside [0, 1)). */
int hdg_ctx_set_trace_solver(hdg_ctx_t ctx, int method, double rtol, int max_it);

/* Entropy variables of Sec. 2.3, v = dH/du for H = -rho s: converts n_points primitive
 * states prim [n][m] = (rho, V_1..V_d, p) to v [n][m] (device). */
int hdg_prim_to_entropy(hdg_ctx_t ctx, const double* prim, int64_t n_points, double* v, void* stream);

/* BDF history of the time term of Eq. hDG1 / hDG_NS1:
 * hist[e][a][i] = c0 (u(v0), phi_a)_K + c1 (u(v1), phi_a)_K. V1 may be NULL (c1 unused).
 * BDF1: mass_coef = 1/dt, c0 = 1/dt. BDF2: mass_coef = 3/(2dt), c0 = 2/dt, c1 = -1/(2dt). */
int hdg_history(hdg_ctx_t ctx, const double* V0, const double* V1, double c0, double c1, double* hist,
                void* stream);

/* Source term of d u/dt + div(F + G) = s (the paper's Couette problem, Sec. 5.2, carries one):
 * the residual R_v of Eq. hDG_NS1 / hDG1 gains -(s_h, w)_K, s_h the nodal interpolant of s, and
 * takes it with the history, so this call adds it there:
 *   hist[e][a][i] += c (s_h, phi_a)_K,   s_h = sum_b src[e][b][i] phi_b.
 * src [E][Np][m] (device, conservative components at the element nodes, hdg_mesh_copy_coords
 * gives the nodes), hist [E][Np][m] (device, read and written: call hdg_history first, or zero
 * it for a steady problem), c a finite scale (1 for the source itself). Meshes of one degree
 * only (HDG_ERR_UNSUPPORTED on a mesh of mixed degree). Asynchronous on the stream. */
int hdg_add_source(hdg_ctx_t ctx, const double* src, double c, double* hist, void* stream);

/* Newton linearisation and static condensation of every element (Sec. 3.2-3.3, local
 * elimination): residuals R_v of Eq. hDG_NS1 / hDG1 (time term mass_coef (u(v), w) - hist)
 * and R_t of Eq. hDG_NS2 / hDG2 (this element's share), q eliminated exactly through the
 * linear Eq. hDG_NS0; Jacobian blocks A = dR_v/dV, B = dR_v/dVhat, C = dR_t/dV,
 * D = dR_t/dVhat; LU of A; S = D - C A^{-1} B, g = R_t - C A^{-1} R_v. Outputs S, g, recov,
 * R as documented above; elem_status [E] (int32, may be NULL) gets HDG_ELEM_* bits and
 * must be zeroed by the caller. precision: HDG_PREC_FP64 or HDG_PREC_MIXED.
 * Does not synchronise; status bits are the way to learn about bad elements. */
int hdg_assemble_condense(hdg_ctx_t ctx, const double* V, const double* Vhat, const double* hist,
                          double mass_coef, int precision, double* S, double* g, double* recov,
                          double* R, int32_t* elem_status, void* stream);

/* hdg_assemble_condense replayed as a CUDA graph (the same local elimination of Sec. 3.2,
 * the same arguments, results and status bits). An execution mechanism of this library: the
 * paper has no counterpart. The first call with a given set of arguments runs
 * hdg_assemble_condense on `stream` (which tunes the kernel shapes and allocates the scratch)
 * and then captures the same launch sequence, without running it, on a private stream; later
 * calls with the same pointers, precision, mass_coef and library scratch launch that graph on
 * `stream`, skipping the per-kernel launches. The graph reads the arrays' current contents, so
 * new values in the same buffers are used. Any other argument (or a scratch reallocated by a
 * call of the other precision) captures again. If the capture fails, the call still returns
 * the ordinary call's results and the context keeps the ordinary path. The graph belongs to
 * the context (freed by hdg_ctx_destroy); one call at a time per context. */
int hdg_assemble_condense_graph(hdg_ctx_t ctx, const double* V, const double* Vhat, const double* hist,
                                double mass_coef, int precision, double* S, double* g, double* recov, double* R,
                                int32_t* elem_status, void* stream);
/* Number of graph launches made by hdg_assemble_condense_graph on this context so far (0 if
 * every call ran the ordinary path, e.g. because the capture failed). */
int hdg_ctx_graph_replays(hdg_ctx_t ctx, int64_t* replays);
/* GMRES restart cycles run by this context's trace solves so far, and how many of them were one
 * replay of the CUDA graph of a cycle's Arnoldi steps (the rest ran the same kernels launch by
 * launch, when no graph could be captured). An execution mechanism of this library. */
int hdg_ctx_trace_cycles(hdg_ctx_t ctx, int64_t* cycles, int64_t* replays);

/* hdg_assemble_condense with S and g delivered to HOST memory (Sec. 3.2, the same local
 * elimination as hdg_assemble_condense). The elements are processed in chunks; each chunk's S
 * goes to one of a ring of four library-owned device buffers and is copied to S_host on an
 * internal copy stream while the next chunks compute, so the copy of S (the bulk of the output)
 * overlaps the kernels. g is copied to g_host at the end.
 *   V, Vhat, hist, recov, R, elem_status: device pointers as in hdg_assemble_condense.
 *   S_host [E][NT][NT], g_host [E][NT]: host memory; page-locked (cudaHostAlloc) memory is
 *   needed for the copies to overlap the kernels.
 * The call is asynchronous on `stream`: S_host and g_host are complete once the stream has
 * reached the end of the call (cudaStreamSynchronize). The first call allocates the ring
 * (4 x chunk x NT x NT doubles) and the context's g. Errors: HDG_ERR_INVALID_ARG for
 * null pointers or an unknown precision, HDG_ERR_CUDA for a failed allocation or launch. */
int hdg_assemble_condense_host(hdg_ctx_t ctx, const double* V, const double* Vhat, const double* hist,
                               double mass_coef, int precision, double* S_host, double* g_host, double* recov,
                               double* R, int32_t* elem_status, void* stream);

/* The same FP64 assemble + condense for callers that must not allocate device memory
 * during the call (the paper has no counterpart: this is a deployment variant). Such
 * callers include runtimes that give the library a fixed memory arena and forbid further
 * cudaMalloc/cudaFree, and loops where an allocation and the implicit device
 * synchronisation of cudaFree are not acceptable.
 * The call allocates nothing: its scratch is a 64 MiB static device array, present on every
 * GPU that loads the library until the process exits; elements are processed in chunks
 * that fit it. A configuration whose single-element scratch exceeds 64 MiB is rejected with
 * HDG_ERR_INVALID_ARG. The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the process; after a
 * cudaDeviceReset of that device the address is stale and further calls are invalid.
 * All calls share the array, so calls whose kernels overlap on the GPU race; order them
 * on one stream (or synchronise). Nothing in the array needs clearing between calls.
 * Arguments as for hdg_assemble_condense with precision FP64; elem_status is required
 * (zeroed by the caller). The context itself is created beforehand by hdg_ctx_create. */
int hdg_assemble_condense_noalloc(hdg_ctx_t ctx, const double* V, const double* Vhat, const double* hist,
                                  double mass_coef, double* S, double* g, double* recov, double* R,
                                  int32_t* elem_status, void* stream);

/* Entropy diagnostics of Eq. PiS (Sec. 5.6) from (v_h, q_h), q_h the gradient of Eq. hDG_NS0
 * (element-local, with Vhat): *int_rho_s = int rho s with s = log(p / rho^gamma) (Sec. 2.3), and
 * *production = (1/c_v) int (Phi / T + kappa |grad T|^2 / T^2), Phi = grad V : tau, the physical
 * entropy production (0 for Euler). The scheme's own part is Pi_S = d/dt int rho s - production:
 * callers difference int_rho_s between time levels. Writes host scalars (synchronises). */
int hdg_entropy_production(hdg_ctx_t ctx, const double* V, const double* Vhat, double* int_rho_s, double* production,
                           void* stream);

/* Global trace system sum_e P_e^T S_e P_e dVhat = -sum_e P_e^T g_e (Sec. 3.2: only vhat
 * is globally coupled). method: HDG_SOLVER_GMRES (restarted GMRES(30), face-block Jacobi
 * preconditioner; each restart cycle's Arnoldi steps run on the device without a host round
 * trip, replayed as a CUDA graph, and the host reads the cycle's outcome once per cycle), HDG_SOLVER_DENSE (assembled dense LU with partial pivoting, for
 * n_trace <= 16384) or HDG_SOLVER_AUTO (dense up to 4096 unknowns, else GMRES).
 * dVhat [F][Nf][m] device output. Writes *iters and
 * *final_res (relative residual) on the host, so it synchronises the stream.
 * HDG_ERR_NOT_CONVERGED if rtol was not reached in max_it iterations. */
int hdg_trace_solve(hdg_ctx_t ctx, const double* S, const double* g, double* dVhat, int method, double rtol,
                    int max_it, int* iters, double* final_res, void* stream);

/* Interior recovery (Sec. 3.2): dV_e = -y_e - X_e P_e dVhat. dV [E][Np][m] device. */
int hdg_recover_interior(hdg_ctx_t ctx, const double* recov, const double* dVhat, double* dV, void* stream);

/* out = a x + b y elementwise over n doubles (device; out may alias x or y). Used for
 * state extrapolation and Newton updates around the calls above. */
int hdg_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, void* stream);

/* Helpers used around the solve. y = K x with K = sum_e P_e^T S_e P_e (trace vectors). */
int hdg_trace_matvec(hdg_ctx_t ctx, const double* S, const double* x, double* y, void* stream);
/* Newton residual norm sqrt(sum_e |R_v,e|^2 + |sum_e P_e^T R_t,e|^2) from R; writes the
 * host scalar *norm (synchronises). */
int hdg_residual_norm(hdg_ctx_t ctx, const double* R, double* norm, void* stream);

/* Newton's method on the discrete equations of Sec. 3.2 / 3.3 with a given time term
 * mass_coef (u(v), w) - hist (hist as for hdg_assemble_condense, NULL for none): repeats
 * assemble_condense, trace_solve (hdg_ctx_set_trace_solver's settings), recover and the
 * update V += dV, Vhat += dVhat until |R| <= tol max(1, |R_0|) or max_newton updates were
 * made. V and Vhat are updated in place; *newton_iters and *res_norm (final) are written on
 * the host; res_history (host, nullable, max_newton + 1 entries) receives the residual norm
 * before each update, trace_iters (host, nullable) the total trace-solver iterations.
 * Context-owned workspaces are allocated on the first call. Synchronises once per Newton
 * iteration (residual norm and status bits). On meshes of one degree each iteration's
 * assemble + condense goes through hdg_assemble_condense_graph (captured on the first
 * iteration, replayed on the others); GMRES cycles are replayed graphs as in hdg_trace_solve. Errors: HDG_ERR_NOT_CONVERGED (max_newton
 * updates made, or the trace solve missed its tolerance), HDG_ERR_NONPHYSICAL,
 * HDG_ERR_SINGULAR, HDG_ERR_REFINE / HDG_ERR_TIMEOUT (mixed form with the FP64 recomputation
 * off). */
int hdg_newton_solve(hdg_ctx_t ctx, double* V, double* Vhat, const double* hist, double mass_coef, int precision,
                     double tol, int max_newton, int* newton_iters, double* res_norm, double* res_history,
                     int* trace_iters, void* stream);

/* One time step of the three-stage, third-order, L-stable DIRK(3,3) method of Alexander, the
 * integrator of the paper's unsteady examples (Sec. 5). Stage i solves the discrete equations
 * (hdg_newton_solve) with the time term (u_i - u_n, w)/(dt a_ii) - sum_{j<i} (a_ij/a_ii)(k_j, w),
 * i.e. mass_coef = 1/(dt a_ii), where the weak stage derivatives follow from the stage
 * equations: (k_j, w) = (u_j - u_n, w)/(dt a_jj) - sum_{l<j} (a_jl/a_jj)(k_l, w). The method is
 * stiffly accurate, so the level n+1 state is the last stage's.
 *   V_n         [E][Np][m] level-n entropy variables (device)
 *   V, Vhat     on entry the first stage's initial guess (usually the level-n state), on exit
 *               the level n+1 state; each stage starts from the previous one
 *   stage_iters host [3]: Newton updates of each stage; *res_norm the last stage's final
 *               residual norm; trace_iters (host, nullable) the total trace-solver iterations
 * Uses context-owned workspaces (4 x E Np m doubles, allocated on the first call). Errors as
 * for hdg_newton_solve. */
int hdg_dirk3_step(hdg_ctx_t ctx, double* V, double* Vhat, const double* V_n, double dt, int precision, double tol,
                   int max_newton, int* stage_iters, double* res_norm, int* trace_iters, void* stream);

/* Learned warm start of hdg_newton_step (no counterpart in the paper; it only supplies the
 * initial guess, and the Newton solve still decides the converged answer). params = NULL
 * gives the element-local start alone (dvhat = 0 below). All pointers are device memory.
 *   params, nin, nh, nout       network of hdg_mlp_* (nin = 4 Nf m, nout = Nf m)
 *   feat_mean, feat_std [nin]   feature standardisation (hdg_mlp_features)
 *   tmean, tscale [nout]        target de-standardisation (hdg_mlp_apply_trace)
 *   vhat_n, dvhat1, dvhat2      [F][Nf][m]: trace of time level n, vhat^n - vhat^{n-1},
 *                               vhat^{n-1} - vhat^{n-2} */
typedef struct {
  const float* params;
  int nin, nh, nout;
  const float *feat_mean, *feat_std, *tmean, *tscale;
  const double *vhat_n, *dvhat1, *dvhat2;
} hdg_warmstart;

/* One implicit time step by Newton's method (Sec. 3.2 / 3.3 in time; the paper integrates
 * with DIRK(3,3), this call with BDF):
 *   bdf_order 0  steady equations (no time term; V_n, V_nm1, dt unused)
 *             1  BDF1: mass_coef = 1/dt, hist = (u(V_n), w)/dt
 *             2  BDF2: mass_coef = 3/(2dt), hist = 2 (u(V_n), w)/dt - (u(V_nm1), w)/(2dt)
 *   V_n, V_nm1  [E][Np][m] entropy variables of time levels n and n-1 (device)
 *   V, Vhat     on entry the initial guess (e.g. extrapolated with hdg_axpby), on exit the
 *               converged state of level n+1
 *   warmstart   NULL: Newton from (V, Vhat). Otherwise the guess is linearised once, the
 *               network's trace vhat_m = vhat_n + dvhat1 + MLP(features of (V_n, vhat_n,
 *               dvhat1, dvhat2)) (or the guess's own trace when params is NULL) replaces the
 *               first global trace solve, and the interior follows from the element-local
 *               recovery dV = -y - X P (vhat_m - Vhat); Newton continues from there. If that
 *               solve fails, the plain solve from the caller's guess runs instead.
 * Other arguments, outputs and errors as for hdg_newton_solve. */
int hdg_newton_step(hdg_ctx_t ctx, double* V, double* Vhat, const double* V_n, const double* V_nm1, double dt,
                    int bdf_order, int precision, double tol, int max_newton, const hdg_warmstart* warmstart,
                    int* newton_iters, double* res_norm, double* res_history, int* trace_iters, void* stream);

/* Learned warm start of the implicit step (no counterpart in the paper: it only supplies
 * the initial guess of the Newton solve above, which still decides the converged answer).
 * A per-face MLP x (nin) -> tanh (nh) -> tanh (nh) -> linear (nout) predicts the correction
 * to the extrapolated trace update dvhat^{n+1} - dvhat^n of one face from the face-node
 * features [V_side0 - vhat^n | V_side1 - vhat^n | dvhat^n | dvhat^{n-1}] (nin = 4 Nf m,
 * nout = Nf m). Weights are applied in BF16 with FP32 accumulation; training keeps FP32
 * master weights and Adam moments. The parameter buffer (device) holds, for
 * P = hdg_mlp_param_count(): P float master weights (W1 [nh][nin], b1, W2 [nh][nh], b2,
 * W3 [nout][nh], b3), P floats Adam m, P floats Adam v, then P bf16 weights: 14 P bytes.
 * Compiled sizes: (nin, nh, nout) = (64, 64, 16) and (48, 32, 12). */
int64_t hdg_mlp_param_count(int nin, int nh, int nout);
/* Glorot-uniform weights from a SplitMix64 counter stream of seed; zero biases and moments. */
int hdg_mlp_init(float* params, int nin, int nh, int nout, uint64_t seed, void* stream);
/* Standardised features feat [F][nin] (float) of every face: (raw - mean) / std, with
 * mean, std [nin] (device; zeros and ones give the raw features). */
int hdg_mlp_features(hdg_ctx_t ctx, const double* V, const double* Vhat, const double* dvhat1,
                     const double* dvhat2, const float* mean, const float* std, float* feat, void* stream);
/* Column mean and standard deviation of x [B][n] (float, device). */
int hdg_mlp_stats(const float* x, int64_t B, int n, float* mean, float* std, void* stream);
/* In place x = (x - mean) / std, columnwise. */
int hdg_mlp_standardize(float* x, int64_t B, int n, const float* mean, const float* std, void* stream);
/* Raw training target of each trace entry: (vhat_next - vhat) - dvhat1, as float. */
int hdg_mlp_target(int64_t n, const double* vhat_next, const double* vhat, const double* dvhat1, float* out,
                   void* stream);
/* y [B][nout] = MLP(x [B][nin]) with the BF16 weights of params. */
int hdg_mlp_forward(const float* params, int nin, int nh, int nout, const float* x, int64_t B, float* y,
                    void* stream);
/* Mean-squared-error gradient grad [P] (float, device) and loss [1] (device) of a batch. */
int hdg_mlp_gradient(const float* params, float* grad, int nin, int nh, int nout, const float* x,
                     const float* target, int64_t B, float* loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step = 1, 2, ...) on a batch. */
int hdg_mlp_train_step(float* params, float* grad, int nin, int nh, int nout, const float* x,
                       const float* target, int64_t B, float lr, int step, float* loss, void* stream);
/* Warm start of the trace: Vhat_out = Vhat + dvhat1 + (pred * tscale + tmean) componentwise,
 * pred [F][nout] from hdg_mlp_forward, tmean / tscale [nout] the target de-standardisation. */
int hdg_mlp_apply_trace(hdg_ctx_t ctx, const double* Vhat, const double* dvhat1, const float* pred,
                        const float* tmean, const float* tscale, double* Vhat_out, void* stream);

/* Measurement support (no counterpart in the paper). Every kernel launch of a context
 * is counted per kernel class; with profiling enabled each launch is also bracketed by
 * CUDA events recorded on its launching stream. hdg_profile_read synchronises on the
 * recorded events and returns, for one class (HDG_KERNEL_*, or -1 for all), the number
 * of launches and their summed device time in milliseconds since the last reset. */
enum {
  HDG_KERNEL_POINTWISE = 0,        /* fluxes and pointwise Jacobians (both forms)          */
  HDG_KERNEL_ASSEMBLE = 1,         /* FP64 form: quadrature contractions into A, B, C, D;
                                      both forms: the boundary faces' rows                   */
  HDG_KERNEL_CONDENSE = 2,         /* FP64 form: LU, X = A^{-1}B, S = D - C X              */
  HDG_KERNEL_MIXED_ASSEMBLE = 3,   /* mixed form: volume contractions (tensor-core slices) */
  HDG_KERNEL_MIXED_CONDENSE = 4,   /* mixed form: refinement, tensor-core slice products   */
  HDG_KERNEL_TRACE = 5,            /* trace operator, preconditioner, solver kernels       */
  HDG_KERNEL_OTHER = 6,            /* history, conversions, recovery, norms, updates       */
  HDG_KERNEL_MIXED_PREP = 7,       /* mixed form: FP32 inverse, scales, operand slices      */
  HDG_KERNEL_MIXED_FACE = 8,       /* mixed form: face contractions (tensor-core slices)    */
  HDG_KERNEL_MIXED_OPERATORS = 9,  /* mixed form: operator slices, FP64 residuals           */
  HDG_KERNEL_PCLASS = 10,          /* mixed-degree meshes: the persistent fused launch      */
  HDG_KERNEL_CLASSES = 11
};
int hdg_profile_enable(hdg_ctx_t ctx, int on);
int hdg_profile_reset(hdg_ctx_t ctx);
int hdg_profile_read(hdg_ctx_t ctx, int kernel_class, int64_t* launches, double* total_ms);

const char* hdg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HDG_H_ */
