"""FP64 CPU oracle for the entropy-variable hybridized DG hot path.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this package: only
tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may
use it. It shares no code with the CUDA path; the only common module is
workloads.py, which holds seeded input fields and no method arithmetic.

Everything here is plain and slow on purpose:
  * refel.py   reference simplex: Gauss-Jacobi rules by Golub-Welsch, equispaced
               Lagrange basis through a monomial Vandermonde.
  * mesh.py    periodic Kuhn-split triangle / tetrahedron meshes, faces, face-node
               matching, affine geometry, DOF / NNZ counting (Tables t:dofs, t:nnz).
  * physics.py entropy variables (Sec. 2.3), inverse map, fluxes (Eqs. flux,
               viscFlux, closuresNS), stabilization (Eq. sLxF); complex-safe.
  * mlp.py     the per-face warm-start MLP in FP64 (forward, loss, chain-rule gradient).
  * hdg.py     local residuals of Eqs. hDG1-2 / hDG_NS0-2 with the numerical
               fluxes of Eqs. numericalFlux and numericalFluxNS_2; Jacobians by
               complex step; dense static condensation; global trace solve;
               interior recovery; BDF1/BDF2 Newton step.
"""
