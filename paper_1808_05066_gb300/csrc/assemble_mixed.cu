// Mixed-precision assemble + condense (FP32 factorisation with refinement to FP64
// accuracy). Not compiled in yet: the entry point reports HDG_ERR_UNSUPPORTED.
#include "ctx.hpp"

namespace hdg {

int assemble_condense_mixed(hdg_ctx* ctx, const double* V, const double* Vhat, const double* hist,
                            double mass_coef, double* S, double* g, double* recov, double* R, int32_t* status,
                            cudaStream_t s) {
  (void)ctx; (void)V; (void)Vhat; (void)hist; (void)mass_coef; (void)S; (void)g; (void)recov; (void)R;
  (void)status; (void)s;
  set_error("assemble_condense: mixed precision form not available in this build");
  return HDG_ERR_UNSUPPORTED;
}

}  // namespace hdg
