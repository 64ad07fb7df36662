// fmm32.cu -- the mixed-precision evaluation path (placeholder until the
// FP32 / tensor-core kernels land).
#include "internal.h"

namespace eifmm {

eifmm_status alloc_mixed_workspace(Tree* t, const Ops* ops, int R) {
  (void)t; (void)ops; (void)R;
  return EIFMM_OK;
}

eifmm_status eval_mixed(Tree* t, const Ops* ops, const double* sigma, int64_t ld_sigma, int R,
                        double* f, int64_t ld_f, cudaStream_t s) {
  (void)t; (void)ops; (void)sigma; (void)ld_sigma; (void)R; (void)f; (void)ld_f; (void)s;
  set_error("eifmm_evaluate: the mixed path is not built yet");
  return EIFMM_EUNSUPPORTED;
}

eifmm_status export_mixed(const Tree& t, const Ops& o, int what, int level, double* out, int64_t n) {
  (void)t; (void)o; (void)what; (void)level; (void)out; (void)n;
  set_error("eifmm_debug_export: no intermediates kept by the mixed path");
  return EIFMM_EUNSUPPORTED;
}

}  // namespace eifmm
