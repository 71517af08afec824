// H-matrix approximation (Sec. 3), H-LU factorisation and H-triangular
// solves (Sec. 4.1).  (placeholder until the factorisation lands)
#include "hfsem_internal.h"

struct hfsem_factor_s {
  hfsem_system* sys = nullptr;
};

namespace hf {
Precond* precond_of(hfsem_system*, hfsem_factor* f) {
  if (f) throw Error(HFSEM_ERR_UNSUPPORTED, "H-LU not built yet");
  return nullptr;
}
}  // namespace hf

extern "C" {
int hfsem_hlu_factor(hfsem_system*, const hfsem_hopts*, hfsem_factor**) {
  return HFSEM_ERR_UNSUPPORTED;
}
int hfsem_hmatrix_dense(const hfsem_factor*, int32_t, double*) { return HFSEM_ERR_UNSUPPORTED; }
int hfsem_precond_apply(hfsem_factor*, int32_t, const double*, double*) {
  return HFSEM_ERR_UNSUPPORTED;
}
void hfsem_factor_free(hfsem_factor* f) { delete f; }
}
