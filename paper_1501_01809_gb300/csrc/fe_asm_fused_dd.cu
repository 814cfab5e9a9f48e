// Double-float (FP32 pair) instantiations of the fused assembly + matrix-free action: P1 and P2
// triangles (with kappa-diffusion) and tetrahedra, the elements compiled in double-float.
#include "fe_kernels.cuh"

namespace fe {
using namespace kern;
using OPS = OpsF32x2;

LaunchFn pick_mat_action_dd(const fe_form_desc &d) {
  FE_FORMS_FOR(2, 1, mat_action_push) FE_FORMS_FOR(2, 2, mat_action_push) FE_KAPPA_FOR(2, 1, mat_action_push)
  FE_KAPPA_FOR(2, 2, mat_action_push) FE_FORMS_FOR(3, 1, mat_action_push) FE_FORMS_FOR(3, 2, mat_action_push)
  return nullptr;
}

}  // namespace fe
