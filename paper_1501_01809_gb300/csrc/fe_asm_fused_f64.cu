// FP64 instantiations of the fused assembly + matrix-free action (every compiled element and form).
#include "fe_kernels.cuh"

namespace fe {
using namespace kern;
using OPS = OpsF64;

LaunchFn pick_mat_action_f64(const fe_form_desc &d) {
  FE_FORMS_FOR(2, 1, mat_action_push) FE_FORMS_FOR(2, 2, mat_action_push) FE_FORMS_FOR(2, 3, mat_action_push)
  FE_FORMS_FOR(2, 4, mat_action_push) FE_FORMS_FOR(3, 1, mat_action_push) FE_FORMS_FOR(3, 2, mat_action_push)
  FE_FORMS_FOR(3, 3, mat_action_push) FE_KAPPA_FOR(2, 1, mat_action_push) FE_KAPPA_FOR(2, 2, mat_action_push)
  FE_KAPPA_FOR(2, 4, mat_action_push) FE_KAPPA_FOR(3, 1, mat_action_push) FE_KAPPA_FOR(3, 2, mat_action_push)
  return nullptr;
}

}  // namespace fe
