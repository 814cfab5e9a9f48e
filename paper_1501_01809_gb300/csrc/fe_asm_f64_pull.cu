// FP64 instantiations of the pull assembly kernels (all compiled-in elements and forms).
#include "fe_kernels.cuh"

namespace fe {
using namespace kern;
using OPS = OpsF64;

#define FE_BILINEAR_TABLE(W) \
  FE_FORMS_FOR(2, 1, W) FE_FORMS_FOR(2, 2, W) FE_FORMS_FOR(2, 3, W) FE_FORMS_FOR(2, 4, W) FE_FORMS_FOR(3, 1, W) \
  FE_FORMS_FOR(3, 2, W) FE_FORMS_FOR(3, 3, W) FE_KAPPA_FOR(2, 1, W) FE_KAPPA_FOR(2, 2, W) FE_KAPPA_FOR(2, 4, W) \
  FE_KAPPA_FOR(3, 1, W) FE_KAPPA_FOR(3, 2, W)

#define VEC vec_pull
LaunchFn pick_mat_pull_f64(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(mat_pull)
  return nullptr;
}
LaunchFn pick_action_pull_f64(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(action_pull)
  return nullptr;
}
LaunchFn pick_vec_pull_f64(const fe_form_desc &d) {
  FE_SRC_FOR(2, 1, 1) FE_SRC_FOR(2, 2, 2) FE_SRC_FOR(2, 2, 1) FE_SRC_FOR(2, 4, 1) FE_SRC_FOR(3, 1, 1) FE_SRC_FOR(3, 2, 2) FE_SRC_FOR(3, 2, 1)
  return nullptr;
}
LaunchFn pick_action_elem_f64(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(action_elem)
  return nullptr;
}
#undef VEC
#define VEC vec_elem
LaunchFn pick_vec_elem_f64(const fe_form_desc &d) {
  FE_SRC_FOR(2, 1, 1) FE_SRC_FOR(2, 2, 2) FE_SRC_FOR(2, 2, 1) FE_SRC_FOR(2, 4, 1) FE_SRC_FOR(3, 1, 1) FE_SRC_FOR(3, 2, 2) FE_SRC_FOR(3, 2, 1)
  return nullptr;
}
#undef VEC

}  // namespace fe
