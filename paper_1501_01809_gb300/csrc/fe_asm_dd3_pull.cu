// Double-float (FP32 pair) instantiations of the pull assembly kernels on tetrahedra: P1 and P2
// for mass, Laplace and Helmholtz (kappa-diffusion and larger elements are compiled in FP64 only).
#include "fe_kernels.cuh"

namespace fe {
using namespace kern;
using OPS = OpsF32x2;

#define FE_BILINEAR_TABLE(W) \
  FE_FORMS_FOR(3, 1, W) FE_FORMS_FOR(3, 2, W)

#define VEC vec_pull
LaunchFn pick_mat_pull_dd3(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(mat_pull)
  return nullptr;
}
LaunchFn pick_action_pull_dd3(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(action_pull)
  return nullptr;
}
LaunchFn pick_vec_pull_dd3(const fe_form_desc &d) {
  FE_SRC_FOR(3, 1, 1) FE_SRC_FOR(3, 2, 2) FE_SRC_FOR(3, 2, 1)
  return nullptr;
}
LaunchFn pick_action_elem_dd3(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(action_elem)
  return nullptr;
}
#undef VEC
#define VEC vec_elem
LaunchFn pick_vec_elem_dd3(const fe_form_desc &d) {
  FE_SRC_FOR(3, 1, 1) FE_SRC_FOR(3, 2, 2) FE_SRC_FOR(3, 2, 1)
  return nullptr;
}
#undef VEC

}  // namespace fe
