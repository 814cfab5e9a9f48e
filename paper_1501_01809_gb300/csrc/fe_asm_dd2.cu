// Double-float (FP32 pair) instantiations of the assembly kernels on triangles: P1 and P2 (the
// element tensors of the larger elements are compiled in FP64 only).
#include "fe_kernels.cuh"

namespace fe {
using namespace kern;
using OPS = OpsF32x2;

#define FE_BILINEAR_TABLE(W) \
  FE_FORMS_FOR(2, 1, W) FE_FORMS_FOR(2, 2, W) FE_KAPPA_FOR(2, 1, W) FE_KAPPA_FOR(2, 2, W)

#define VEC vec_push
LaunchFn pick_mat_push_dd2(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(mat_push)
  return nullptr;
}
LaunchFn pick_action_push_dd2(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(action_push)
  return nullptr;
}
LaunchFn pick_vec_push_dd2(const fe_form_desc &d) {
  FE_SRC_FOR(2, 1, 1) FE_SRC_FOR(2, 2, 2) FE_SRC_FOR(2, 2, 1)
  return nullptr;
}
#undef VEC

#define VEC vec_pull
LaunchFn pick_mat_pull_dd2(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(mat_pull)
  return nullptr;
}
LaunchFn pick_action_pull_dd2(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(action_pull)
  return nullptr;
}
LaunchFn pick_vec_pull_dd2(const fe_form_desc &d) {
  FE_SRC_FOR(2, 1, 1) FE_SRC_FOR(2, 2, 2) FE_SRC_FOR(2, 2, 1)
  return nullptr;
}
LaunchFn pick_action_elem_dd2(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(action_elem)
  return nullptr;
}
#undef VEC
#define VEC vec_elem
LaunchFn pick_vec_elem_dd2(const fe_form_desc &d) {
  FE_SRC_FOR(2, 1, 1) FE_SRC_FOR(2, 2, 2) FE_SRC_FOR(2, 2, 1)
  return nullptr;
}
#undef VEC

}  // namespace fe
