// Single-FP32 instantiations of the assembly kernels on triangles, P1/P2/P4 (the precision study of
// the high-order elements: FP32 element tensors, FP64 global accumulation).
#include "fe_kernels.cuh"

namespace fe {
using namespace kern;
using OPS = OpsF32;

#define FE_BILINEAR_TABLE(W) \
  FE_FORMS_FOR(2, 1, W) FE_FORMS_FOR(2, 2, W) FE_FORMS_FOR(2, 4, W) FE_KAPPA_FOR(2, 1, W) FE_KAPPA_FOR(2, 2, W) \
  FE_KAPPA_FOR(2, 4, W)

#define VEC vec_push
LaunchFn pick_mat_push_f32(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(mat_push)
  return nullptr;
}
LaunchFn pick_action_push_f32(const fe_form_desc &d) {
  FE_BILINEAR_TABLE(action_push)
  return nullptr;
}
LaunchFn pick_vec_push_f32(const fe_form_desc &d) {
  FE_SRC_FOR(2, 1, 1) FE_SRC_FOR(2, 2, 2) FE_SRC_FOR(2, 2, 1) FE_SRC_FOR(2, 4, 1)
  return nullptr;
}
#undef VEC

}  // namespace fe
