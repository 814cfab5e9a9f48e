// Dispatch of the assembly par_loops to the compiled kernel instantiations.
#include <cuda_runtime.h>

#include "fe_internal.h"

namespace fe {

LaunchFn pick_mat_push_f64(const fe_form_desc &d);
LaunchFn pick_action_push_f64(const fe_form_desc &d);
LaunchFn pick_vec_push_f64(const fe_form_desc &d);
LaunchFn pick_mat_push_dd2(const fe_form_desc &d);
LaunchFn pick_action_push_dd2(const fe_form_desc &d);
LaunchFn pick_vec_push_dd2(const fe_form_desc &d);
LaunchFn pick_mat_push_dd3(const fe_form_desc &d);
LaunchFn pick_action_push_dd3(const fe_form_desc &d);
LaunchFn pick_vec_push_dd3(const fe_form_desc &d);

namespace {

LaunchFn pick_mat(const fe_form_desc &d) {
  if (d.form == FE_FORM_SOURCE || d.strategy == FE_STRATEGY_PULL) return nullptr;
  if (d.precision == FE_PREC_FP64) return pick_mat_push_f64(d);
  if (d.precision == FE_PREC_F32X2) return d.dim == 2 ? pick_mat_push_dd2(d) : pick_mat_push_dd3(d);
  return nullptr;
}
LaunchFn pick_action(const fe_form_desc &d) {
  if (d.form == FE_FORM_SOURCE || d.strategy == FE_STRATEGY_PULL) return nullptr;
  if (d.precision == FE_PREC_FP64) return pick_action_push_f64(d);
  if (d.precision == FE_PREC_F32X2) return d.dim == 2 ? pick_action_push_dd2(d) : pick_action_push_dd3(d);
  return nullptr;
}
LaunchFn pick_vec(const fe_form_desc &d) {
  if (d.form != FE_FORM_SOURCE || d.strategy == FE_STRATEGY_PULL) return nullptr;
  if (d.precision == FE_PREC_FP64) return pick_vec_push_f64(d);
  if (d.precision == FE_PREC_F32X2) return d.dim == 2 ? pick_vec_push_dd2(d) : pick_vec_push_dd3(d);
  return nullptr;
}

}  // namespace

bool kernel_supported(const fe_form_desc &d) {
  if (d.form == FE_FORM_SOURCE) return pick_vec(d) != nullptr;
  return pick_mat(d) != nullptr;
}

cudaError_t launch_assemble_mat(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported) {
  LaunchFn f = pick_mat(d);
  *unsupported = f == nullptr;
  return f ? f(a, s) : cudaSuccess;
}

cudaError_t launch_action(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported) {
  LaunchFn f = pick_action(d);
  *unsupported = f == nullptr;
  return f ? f(a, s) : cudaSuccess;
}

cudaError_t launch_assemble_vec(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported) {
  LaunchFn f = pick_vec(d);
  *unsupported = f == nullptr;
  return f ? f(a, s) : cudaSuccess;
}

}  // namespace fe
