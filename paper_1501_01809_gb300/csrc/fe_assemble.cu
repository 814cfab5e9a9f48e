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
LaunchFn pick_mat_push_f32(const fe_form_desc &d);
LaunchFn pick_action_push_f32(const fe_form_desc &d);
LaunchFn pick_vec_push_f32(const fe_form_desc &d);
LaunchFn pick_mat_pull_f64(const fe_form_desc &d);
LaunchFn pick_action_pull_f64(const fe_form_desc &d);
LaunchFn pick_vec_pull_f64(const fe_form_desc &d);
LaunchFn pick_mat_pull_dd2(const fe_form_desc &d);
LaunchFn pick_action_pull_dd2(const fe_form_desc &d);
LaunchFn pick_vec_pull_dd2(const fe_form_desc &d);
LaunchFn pick_mat_pull_dd3(const fe_form_desc &d);
LaunchFn pick_action_pull_dd3(const fe_form_desc &d);
LaunchFn pick_vec_pull_dd3(const fe_form_desc &d);
LaunchFn pick_mat_push_tc(const fe_form_desc &d);
LaunchFn pick_mat_action_f64(const fe_form_desc &d);
LaunchFn pick_mat_action_dd(const fe_form_desc &d);
LaunchFn pick_action_elem_f64(const fe_form_desc &d);
LaunchFn pick_vec_elem_f64(const fe_form_desc &d);
LaunchFn pick_action_elem_dd2(const fe_form_desc &d);
LaunchFn pick_vec_elem_dd2(const fe_form_desc &d);
LaunchFn pick_action_elem_dd3(const fe_form_desc &d);
LaunchFn pick_vec_elem_dd3(const fe_form_desc &d);
StoreFn pick_elem_store_f64(const fe_form_desc &d);
StoreFn pick_elem_store_dd(const fe_form_desc &d);
StoredActionFn pick_action_stored_f64(int nd);
StoredActionFn pick_action_stored_dd(int nd);

namespace {

// strategy: FE_STRATEGY_PUSH or FE_STRATEGY_PULL (already resolved)
LaunchFn pick_mat(const fe_form_desc &d, int strategy) {
  if (d.form == FE_FORM_SOURCE) return nullptr;
  const bool pull = strategy == FE_STRATEGY_PULL;
  if (d.precision == FE_PREC_FP64) return pull ? pick_mat_pull_f64(d) : pick_mat_push_f64(d);
  if (d.precision == FE_PREC_FP32) return pull || d.dim != 2 ? nullptr : pick_mat_push_f32(d);
  if (d.precision == FE_PREC_TF32X3) return pull ? nullptr : pick_mat_push_tc(d);
  if (d.precision == FE_PREC_F32X2) {
    if (d.dim == 2) return pull ? pick_mat_pull_dd2(d) : pick_mat_push_dd2(d);
    return pull ? pick_mat_pull_dd3(d) : pick_mat_push_dd3(d);
  }
  return nullptr;
}
LaunchFn pick_action(const fe_form_desc &d, int strategy) {
  if (d.form == FE_FORM_SOURCE) return nullptr;
  const bool pull = strategy == FE_STRATEGY_PULL;
  if (d.precision == FE_PREC_FP64) return pull ? pick_action_pull_f64(d) : pick_action_push_f64(d);
  if (d.precision == FE_PREC_FP32) return pull || d.dim != 2 ? nullptr : pick_action_push_f32(d);
  if (d.precision == FE_PREC_F32X2) {
    if (d.dim == 2) return pull ? pick_action_pull_dd2(d) : pick_action_push_dd2(d);
    return pull ? pick_action_pull_dd3(d) : pick_action_push_dd3(d);
  }
  return nullptr;
}
LaunchFn pick_vec(const fe_form_desc &d, int strategy) {
  if (d.form != FE_FORM_SOURCE) return nullptr;
  const bool pull = strategy == FE_STRATEGY_PULL;
  if (d.precision == FE_PREC_FP64) return pull ? pick_vec_pull_f64(d) : pick_vec_push_f64(d);
  if (d.precision == FE_PREC_FP32) return pull || d.dim != 2 ? nullptr : pick_vec_push_f32(d);
  if (d.precision == FE_PREC_F32X2) {
    if (d.dim == 2) return pull ? pick_vec_pull_dd2(d) : pick_vec_push_dd2(d);
    return pull ? pick_vec_pull_dd3(d) : pick_vec_push_dd3(d);
  }
  return nullptr;
}

int nodes_of(int dim, int p) { return dim == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6; }

}  // namespace

int resolve_strategy(const fe_form_desc &d, bool have_incidence) {
  (void)have_incidence;
  // AUTO = PUSH: the faster INC on this hardware for these kernels (the FP64 atomics stay in L2);
  // PULL is chosen explicitly when bitwise-reproducible results are required.
  return d.strategy == FE_STRATEGY_PULL ? FE_STRATEGY_PULL : FE_STRATEGY_PUSH;
}

size_t stage_bytes_mat(const fe_form_desc &d, int64_t ncell) {
  // (the FP32 element tensors have no pull kernels; sizes below are for FP64 and FP32 pairs)
  const int nd = nodes_of(d.dim, d.degree);
  const size_t elem = d.precision == FE_PREC_F32X2 ? 2 * sizeof(float) : sizeof(double);
  return (size_t)ncell * (size_t)(nd * nd) * elem;  // full element rows
}

size_t stage_bytes_vec(const fe_form_desc &d, int64_t ncell, int nd) {
  const size_t elem = d.precision == FE_PREC_F32X2 ? 2 * sizeof(float) : sizeof(double);
  return (size_t)ncell * (size_t)nd * elem;
}

bool kernel_supported(const fe_form_desc &d) {
  if (d.form == FE_FORM_SOURCE) return pick_vec(d, FE_STRATEGY_PUSH) != nullptr;
  return pick_mat(d, FE_STRATEGY_PUSH) != nullptr;
}

cudaError_t launch_assemble_mat(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported) {
  LaunchFn f = pick_mat(d, resolve_strategy(d, a.adj != nullptr));
  *unsupported = f == nullptr;
  return f ? f(a, s) : cudaSuccess;
}

cudaError_t launch_action(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported) {
  LaunchFn f = pick_action(d, resolve_strategy(d, a.adj != nullptr));
  *unsupported = f == nullptr;
  return f ? f(a, s) : cudaSuccess;
}

cudaError_t launch_assemble_vec(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported) {
  LaunchFn f = pick_vec(d, resolve_strategy(d, a.adj != nullptr));
  *unsupported = f == nullptr;
  return f ? f(a, s) : cudaSuccess;
}

// Assembly and action in one pass (push): FP64 or double-float element arithmetic.
cudaError_t launch_mat_action(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported) {
  LaunchFn f = nullptr;
  if (d.form != FE_FORM_SOURCE && resolve_strategy(d, false) == FE_STRATEGY_PUSH) {
    if (d.precision == FE_PREC_FP64) f = pick_mat_action_f64(d);
    else if (d.precision == FE_PREC_F32X2) f = pick_mat_action_dd(d);
  }
  *unsupported = f == nullptr;
  return f ? f(a, s) : cudaSuccess;
}

// The element stage of a rank-0 form: K_e x_e per cell (bilinear kernels) or b_e (linear), in the
// precisions that have pull kernels (FP64, double-float).
cudaError_t launch_elem_stage(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported) {
  LaunchFn f = nullptr;
  const bool lin = d.form == FE_FORM_SOURCE;
  if (d.precision == FE_PREC_FP64) f = lin ? pick_vec_elem_f64(d) : pick_action_elem_f64(d);
  else if (d.precision == FE_PREC_F32X2 && d.dim == 2) f = lin ? pick_vec_elem_dd2(d) : pick_action_elem_dd2(d);
  else if (d.precision == FE_PREC_F32X2 && d.dim == 3) f = lin ? pick_vec_elem_dd3(d) : pick_action_elem_dd3(d);
  *unsupported = f == nullptr;
  return f ? f(a, s) : cudaSuccess;
}

// Stored element matrices: FP64 and double-float element arithmetic, bilinear forms.
static StoreFn pick_elem_store(const fe_form_desc &d) {
  if (d.form == FE_FORM_SOURCE) return nullptr;
  if (d.precision == FE_PREC_FP64) return pick_elem_store_f64(d);
  if (d.precision == FE_PREC_F32X2) return pick_elem_store_dd(d);
  return nullptr;
}

cudaError_t launch_elem_store(const fe_form_desc &d, const AsmArgs &a, double *Ke, cudaStream_t s, int *unsupported) {
  StoreFn f = pick_elem_store(d);
  *unsupported = f == nullptr;
  return f ? f(a, Ke, s) : cudaSuccess;
}

cudaError_t launch_action_stored(const fe_form_desc &d, int nd, const AsmArgs &a, const double *Ke, cudaStream_t s,
                                 int *unsupported) {
  StoredActionFn f = nullptr;
  if (pick_elem_store(d)) f = d.precision == FE_PREC_FP64 ? pick_action_stored_f64(nd) : pick_action_stored_dd(nd);
  *unsupported = f == nullptr;
  return f ? f(a, Ke, s) : cudaSuccess;
}

}  // namespace fe
