// Cell-wise assembly par_loops (Sec. 4.4 of the paper): for every cell, staging in (gather the
// vertex coordinates through the coordinate map and the coefficients through their maps), the
// local kernel (geometry + generated element-tensor contraction), and staging out (INC into the
// global CSR Mat through the per-cell lookup table, or into a Dat through the map).
//
// Push strategy: one thread per cell, FP64 atomic adds (red.global.add.f64) for the INC.  The
// element tensor is computed in native FP64 (OpsF64) or in double-float (OpsF32x2); the INC is
// FP64 in both.  Instantiated per precision in fe_asm_f64.cu and fe_asm_dd.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fe_dd.cuh"
#include "fe_internal.h"
#include "fe_ops.cuh"
#include "generated/fe_local.cuh"

namespace fe {
namespace kern {

constexpr int kPushThreads = 128;

__device__ __forceinline__ void flag(int *err, int bit, int64_t idx) {
  if (atomicOr(err, bit) == 0) err[1] = (int)idx;
}

template <int DIM, int P, int FORM, class Ops>
__device__ __forceinline__ void element_upper(const typename Ops::T *Lam, const typename Ops::T &vol,
                                              const typename Ops::T *kap, typename Ops::T *K) {
  using E = fe_gen::Elem<DIM, P>;
  if constexpr (FORM == FE_FORM_MASS) {
    E::template mass_upper<Ops>(vol, K);
  } else if constexpr (FORM == FE_FORM_LAPLACE) {
    E::template stiffness_upper<Ops>(Lam, K);
  } else if constexpr (FORM == FE_FORM_HELMHOLTZ) {
    E::template stiffness_upper<Ops>(Lam, K);
    E::template mass_upper_add<Ops>(vol, K);
  } else {
    constexpr int NL = Geo<DIM>::NLAM;
    typename Ops::T KL[(DIM + 1) * NL];
#pragma unroll
    for (int k = 0; k <= DIM; k++)
#pragma unroll
      for (int t = 0; t < NL; t++) KL[k * NL + t] = Ops::mul(kap[k], Lam[t]);
    fe_gen::Kappa<DIM, P>::template upper<Ops>(KL, K);
  }
}

// staging in of the vertex coordinates; returns false on an out-of-range coordinate-map value
template <int DIM>
__device__ __forceinline__ bool gather_coords(const AsmArgs &a, int64_t e, double (&x)[DIM + 1][DIM], int32_t (&v)[DIM + 1]) {
  bool ok = true;
#pragma unroll
  for (int m = 0; m <= DIM; m++) {
    v[m] = a.cmapv[e * (DIM + 1) + m];
    if (a.checks && (v[m] < 0 || v[m] >= a.nvert)) {
      ok = false;
      v[m] = 0;
    }
#pragma unroll
    for (int c = 0; c < DIM; c++) x[m][c] = a.coords[(int64_t)v[m] * DIM + c];
  }
  return ok;
}

template <int ND>
__device__ __forceinline__ bool gather_rows(const AsmArgs &a, int64_t e, int32_t (&rows)[ND]) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < ND; i++) {
    rows[i] = a.map[e * ND + i];
    if (a.checks && (rows[i] < 0 || rows[i] >= a.nrows)) {
      ok = false;
      rows[i] = 0;
    }
  }
  return ok;
}

template <int DIM>
__device__ __forceinline__ bool gather_kappa(const AsmArgs &a, int64_t e, double (&kap)[DIM + 1]) {
  bool ok = true;
#pragma unroll
  for (int m = 0; m <= DIM; m++) {
    int32_t v = a.coefmap[e * (DIM + 1) + m];
    if (a.checks && (v < 0 || v >= a.ncoef)) {
      ok = false;
      v = 0;
    }
    kap[m] = a.coef[v];
  }
  return ok;
}

// ---------------------------------------------------------------------------- Mat, push
template <int DIM, int P, int FORM, class Ops>
__global__ void __launch_bounds__(kPushThreads) k_mat_push(const AsmArgs a) {
  using T = typename Ops::T;
  using E = fe_gen::Elem<DIM, P>;
  constexpr int ND = E::ND;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.ncell) return;
  double x[DIM + 1][DIM], kap[DIM + 1];
  int32_t v[DIM + 1], rows[ND];
  bool ok = gather_coords<DIM>(a, e, x, v);
  ok &= gather_rows<ND>(a, e, rows);
  if constexpr (FORM == FE_FORM_KAPPA_DIFFUSION) ok &= gather_kappa<DIM>(a, e, kap);
  if (!ok) {
    flag(a.err, ERR_RANGE, e);
    return;
  }
  T Lam[Geo<DIM>::NLAM], vol, kp[DIM + 1];
  Geo<DIM>::template compute<Ops>(x, Lam, vol);
#pragma unroll
  for (int m = 0; m <= DIM; m++) kp[m] = Ops::from_f64(kap[m]);
  T K[E::NUP];
  element_upper<DIM, P, FORM, Ops>(Lam, vol, kp, K);
  double Kd[E::NUP];
#pragma unroll
  for (int u = 0; u < E::NUP; u++) Kd[u] = Ops::to_f64(K[u]);
  const uint8_t *L = a.lut + e * (ND * ND);
#pragma unroll
  for (int i = 0; i < ND; i++) {
    double *rowv = a.vals + a.rowptr[rows[i]];
#pragma unroll
    for (int j = 0; j < ND; j++) red_add_f64(rowv + L[i * ND + j], Kd[E::upper_index(i, j)]);
  }
}

// ---------------------------------------------------------------------------- action, push
template <int DIM, int P, int FORM, class Ops>
__global__ void __launch_bounds__(kPushThreads) k_action_push(const AsmArgs a) {
  using T = typename Ops::T;
  using E = fe_gen::Elem<DIM, P>;
  constexpr int ND = E::ND;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.ncell) return;
  double x[DIM + 1][DIM], kap[DIM + 1];
  int32_t v[DIM + 1], rows[ND];
  bool ok = gather_coords<DIM>(a, e, x, v);
  ok &= gather_rows<ND>(a, e, rows);
  if constexpr (FORM == FE_FORM_KAPPA_DIFFUSION) ok &= gather_kappa<DIM>(a, e, kap);
  if (!ok) {
    flag(a.err, ERR_RANGE, e);
    return;
  }
  T xe[ND];
#pragma unroll
  for (int j = 0; j < ND; j++) xe[j] = Ops::from_f64(a.x[rows[j]]);
  T Lam[Geo<DIM>::NLAM], vol, kp[DIM + 1];
  Geo<DIM>::template compute<Ops>(x, Lam, vol);
#pragma unroll
  for (int m = 0; m <= DIM; m++) kp[m] = Ops::from_f64(kap[m]);
  T K[E::NUP];
  element_upper<DIM, P, FORM, Ops>(Lam, vol, kp, K);
#pragma unroll
  for (int i = 0; i < ND; i++) {
    T yi = Ops::mul(K[E::upper_index(i, 0)], xe[0]);
#pragma unroll
    for (int j = 1; j < ND; j++) yi = Ops::fma3(K[E::upper_index(i, j)], xe[j], yi);
    red_add_f64(a.y + rows[i], Ops::to_f64(yi));
  }
}

// ---------------------------------------------------------------------------- vector (f v dx), push
template <int DIM, int P, int Q, class Ops>
__global__ void __launch_bounds__(kPushThreads) k_vec_push(const AsmArgs a) {
  using T = typename Ops::T;
  using S = fe_gen::Source<DIM, P, Q>;
  constexpr int ND = S::ND, NF = S::NF;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.ncell) return;
  double x[DIM + 1][DIM];
  int32_t v[DIM + 1], rows[ND];
  bool ok = gather_coords<DIM>(a, e, x, v);
  ok &= gather_rows<ND>(a, e, rows);
  double fed[NF];
#pragma unroll
  for (int k = 0; k < NF; k++) {
    int32_t c = a.coefmap[e * NF + k];
    if (a.checks && (c < 0 || c >= a.ncoef)) {
      ok = false;
      c = 0;
    }
    fed[k] = a.coef[c];
  }
  if (!ok) {
    flag(a.err, ERR_RANGE, e);
    return;
  }
  T Lam[Geo<DIM>::NLAM], vol, fe[NF];
  Geo<DIM>::template compute<Ops>(x, Lam, vol);
#pragma unroll
  for (int k = 0; k < NF; k++) fe[k] = Ops::from_f64(fed[k]);
  T b[ND];
  S::template vec<Ops>(vol, fe, b);
#pragma unroll
  for (int i = 0; i < ND; i++) red_add_f64(a.y + rows[i], Ops::to_f64(b[i]));
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <int DIM, int P, int FORM, class Ops>
cudaError_t mat_push(const AsmArgs &a, cudaStream_t s) {
  if (a.ncell > 0) k_mat_push<DIM, P, FORM, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a);
  return cudaGetLastError();
}
template <int DIM, int P, int FORM, class Ops>
cudaError_t action_push(const AsmArgs &a, cudaStream_t s) {
  if (a.ncell > 0) k_action_push<DIM, P, FORM, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a);
  return cudaGetLastError();
}
template <int DIM, int P, int Q, class Ops>
cudaError_t vec_push(const AsmArgs &a, cudaStream_t s) {
  if (a.ncell > 0) k_vec_push<DIM, P, Q, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a);
  return cudaGetLastError();
}


#define FE_FORMS_FOR(D, P, W)                                                    \
  if (d.dim == D && d.degree == P) {                                             \
    if (d.form == FE_FORM_MASS) return &W<D, P, FE_FORM_MASS, OPS>;              \
    if (d.form == FE_FORM_LAPLACE) return &W<D, P, FE_FORM_LAPLACE, OPS>;        \
    if (d.form == FE_FORM_HELMHOLTZ) return &W<D, P, FE_FORM_HELMHOLTZ, OPS>;    \
  }
#define FE_KAPPA_FOR(D, P, W) \
  if (d.dim == D && d.degree == P && d.form == FE_FORM_KAPPA_DIFFUSION) return &W<D, P, FE_FORM_KAPPA_DIFFUSION, OPS>;
#define FE_SRC_FOR(D, P, Q) \
  if (d.dim == D && d.degree == P && d.coeff_degree == Q) return &vec_push<D, P, Q, OPS>;

}  // namespace kern
}  // namespace fe
