// Stored element matrices: the alternative to the matrix-free action (Sec. 6.3) that keeps every
// cell's element matrix on the device instead of recomputing it at each application.
//
//  * k_elem_store runs the local kernel of the Mat assembly (gather of the vertex coordinates and
//    coefficients, geometry, generated element-tensor contraction; Sec. 4.4, 5.2) and stores the
//    upper triangle of K_e in FP64, entry-major: Ke[u * ncell + e], u counting the pairs i <= j
//    row by row.  A warp's store (and later load) of one entry touches 32 consecutive doubles.
//  * k_action_stored applies them: y[map(e)[i]] += sum_j K_e[i][j] x[map(e)[j]], one thread per
//    cell, the stored values read once with evict-first loads (so x and y keep the L2), the
//    products in the kernel's arithmetic (FP64, or FP32 pairs widened exactly from the stored FP64
//    values), the INC by FP64 atomics.
//
// The stored path trades nd(nd+1)/2 * 8 bytes of HBM per cell (440 B for P2 tetrahedra) for the
// element arithmetic of every action.
#pragma once
#include "fe_kernels.cuh"

namespace fe {
namespace kern {

template <int DIM, int P, int FORM, class Ops>
__global__ void __launch_bounds__(kPushThreads) k_elem_store(const AsmArgs a, double *__restrict__ Ke) {
  using T = typename Ops::T;
  using E = fe_gen::Elem<DIM, P>;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.ncell) return;
  double x[DIM + 1][DIM], kap[DIM + 1];
  int32_t v[DIM + 1];
  bool ok = gather_coords<DIM>(a, e, x, v);
  if constexpr (FORM == FE_FORM_KAPPA_DIFFUSION) ok &= gather_kappa<DIM>(a, e, kap);
  if (!ok) {
    flag(a.err, ERR_RANGE, e);
    return;
  }
  T Lam[Geo<DIM>::NLAM], vol, kp[DIM + 1];
  Geo<DIM>::template compute<Ops>(x, Lam, vol);
  if constexpr (FORM == FE_FORM_KAPPA_DIFFUSION) {
#pragma unroll
    for (int m = 0; m <= DIM; m++) kp[m] = Ops::from_f64(kap[m]);
  }
  T K[E::NUP];
  element_upper<DIM, P, FORM, Ops>(Lam, vol, kp, K);
#pragma unroll
  for (int u = 0; u < E::NUP; u++) Ke[(int64_t)u * a.ncell + e] = Ops::to_f64(K[u]);
}

template <int ND, class Ops>
__global__ void __launch_bounds__(kPushThreads) k_action_stored(const AsmArgs a, const double *__restrict__ Ke) {
  using T = typename Ops::T;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.ncell) return;
  int32_t rows[ND];
  if (!gather_rows<ND>(a, e, rows)) {
    flag(a.err, ERR_RANGE, e);
    return;
  }
  T xe[ND], ye[ND];
#pragma unroll
  for (int j = 0; j < ND; j++) {
    xe[j] = Ops::from_f64(a.x[rows[j]]);
    ye[j] = Ops::zero();
  }
  const double *k = Ke + e;
#pragma unroll
  for (int i = 0; i < ND; i++) {
#pragma unroll
    for (int j = i; j < ND; j++) {
      const T kij = Ops::from_f64(__ldcs(k));  // entry u = (i, j) of the upper triangle
      k += a.ncell;
      ye[i] = Ops::fma3(kij, xe[j], ye[i]);
      if (i != j) ye[j] = Ops::fma3(kij, xe[i], ye[j]);
    }
  }
#pragma unroll
  for (int i = 0; i < ND; i++) red_add_f64(a.y + rows[i], Ops::to_f64(ye[i]));
}

template <int DIM, int P, int FORM, class Ops>
cudaError_t elem_store(const AsmArgs &a, double *Ke, cudaStream_t s) {
  if (a.ncell > 0) k_elem_store<DIM, P, FORM, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a, Ke);
  return cudaGetLastError();
}

template <int ND, class Ops>
cudaError_t action_stored(const AsmArgs &a, const double *Ke, cudaStream_t s) {
  if (a.ncell > 0) k_action_stored<ND, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a, Ke);
  return cudaGetLastError();
}

}  // namespace kern
}  // namespace fe
