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
    E::template helmholtz_upper<Ops>(Lam, vol, K);
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
// One cell: gather, geometry, element tensor, 100 (P2 tet) FP64 atomic adds through the lookup table.
template <int DIM, int P, int FORM, class Ops>
__device__ __forceinline__ void mat_push_cell(const AsmArgs &a, int64_t e) {
  using T = typename Ops::T;
  using E = fe_gen::Elem<DIM, P>;
  constexpr int ND = E::ND;
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
  if (a.checks) {  // check mode: every lookup-table entry must lie inside its row (Sec. 4.4.1, INC)
#pragma unroll
    for (int i = 0; i < ND; i++) {
      const int64_t b = a.rowptr[rows[i]], len = a.rowptr[rows[i] + 1] - b;
#pragma unroll
      for (int j = 0; j < ND; j++) {
        const int q = L[i * ND + j];
        if (q < len) red_add_f64(a.vals + b + q, Kd[E::upper_index(i, j)]);
        else flag(a.err, ERR_LUT, e);
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < ND; i++) {
    double *rowv = a.vals + a.rowptr[rows[i]];
#pragma unroll
    for (int j = 0; j < ND; j++) red_add_f64(rowv + L[i * ND + j], Kd[E::upper_index(i, j)]);
  }
}

// Blocks per SM the push Mat kernel is compiled for.  The FP64 atomics bind it, so more resident
// warps keep more of them in flight: double-float builds fit 128 registers (four 128-thread blocks
// per SM instead of three at 167 registers, a few words spilled), which measured 6% faster for P2
// tetrahedra.  FP64 and FP32 builds keep the compiler's choice (P3/P4 would spill hundreds of bytes).
template <class Ops>
struct MatOcc {
  static constexpr int kMinBlocks = 1;
};
template <>
struct MatOcc<OpsF32x2> {
  static constexpr int kMinBlocks = 4;
};

template <int DIM, int P, int FORM, class Ops>
__global__ void __launch_bounds__(kPushThreads, MatOcc<Ops>::kMinBlocks) k_mat_push(const AsmArgs a) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < a.ncell) mat_push_cell<DIM, P, FORM, Ops>(a, e);
}

// ---------------------------------------------------------------------------- assembly + action, push
// The CSR assembly and the matrix-free action of the same form in one pass over the cells: each
// cell's element matrix is built once, in registers, and serves both outputs.  Its entries go into
// the CSR values through the lookup table (as k_mat_push), and y_e = K_e x_e into y (as
// k_action_push); the action still reads no assembled matrix.  Row i's products with x_e are
// formed beside that row's reductions, in the kernel's arithmetic (FP64 or double-float), and
// added to y[rows[i]] with one FP64 reduction.
template <int DIM, int P, int FORM, class Ops>
__device__ __forceinline__ void mat_action_push_cell(const AsmArgs &a, int64_t e, const uint8_t *L) {
  using T = typename Ops::T;
  using E = fe_gen::Elem<DIM, P>;
  constexpr int ND = E::ND;
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
    const int64_t b = a.rowptr[rows[i]];
    const int64_t len = a.checks ? a.rowptr[rows[i] + 1] - b : 0;
    T yi = Ops::mul(K[E::upper_index(i, 0)], xe[0]);
#pragma unroll
    for (int j = 1; j < ND; j++) yi = Ops::fma3(K[E::upper_index(i, j)], xe[j], yi);
#pragma unroll
    for (int j = 0; j < ND; j++) {
      const int q = L[i * ND + j];
      if (a.checks && q >= len) {  // check mode: a lookup-table entry beyond its row is skipped
        flag(a.err, ERR_LUT, e);
        continue;
      }
      red_add_f64(a.vals + b + q, Ops::to_f64(K[E::upper_index(i, j)]));
    }
    red_add_f64(a.y + rows[i], Ops::to_f64(yi));
  }
}

// Blocks per SM the fused kernel is compiled for.  The loads of the lookup table, row pointers and
// x wait longest, so resident warps matter more than a few spilled words: FP64 elements of at most
// 55 upper entries (P2 tetrahedra, P1-P3 triangles) take four 128-thread blocks per SM at 128
// registers (about 230 bytes spilled for P2 tetrahedra), which measured 1.106 -> 1.011 ms at 64^3
// against three blocks at 162 registers; larger elements keep the compiler's choice.
template <int DIM, int P, class Ops>
struct FusedOcc {
  static constexpr int kMinBlocks = MatOcc<Ops>::kMinBlocks;
};
template <int DIM, int P>
struct FusedOcc<DIM, P, OpsF64> {
  static constexpr int kMinBlocks = fe_gen::Elem<DIM, P>::NUP <= 55 ? 4 : 1;
};

// The block's lookup-table bytes are one contiguous range (its kPushThreads cells, ND^2 bytes each,
// 16-byte aligned): staged into shared memory with 16-byte loads, they replace each thread's ND^2
// byte loads at a stride of ND^2 bytes (one sector per lane per load) by reads of shared memory
// (free of bank conflicts when ND^2 / 4 is odd, as for P2 tetrahedra and triangles).  Elements
// whose staged table would pass 32 KB per block read the table from global memory.
template <int DIM, int P, int FORM, class Ops>
__global__ void __launch_bounds__(kPushThreads, FusedOcc<DIM, P, Ops>::kMinBlocks) k_mat_action_push(const AsmArgs a) {
  constexpr int NN = fe_gen::Elem<DIM, P>::ND * fe_gen::Elem<DIM, P>::ND;
  const int64_t e0 = blockIdx.x * (int64_t)kPushThreads, e = e0 + threadIdx.x;
  if constexpr (NN * kPushThreads <= 32 * 1024) {
    __shared__ __align__(16) uint8_t sL[NN * kPushThreads];
    const int64_t left = a.ncell - e0;
    const int nb = (int)(left < kPushThreads ? left : kPushThreads) * NN;  // bytes of this block's cells
    const uint8_t *src = a.lut + e0 * NN;
    for (int q = threadIdx.x; q < nb / 16; q += kPushThreads)
      reinterpret_cast<uint4 *>(sL)[q] = __ldg(reinterpret_cast<const uint4 *>(src) + q);
    for (int q = (nb / 16) * 16 + threadIdx.x; q < nb; q += kPushThreads) sL[q] = src[q];
    __syncthreads();
    if (e < a.ncell) mat_action_push_cell<DIM, P, FORM, Ops>(a, e, sL + threadIdx.x * NN);
  } else {
    if (e < a.ncell) mat_action_push_cell<DIM, P, FORM, Ops>(a, e, a.lut + e * NN);
  }
}

// ---------------------------------------------------------------------------- action, push
// Blocks per SM the push action is compiled for.  Double-float element arithmetic fits 96
// registers (five 128-thread blocks per SM) with at most a few words spilled, which measured 3%
// faster than 128 registers at four blocks; FP64 and FP32 builds keep the compiler's choice (the
// FP64 ones would spill hundreds of bytes).
template <class Ops>
struct ActionOcc {
  static constexpr int kMinBlocks = 1;
};
template <>
struct ActionOcc<OpsF32x2> {
  static constexpr int kMinBlocks = 5;
};

template <int DIM, int P, int FORM, class Ops>
__global__ void __launch_bounds__(kPushThreads, ActionOcc<Ops>::kMinBlocks) k_action_push(const AsmArgs a) {
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
  T ye[ND];
  if constexpr (FORM == FE_FORM_KAPPA_DIFFUSION) {
#pragma unroll
    for (int m = 0; m <= DIM; m++) kp[m] = Ops::from_f64(kap[m]);
    T K[E::NUP];
    element_upper<DIM, P, FORM, Ops>(Lam, vol, kp, K);
#pragma unroll
    for (int i = 0; i < ND; i++) {
      ye[i] = Ops::mul(K[E::upper_index(i, 0)], xe[0]);
#pragma unroll
      for (int j = 1; j < ND; j++) ye[i] = Ops::fma3(K[E::upper_index(i, j)], xe[j], ye[i]);
    }
  } else {
    E::template action_upper<Ops, FORM != FE_FORM_MASS, FORM != FE_FORM_LAPLACE>(Lam, vol, xe, ye);
  }
#pragma unroll
  for (int i = 0; i < ND; i++) red_add_f64(a.y + rows[i], Ops::to_f64(ye[i]));
}

// ---------------------------------------------------------------------------- vector (f v dx), push
template <int DIM, int P, int Q, class Ops>
__device__ __forceinline__ void vec_push_cell(const AsmArgs &a, int64_t e) {
  using T = typename Ops::T;
  using S = fe_gen::Source<DIM, P, Q>;
  constexpr int ND = S::ND, NF = S::NF;
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

template <int DIM, int P, int Q, class Ops>
__global__ void __launch_bounds__(kPushThreads) k_vec_push(const AsmArgs a) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < a.ncell) vec_push_cell<DIM, P, Q, Ops>(a, e);
}

// ---------------------------------------------------------------------------- staged pull
// Deterministic INC without atomics, in two kernels.  (1) One thread per cell stores its element
// tensor (K_e for a Mat, as full rows so that a row owner reads each incidence's row contiguously;
// the element vector for the action and the linear form) with plain stores to a staging buffer.  (2) One thread per row, the row's owner, walks the
// row's incidence list {(e, i)} -- ascending (sparsity_canonical, before the launch) -- and adds the
// contributions in that order; a Mat row accumulates in shared memory (slots given by the lookup
// table) and is written once.  The summation order is the same on every run: results are bitwise
// reproducible.


// Staging of element tensors through shared memory: used while a block's tensors fit in 64 KB.
template <class T, int NUP>
struct ElemStaging {
  static constexpr size_t kSmem = (size_t)NUP * sizeof(T) * 128;  // dynamic shared memory per block
  static constexpr bool kTransposed = kSmem <= 64 * 1024;
};

// One cell's element tensor (upper triangle) to the staging buffer, or (transposed staging) to the
// block's shared memory; false (the error flagged) on a bad map value.
template <int DIM, int P, int FORM, class Ops>
__device__ __forceinline__ bool mat_elem_cell(const AsmArgs &a, typename Ops::T *__restrict__ stage, int64_t e) {
  using T = typename Ops::T;
  using E = fe_gen::Elem<DIM, P>;
  double x[DIM + 1][DIM], kap[DIM + 1];
  int32_t v[DIM + 1];
  bool ok = gather_coords<DIM>(a, e, x, v);
  if constexpr (FORM == FE_FORM_KAPPA_DIFFUSION) ok &= gather_kappa<DIM>(a, e, kap);
  if (!ok) {
    flag(a.err, ERR_RANGE, e);
    return false;
  }
  T Lam[Geo<DIM>::NLAM], vol, kp[DIM + 1];
  Geo<DIM>::template compute<Ops>(x, Lam, vol);
#pragma unroll
  for (int m = 0; m <= DIM; m++) kp[m] = Ops::from_f64(kap[m]);
  T K[E::NUP];
  element_upper<DIM, P, FORM, Ops>(Lam, vol, kp, K);
  if constexpr (ElemStaging<T, E::NUP>::kTransposed) {
    // the block's element tensors are one contiguous range of the staging buffer: through shared
    // memory, every store instruction of the block writes consecutive addresses
    extern __shared__ __align__(16) unsigned char smem_elem[];
    T *sK = reinterpret_cast<T *>(smem_elem);
#pragma unroll
    for (int u = 0; u < E::NUP; u++) sK[(size_t)threadIdx.x * E::NUP + u] = K[u];
  } else {
    T *out = stage + e * (E::ND * E::ND);  // full rows, expanded from the upper triangle
#pragma unroll
    for (int i = 0; i < E::ND; i++)
#pragma unroll
      for (int j = 0; j < E::ND; j++) out[i * E::ND + j] = K[E::upper_index(i, j)];
  }
  return true;
}

// The same kernel's block epilogue (transposed staging): the cells of the block that were built
// (flagged cells leave their slots as they were) copied to the staging buffer in address order,
// each as its full ND x ND matrix (row i of cell e at (e ND + i) ND: the rows the row owners read).
template <class T, int ND>
__device__ __forceinline__ void copy_elem_block(T *__restrict__ stage, int64_t e0, int64_t ncell, const unsigned char *ok) {
  constexpr int NUP = ND * (ND + 1) / 2, NN = ND * ND;
  extern __shared__ __align__(16) unsigned char smem_elem[];
  const T *sK = reinterpret_cast<const T *>(smem_elem);
  const int64_t left = ncell - e0;
  const int n = (left < (int64_t)blockDim.x ? (int)left : (int)blockDim.x) * NN;
  T *out = stage + e0 * NN;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int m = q / NN, idx = q - m * NN, i = idx / ND, j = idx - (idx / ND) * ND;
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    if (ok[m]) out[q] = sK[m * NUP + lo * ND - lo * (lo - 1) / 2 + (hi - lo)];
  }
}

template <int DIM, int P, int FORM, class Ops>
__global__ void __launch_bounds__(kPushThreads) k_mat_elem(const AsmArgs a, typename Ops::T *__restrict__ stage) {
  using T = typename Ops::T;
  using E = fe_gen::Elem<DIM, P>;
  const int64_t e0 = blockIdx.x * (int64_t)blockDim.x, e = e0 + threadIdx.x;
  if constexpr (ElemStaging<T, E::NUP>::kTransposed) {
    __shared__ unsigned char ok[kPushThreads];
    ok[threadIdx.x] = e < a.ncell && mat_elem_cell<DIM, P, FORM, Ops>(a, stage, e);
    __syncthreads();
    copy_elem_block<T, E::ND>(stage, e0, a.ncell, ok);
  } else {
    if (e < a.ncell) mat_elem_cell<DIM, P, FORM, Ops>(a, stage, e);
  }
}


template <int DIM, int P, int FORM, class Ops>
__global__ void __launch_bounds__(kPushThreads) k_action_elem(const AsmArgs a, typename Ops::T *__restrict__ stage) {
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
  T ye[ND];
  if constexpr (P == 1 && FORM == FE_FORM_LAPLACE) {
    p1_laplace_action<DIM, Ops>(x, xe, ye);  // through grad(u): no element matrix
  } else {
    T Lam[Geo<DIM>::NLAM], vol, kp[DIM + 1];
    Geo<DIM>::template compute<Ops>(x, Lam, vol);
    if constexpr (FORM == FE_FORM_KAPPA_DIFFUSION) {
#pragma unroll
      for (int m = 0; m <= DIM; m++) kp[m] = Ops::from_f64(kap[m]);
      T K[E::NUP];
      element_upper<DIM, P, FORM, Ops>(Lam, vol, kp, K);
#pragma unroll
      for (int i = 0; i < ND; i++) {
        ye[i] = Ops::mul(K[E::upper_index(i, 0)], xe[0]);
#pragma unroll
        for (int j = 1; j < ND; j++) ye[i] = Ops::fma3(K[E::upper_index(i, j)], xe[j], ye[i]);
      }
    } else {
      E::template action_upper<Ops, FORM != FE_FORM_MASS, FORM != FE_FORM_LAPLACE>(Lam, vol, xe, ye);
    }
  }
  T *out = stage + e * ND;
#pragma unroll
  for (int i = 0; i < ND; i++) out[i] = ye[i];
}

// One cell's source vector (f v dx) to the staging buffer (ND values at e ND); false (the error
// flagged) on a bad map value.
template <int DIM, int P, int Q, class Ops>
__device__ __forceinline__ bool vec_elem_cell(const AsmArgs &a, typename Ops::T *__restrict__ stage, int64_t e) {
  using T = typename Ops::T;
  using S = fe_gen::Source<DIM, P, Q>;
  constexpr int ND = S::ND, NF = S::NF;
  double x[DIM + 1][DIM];
  int32_t v[DIM + 1];
  bool ok = gather_coords<DIM>(a, e, x, v);
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
    return false;
  }
  T Lam[Geo<DIM>::NLAM], vol, fe[NF];
  Geo<DIM>::template compute<Ops>(x, Lam, vol);
#pragma unroll
  for (int k = 0; k < NF; k++) fe[k] = Ops::from_f64(fed[k]);
  T b[ND];
  S::template vec<Ops>(vol, fe, b);
  T *out = stage + e * ND;
#pragma unroll
  for (int i = 0; i < ND; i++) out[i] = b[i];
  return true;
}

template <int DIM, int P, int Q, class Ops>
__global__ void __launch_bounds__(kPushThreads) k_vec_elem(const AsmArgs a, typename Ops::T *__restrict__ stage) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < a.ncell) vec_elem_cell<DIM, P, Q, Ops>(a, stage, e);
}

// The row-owner loop itself, for one group of ND lanes (lane j of it, `on` false for the lanes
// beyond the warp's NG groups, which still take part in its warp-wide steps): rows first,
// first + step, ... below rend, accumulated in buf (rowcap slots).  Called by every lane of the
// warp.  With BC, the rows and columns of the nodes flagged in is_bc are eliminated as each row
// is written out (symmetric elimination for u = 0 on the boundary: a flagged row keeps 1 on its
// diagonal and 0 elsewhere, a flagged column 0), exactly the values the separate elimination
// kernel writes.
template <int ND, class Ops, bool BC = false>
__device__ __forceinline__ void pull_mat_rows(int64_t first, int64_t step, int64_t rend, bool on, int j,
                                              typename Ops::T *buf, const int64_t *__restrict__ adjptr,
                                              const int32_t *__restrict__ adj, const int64_t *__restrict__ rowptr,
                                              const uint8_t *__restrict__ lut,
                                              const typename Ops::T *__restrict__ stage, double *__restrict__ vals,
                                              int rowcap, int zero_first, int *err, int checks,
                                              const int32_t *__restrict__ colidx = nullptr,
                                              const uint8_t *__restrict__ is_bc = nullptr) {
  using T = typename Ops::T;
  constexpr int U = 4;  // incidences per round
  int64_t r = first, b = 0, a0 = 0;
  int len = 0, na = 0, a = 0;
  bool have = false;
  auto start_row = [&]() {  // the group's next row: its range, incidence list and zeroed slots
    have = on && r < rend;
    a = 0;
    if (have) {
      b = rowptr[r];
      len = (int)(rowptr[r + 1] - b);
      a0 = adjptr[r];
      na = (int)(adjptr[r + 1] - a0);
      if (len > rowcap) {
        if (j == 0) flag(err, ERR_ROW_TOO_LONG, r);
        len = 0;
        na = 0;
      }
      for (int q = j; q < len; q += ND) buf[q] = Ops::zero();
    }
  };
  start_row();
  __syncwarp();
  while (__any_sync(0xffffffffu, have)) {
    // one round: each group with incidences left loads up to U of them, then adds them in order
    T v[U];
    int q[U];
    bool act[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      act[u] = have && a + u < na;
      v[u] = Ops::zero();
      q[u] = 0;
      if (act[u]) {
        const int64_t k = adj[a0 + a + u];  // incidence (e, i) = e ND + i
        v[u] = stage[k * ND + j];           // row i of cell e's element matrix, contiguous
        q[u] = lut[k * ND + j];
        if (checks && q[u] >= len) {  // check mode: a lookup-table entry beyond the row is skipped
          flag(err, ERR_LUT, k / ND);
          act[u] = false;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (act[u]) buf[q[u]] = Ops::add(buf[q[u]], v[u]);
      __syncwarp();
    }
    a += U;
    if (have && a >= na) {  // the row is complete: write it out, take the group's next row
      double *out = vals + b;
      bool bc_row = false;
      if constexpr (BC) bc_row = is_bc[r] != 0;
      for (int qq = j; qq < len; qq += ND) {
        double d = Ops::to_f64(buf[qq]);
        if constexpr (BC) {
          const int32_t col = colidx[b + qq];
          if (bc_row) d = col == r ? 1.0 : 0.0;
          else if (is_bc[col]) d = 0.0;
        }
        out[qq] = zero_first ? d : out[qq] + d;
      }
      r += step;
      start_row();
    }
    __syncwarp();
  }
}

// Row owners of a Mat.  Each warp holds NG = 32 / ND groups of ND lanes, and each group owns a
// row at a time (rows r = group, group + groups, ...).  A group walks its row's incidence list
// {(e, i)} -- ascending (sparsity_canonical, before the launch) -- U incidences per round: lane j
// of the group loads entry j of row i of cell e's staged element matrix (one contiguous ND-value
// row per incidence) and its lookup-table slot for all U incidences first, then adds them into
// the row's shared-memory accumulators one incidence after another.  Every slot therefore
// receives its contributions in incidence order, as a single row owner would add them: the
// result is bitwise reproducible.  The groups of a warp advance independently (a group that
// finishes its row writes it out and starts its next one), and one FP64 add instruction serves
// all of them, so the FP64 pipe -- 1/16 of a warp instruction per clock on this GPU -- is not
// spent on idle lanes.  INC semantics: the row's values are read once (unless zero_first) and
// written once.  Shared memory: rowcap accumulators per group.
template <int ND, class Ops>
__global__ void __launch_bounds__(256) k_mat_pull(int64_t nrows, const int64_t *__restrict__ adjptr,
                                                  const int32_t *__restrict__ adj, const int64_t *__restrict__ rowptr,
                                                  const uint8_t *__restrict__ lut,
                                                  const typename Ops::T *__restrict__ stage, double *__restrict__ vals,
                                                  int rowcap, int zero_first, int *err, int checks) {
  using T = typename Ops::T;
  constexpr int NG = 32 / ND > 0 ? 32 / ND : 1;  // row groups per warp
  extern __shared__ __align__(16) unsigned char smp[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int gi = lane / ND, j = lane - (lane / ND) * ND;
  const bool on = gi < NG;  // lanes beyond NG groups idle (and take part in the warp-wide steps)
  T *buf = reinterpret_cast<T *>(smp) + ((size_t)wid * NG + (on ? gi : 0)) * rowcap;
  const int64_t groups = (int64_t)gridDim.x * wpb * NG;
  pull_mat_rows<ND, Ops>(((int64_t)blockIdx.x * wpb + wid) * NG + gi, groups, nrows, on, j, buf, adjptr, adj, rowptr,
                         lut, stage, vals, rowcap, zero_first, err, checks);
}

// Row owners of a Dat: y[r] (+)= sum over the row's incidence list of stage[e*ND + i], in order.
template <int ND, class Ops>
__global__ void k_vec_pull(int64_t nrows, const int64_t *__restrict__ adjptr, const int32_t *__restrict__ adj,
                           const typename Ops::T *__restrict__ stage, double *__restrict__ y, int zero_first) {
  using T = typename Ops::T;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
    T s = Ops::zero();
    for (int64_t ai = adjptr[r]; ai < adjptr[r + 1]; ai++) s = Ops::add(s, stage[adj[ai]]);
    const double v = Ops::to_f64(s);
    y[r] = zero_first ? v : y[r] + v;
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <int DIM, int P, int FORM, class Ops>
cudaError_t mat_push(const AsmArgs &a, cudaStream_t s) {
  if (a.ncell > 0) k_mat_push<DIM, P, FORM, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a);
  return cudaGetLastError();
}
template <int DIM, int P, int FORM, class Ops>
cudaError_t mat_action_push(const AsmArgs &a, cudaStream_t s) {
  if (a.ncell > 0) k_mat_action_push<DIM, P, FORM, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a);
  return cudaGetLastError();
}
template <int DIM, int P, int FORM, class Ops>
cudaError_t action_push(const AsmArgs &a, cudaStream_t s) {
  if (a.ncell > 0) k_action_push<DIM, P, FORM, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a);
  return cudaGetLastError();
}
// The staging buffer (a.stage) holds ncell * ND * ND (Mat: full element rows) or ncell * ND (action,
// vector) values of the arithmetic type; AsmArgs.zero_first selects overwrite instead of INC in the
// row kernels.
inline int pull_blocks(int64_t n, int t) {
  int64_t b = (n + t - 1) / t;
  return (int)(b < 1 ? 1 : b > 152 * 32 ? 152 * 32 : b);
}

template <int DIM, int P, int FORM, class Ops>
cudaError_t mat_pull(const AsmArgs &a, cudaStream_t s) {
  using E = fe_gen::Elem<DIM, P>;
  using T = typename Ops::T;
  T *stage = static_cast<T *>(a.stage);
  constexpr size_t esm = ElemStaging<T, E::NUP>::kTransposed ? ElemStaging<T, E::NUP>::kSmem : 0;
  if (esm > 48 * 1024) {  // opt in once per kernel and device (the first call is never inside a capture)
    static bool opted[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !opted[dev]) {
      cudaError_t e = cudaFuncSetAttribute(k_mat_elem<DIM, P, FORM, Ops>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)esm);
      if (e != cudaSuccess) return e;
      if (dev >= 0 && dev < 64) opted[dev] = true;
    }
  }
  if (a.ncell > 0)
    k_mat_elem<DIM, P, FORM, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, esm, s>>>(a, stage);
  const int TB = 256, warps = TB / 32, groups = 32 / E::ND > 0 ? 32 / E::ND : 1;
  const size_t smem = (size_t)a.rowcap * warps * groups * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_mat_pull<E::ND, Ops>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (a.nrows > 0)
    k_mat_pull<E::ND, Ops><<<pull_blocks(a.nrows, warps * groups), TB, smem, s>>>(a.nrows, a.adjptr, a.adj, a.rowptr, a.lut,
                                                                          stage, a.vals, a.rowcap, a.zero_first,
                                                                          a.err, a.checks);
  return cudaGetLastError();
}

template <int DIM, int P, int FORM, class Ops>
cudaError_t action_pull(const AsmArgs &a, cudaStream_t s) {
  using E = fe_gen::Elem<DIM, P>;
  using T = typename Ops::T;
  T *stage = static_cast<T *>(a.stage);
  if (a.ncell > 0) k_action_elem<DIM, P, FORM, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a, stage);
  if (a.nrows > 0)
    k_vec_pull<E::ND, Ops><<<pull_blocks(a.nrows, 256), 256, 0, s>>>(a.nrows, a.adjptr, a.adj, stage, a.y, a.zero_first);
  return cudaGetLastError();
}

template <int DIM, int P, int Q, class Ops>
cudaError_t vec_pull(const AsmArgs &a, cudaStream_t s) {
  using S = fe_gen::Source<DIM, P, Q>;
  using T = typename Ops::T;
  T *stage = static_cast<T *>(a.stage);
  if (a.ncell > 0) k_vec_elem<DIM, P, Q, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a, stage);
  if (a.nrows > 0)
    k_vec_pull<S::ND, Ops><<<pull_blocks(a.nrows, 256), 256, 0, s>>>(a.nrows, a.adjptr, a.adj, stage, a.y, a.zero_first);
  return cudaGetLastError();
}

// The element stage alone (no row pass): each cell's K_e x_e (action) or b_e (linear form) into
// a.stage, ND values per cell at e ND, for reductions that consume them directly (rank-0 forms).
template <int DIM, int P, int FORM, class Ops>
cudaError_t action_elem(const AsmArgs &a, cudaStream_t s) {
  using T = typename Ops::T;
  if (a.ncell > 0)
    k_action_elem<DIM, P, FORM, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a, static_cast<T *>(a.stage));
  return cudaGetLastError();
}
template <int DIM, int P, int Q, class Ops>
cudaError_t vec_elem(const AsmArgs &a, cudaStream_t s) {
  using T = typename Ops::T;
  if (a.ncell > 0)
    k_vec_elem<DIM, P, Q, Ops><<<blocks_for(a.ncell, kPushThreads), kPushThreads, 0, s>>>(a, static_cast<T *>(a.stage));
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
  if (d.dim == D && d.degree == P && d.coeff_degree == Q) return &VEC<D, P, Q, OPS>;

}  // namespace kern
}  // namespace fe
