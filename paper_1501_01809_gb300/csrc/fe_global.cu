// Reductions into a Global (Sec. 4.3; "Global arguments", Sec. 4.4): the sum of a rank-0 form
// over the cells, and the sum, minimum or maximum of the cells' volumes.
//
// Each block takes kRedCells consecutive cells; thread t adds cells t, t + kRedThreads, ... of
// that range in order, the block combines its threads in a fixed tree, and writes one partial;
// a single block then combines the partials in block order into the Global.  The paper lets the
// runtime keep one variable per parallel worker and reduce them afterwards; here the workers and
// the order of that last reduction are fixed, so nothing depends on scheduling and a result is
// the same on every run.
#include "fe_kernels.cuh"

namespace fe {
namespace {
using namespace kern;

constexpr int kRedThreads = 256;
constexpr int kRedCells = 2048;

template <int OP>
__device__ __forceinline__ double combine(double a, double b) {
  if constexpr (OP == FE_REDUCE_SUM) return a + b;
  else if constexpr (OP == FE_REDUCE_MIN) return b < a ? b : a;
  else return b > a ? b : a;
}
template <int OP>
__device__ __forceinline__ double identity() {
  if constexpr (OP == FE_REDUCE_SUM) return 0.0;
  else if constexpr (OP == FE_REDUCE_MIN) return __longlong_as_double(0x7FF0000000000000ll);  // +inf
  else return __longlong_as_double((long long)0xFFF0000000000000ull);                         // -inf
}

// Fixed-shape tree over the block's kRedThreads values; the result in every thread.
template <int OP>
__device__ __forceinline__ double block_reduce(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = combine<OP>(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// part[b] = sum over block b's cells e of sum_i x[map(e)[i]] stage[e nd + i], each cell's nd terms
// added in order.  In check mode a map value outside x is flagged and its term skipped.
template <class Ops>
__global__ void __launch_bounds__(kRedThreads) k_global_dot(int64_t ncell, int nd, const int32_t *__restrict__ map,
                                                            const typename Ops::T *__restrict__ stage,
                                                            const double *__restrict__ x, int64_t nx,
                                                            double *__restrict__ part, int checks, int *err) {
  __shared__ double sh[kRedThreads];
  const int64_t e0 = (int64_t)blockIdx.x * kRedCells;
  const int64_t e1 = e0 + kRedCells < ncell ? e0 + kRedCells : ncell;
  double s = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += kRedThreads) {
    double c = 0.0;
    for (int i = 0; i < nd; i++) {
      const int32_t r = map[e * nd + i];
      if (checks && (r < 0 || r >= nx)) {
        flag(err, ERR_RANGE, e);
        continue;
      }
      c += x[r] * Ops::to_f64(stage[e * nd + i]);
    }
    s += c;
  }
  const double b = block_reduce<FE_REDUCE_SUM>(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// part[b] = op over block b's cells of |det J| / dim!, J the edge vectors from vertex 0.
template <int DIM, int OP>
__global__ void __launch_bounds__(kRedThreads) k_volume(int64_t ncell, const int32_t *__restrict__ cmapv,
                                                        const double *__restrict__ coords, int64_t nvert,
                                                        double *__restrict__ part, int checks, int *err) {
  __shared__ double sh[kRedThreads];
  const int64_t e0 = (int64_t)blockIdx.x * kRedCells;
  const int64_t e1 = e0 + kRedCells < ncell ? e0 + kRedCells : ncell;
  double s = identity<OP>();
  for (int64_t e = e0 + threadIdx.x; e < e1; e += kRedThreads) {
    double x[DIM + 1][DIM];
    bool ok = true;
#pragma unroll
    for (int v = 0; v <= DIM; v++) {
      int32_t q = cmapv[e * (DIM + 1) + v];
      if (checks && (q < 0 || q >= nvert)) {
        ok = false;
        q = 0;
      }
#pragma unroll
      for (int k = 0; k < DIM; k++) x[v][k] = coords[(int64_t)q * DIM + k];
    }
    if (!ok) {
      flag(err, ERR_RANGE, e);
      continue;
    }
    double det;
    if constexpr (DIM == 2) {
      det = (x[1][0] - x[0][0]) * (x[2][1] - x[0][1]) - (x[2][0] - x[0][0]) * (x[1][1] - x[0][1]);
    } else {
      const double a[3] = {x[1][0] - x[0][0], x[1][1] - x[0][1], x[1][2] - x[0][2]};
      const double b[3] = {x[2][0] - x[0][0], x[2][1] - x[0][1], x[2][2] - x[0][2]};
      const double c[3] = {x[3][0] - x[0][0], x[3][1] - x[0][1], x[3][2] - x[0][2]};
      det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    s = combine<OP>(s, fabs(det) / (DIM == 2 ? 2.0 : 6.0));
  }
  const double b = block_reduce<OP>(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// One block: *g = (or op=) the partials combined in block order.
template <int OP>
__global__ void __launch_bounds__(kRedThreads) k_reduce_parts(const double *__restrict__ part, int64_t n, double *g,
                                                              int zero_first) {
  __shared__ double sh[kRedThreads];
  double s = identity<OP>();
  for (int64_t b = threadIdx.x; b < n; b += kRedThreads) s = combine<OP>(s, part[b]);
  const double t = block_reduce<OP>(s, sh);
  if (threadIdx.x == 0) *g = zero_first ? t : combine<OP>(*g, t);
}

template <int DIM, int OP>
cudaError_t volume(int64_t ncell, const int32_t *cmapv, const double *coords, int64_t nvert, double *part, double *g,
                   int zero_first, int checks, int *err, cudaStream_t s) {
  const int64_t nb = global_parts(ncell);
  if (ncell > 0) k_volume<DIM, OP><<<(unsigned)nb, kRedThreads, 0, s>>>(ncell, cmapv, coords, nvert, part, checks, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_parts<OP><<<1, kRedThreads, 0, s>>>(part, ncell > 0 ? nb : 0, g, zero_first);
  return cudaGetLastError();
}

}  // namespace

int64_t global_parts(int64_t ncell) { return ncell > 0 ? (ncell + kRedCells - 1) / kRedCells : 1; }

cudaError_t launch_global_dot(int precision, int64_t ncell, int nd, const int32_t *map, const void *stage,
                              const double *x, int64_t nx, double *part, double *g, int zero_first, int checks,
                              int *err, cudaStream_t s) {
  const int64_t nb = global_parts(ncell);
  if (nb > INT32_MAX) return cudaErrorInvalidValue;
  if (ncell > 0) {
    if (precision == FE_PREC_F32X2)
      k_global_dot<OpsF32x2><<<(unsigned)nb, kRedThreads, 0, s>>>(
          ncell, nd, map, static_cast<const OpsF32x2::T *>(stage), x, nx, part, checks, err);
    else
      k_global_dot<OpsF64><<<(unsigned)nb, kRedThreads, 0, s>>>(ncell, nd, map, static_cast<const double *>(stage), x,
                                                                nx, part, checks, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_reduce_parts<FE_REDUCE_SUM><<<1, kRedThreads, 0, s>>>(part, ncell > 0 ? nb : 0, g, zero_first);
  return cudaGetLastError();
}

cudaError_t launch_cell_volume_reduce(int dim, int op, int64_t ncell, const int32_t *cmapv, const double *coords,
                                      int64_t nvert, double *part, double *g, int zero_first, int checks, int *err,
                                      cudaStream_t s) {
  if (global_parts(ncell) > INT32_MAX) return cudaErrorInvalidValue;
  const auto go = [&](auto fn) { return fn(ncell, cmapv, coords, nvert, part, g, zero_first, checks, err, s); };
  if (dim == 2) {
    if (op == FE_REDUCE_SUM) return go(volume<2, FE_REDUCE_SUM>);
    if (op == FE_REDUCE_MIN) return go(volume<2, FE_REDUCE_MIN>);
    return go(volume<2, FE_REDUCE_MAX>);
  }
  if (op == FE_REDUCE_SUM) return go(volume<3, FE_REDUCE_SUM>);
  if (op == FE_REDUCE_MIN) return go(volume<3, FE_REDUCE_MIN>);
  return go(volume<3, FE_REDUCE_MAX>);
}

}  // namespace fe
