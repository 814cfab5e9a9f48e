// Assembly of the systems that the request loop admits together: two launches for all of them,
// so the fixed cost per field and par_loop that the paper measures (Sec. 6.4.2) is paid once per
// admission round instead of once per request and kernel.
//
// Each system is the Poisson problem of Sec. 3.1: a = inner(grad u, grad v) dx on P1 or P2
// triangles, L = f v dx with f in the same space, u = 0 on the flagged nodes.  Launch 1 takes
// tiles of kServeCellTile cells of any system (a block finds its system from its tile number) and
// stages every cell's element matrix and element vector.  Launch 2 takes tiles of kServeRowTile
// rows: the deterministic row owners of the Mat (incidence order, the loop of the single-system
// pull kernel) with the boundary rows and columns eliminated as each row is written out, then
// the right-hand side rows.  Every value is the one that the per-request launches (pull assembly
// of the Mat and of the vector, then the elimination kernel) give, bit for bit: the same device
// functions add the same terms in the same order.
#include "fe_kernels.cuh"

namespace fe {
namespace {
using namespace kern;

constexpr int kRowThreads = 256;

// The last system whose first tile is at most t.  A system without tiles is never chosen: the
// next one starts at the same tile, and none follows the last tile of the last system.
__device__ __forceinline__ int find_item(const ServeItem *__restrict__ items, int n, int64_t t, bool rows) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int64_t f = rows ? items[mid].row_tile0 : items[mid].cell_tile0;
    if (f <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One tile of cells: the element matrix (staged as full rows) and the element vector of each.
template <int P, class Ops>
__device__ __forceinline__ void elem_tile(const ServeItem &it, int64_t e0) {
  using T = typename Ops::T;
  using E = fe_gen::Elem<2, P>;
  T *ms = static_cast<T *>(it.mstage);
  const int64_t e = e0 + threadIdx.x;
  if constexpr (ElemStaging<T, E::NUP>::kTransposed) {
    __shared__ unsigned char ok[kServeCellTile];
    ok[threadIdx.x] = e < it.mat.ncell && mat_elem_cell<2, P, FE_FORM_LAPLACE, Ops>(it.mat, ms, e);
    __syncthreads();
    copy_elem_block<T, E::ND>(ms, e0, it.mat.ncell, ok);
  } else {
    if (e < it.mat.ncell) mat_elem_cell<2, P, FE_FORM_LAPLACE, Ops>(it.mat, ms, e);
  }
  if (e < it.vec.ncell) vec_elem_cell<2, P, P, Ops>(it.vec, static_cast<T *>(it.vstage), e);
}

template <class Ops>
__global__ void __launch_bounds__(kServeCellTile) k_serve_elem(const ServeItem *__restrict__ items, int n) {
  __shared__ int s_item;
  if (threadIdx.x == 0) s_item = find_item(items, n, blockIdx.x, false);
  __syncthreads();
  const ServeItem &it = items[s_item];
  const int64_t e0 = ((int64_t)blockIdx.x - it.cell_tile0) * kServeCellTile;
  if (it.p == 1) elem_tile<1, Ops>(it, e0);  // uniform across the block
  else elem_tile<2, Ops>(it, e0);
}

// One tile of rows: the Mat rows (row groups of ND lanes, boundary elimination on write-out),
// then the right-hand side rows (one thread per row, its incidence list in order).
template <int ND, class Ops>
__device__ __forceinline__ void rows_tile(const ServeItem &it, int64_t r0) {
  using T = typename Ops::T;
  constexpr int NG = 32 / ND;
  extern __shared__ __align__(16) unsigned char sm_rows[];
  const AsmArgs &a = it.mat;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int gi = lane / ND, j = lane - (lane / ND) * ND;
  const bool on = gi < NG;
  T *buf = reinterpret_cast<T *>(sm_rows) + ((size_t)wid * NG + (on ? gi : 0)) * a.rowcap;
  const int64_t rend = r0 + kServeRowTile < a.nrows ? r0 + kServeRowTile : a.nrows;
  pull_mat_rows<ND, Ops, true>(r0 + (int64_t)wid * NG + gi, (int64_t)wpb * NG, rend, on, j, buf, a.adjptr, a.adj,
                               a.rowptr, a.lut, static_cast<const T *>(it.mstage), a.vals, a.rowcap, a.zero_first,
                               a.err, a.checks, it.colidx, it.is_bc);
  const T *vs = static_cast<const T *>(it.vstage);
  for (int64_t r = r0 + threadIdx.x; r < rend; r += blockDim.x) {
    T s = Ops::zero();
    for (int64_t ai = a.adjptr[r]; ai < a.adjptr[r + 1]; ai++) s = Ops::add(s, vs[a.adj[ai]]);
    const double v = Ops::to_f64(s), y = it.vec.zero_first ? v : it.vec.y[r] + v;
    it.vec.y[r] = it.is_bc[r] ? 0.0 : y;  // a flagged row's right-hand side is its boundary value, 0
  }
}

template <class Ops>
__global__ void __launch_bounds__(kRowThreads) k_serve_rows(const ServeItem *__restrict__ items, int n) {
  __shared__ int s_item;
  if (threadIdx.x == 0) s_item = find_item(items, n, blockIdx.x, true);
  __syncthreads();
  const ServeItem &it = items[s_item];
  const int64_t r0 = ((int64_t)blockIdx.x - it.row_tile0) * kServeRowTile;
  if (it.p == 1) rows_tile<fe_gen::Elem<2, 1>::ND, Ops>(it, r0);  // uniform across the block
  else rows_tile<fe_gen::Elem<2, 2>::ND, Ops>(it, r0);
}

template <class T, int NUP>
constexpr size_t elem_smem() {
  return ElemStaging<T, NUP>::kTransposed ? ElemStaging<T, NUP>::kSmem : 0;
}

template <class Ops>
cudaError_t launch(const ServeItem *d, int n, int64_t cell_tiles, int64_t row_tiles, size_t row_smem, cudaStream_t s) {
  using T = typename Ops::T;
  constexpr size_t e1 = elem_smem<T, fe_gen::Elem<2, 1>::NUP>(), e2 = elem_smem<T, fe_gen::Elem<2, 2>::NUP>();
  constexpr size_t esm = e1 > e2 ? e1 : e2;
  static_assert(esm <= 48 * 1024, "element staging of the serving batch needs no opt-in");
  if (cell_tiles > 0) {
    k_serve_elem<Ops><<<(unsigned)cell_tiles, kServeCellTile, esm, s>>>(d, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (row_tiles > 0) {
    if (row_smem > 48 * 1024) {
      const cudaError_t e =
          cudaFuncSetAttribute(k_serve_rows<Ops>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem);
      if (e != cudaSuccess) return e;
    }
    k_serve_rows<Ops><<<(unsigned)row_tiles, kRowThreads, row_smem, s>>>(d, n);
  }
  return cudaGetLastError();
}

}  // namespace

size_t serve_row_smem(int p, int rowcap, int precision) {
  const int nd = (p + 1) * (p + 2) / 2, ng = 32 / nd;
  const size_t t = precision == FE_PREC_F32X2 ? sizeof(OpsF32x2::T) : sizeof(double);
  return (size_t)(rowcap > 0 ? rowcap : 1) * (kRowThreads / 32) * ng * t;
}

cudaError_t launch_serve_assembly(const ServeItem *d_items, int nitems, int64_t cell_tiles, int64_t row_tiles,
                                  size_t row_smem, int precision, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (cell_tiles > INT32_MAX || row_tiles > INT32_MAX) return cudaErrorInvalidValue;
  if (precision == FE_PREC_F32X2) return launch<OpsF32x2>(d_items, nitems, cell_tiles, row_tiles, row_smem, s);
  return launch<OpsF64>(d_items, nitems, cell_tiles, row_tiles, row_smem, s);
}

}  // namespace fe
