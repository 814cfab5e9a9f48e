// Strong Dirichlet conditions and a batched Jacobi-preconditioned CG engine.
//
// Dirichlet: symmetric elimination on the assembled CSR system, one thread per row (the row
// owner reads and rewrites only its own row, so the lift b_i -= A_ij g_j sees the assembled
// A_ij and no two threads touch the same entry).
//
// CG (Hestenes-Stiefel with M = diag(A), the solver of the Poisson experiment, Sec. 6.2): many
// independent systems advance together, two persistent launches per iteration for all of them.
// A system is cut into fixed tiles: 512 rows, or for a large system its rows split evenly over
// the resident blocks (one wave, no tail).  Dot products are Globals with SUM access
// (Sec. 4.4.2): every tile writes its partial sum to its own slot, and the tile that finishes
// last for that system (a device counter, no waiting) adds the slots in tile order.  So every
// system's arithmetic depends only on its own data and tiling: the iterates are bitwise the same
// whichever other systems share the launches.
//
//   launch A, per tile: w = A z (one FMA per nonzero), then per row q = w + beta q and
//            p = z + beta p (q = A p follows from p = z + beta p_old: A p = A z + beta A p_old),
//            partial p.q; last tile: alpha = rz / p.q
//   launch B, per tile: x += alpha p, r -= alpha q, z = r / diag, partials r.z and r.r;
//            last tile: beta = rz' / rz, convergence test ||r|| <= rtol ||b||
// FP64 arithmetic is the scarce resource on this GPU (about 1/64 of the FP32 rate), so the SpMV
// runs on z, which needs no per-entry update, instead of gathering z_j + beta p_old_j.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "fe_internal.h"

namespace fe {
namespace {

#ifndef FE_CG_TILE_ROWS
#define FE_CG_TILE_ROWS 512
#endif
// (tile rows and SELL batch were swept on GB300 over 256..2048 rows and 4..8 columns: 512 / 4
// balances large systems against the per-iteration latency of small ones)
constexpr int kCgThreads = 256;
constexpr int64_t kCgTileRows = FE_CG_TILE_ROWS;  // smallest tile (a multiple of 32 rows)
#ifndef FE_CG_SELL_BATCH
#define FE_CG_SELL_BATCH 4
#endif
constexpr int kSellBatch = FE_CG_SELL_BATCH;  // SELL columns whose loads are issued together
static_assert(FE_CG_TILE_ROWS % 32 == 0, "tiles are whole SELL-32 slices");

// Rows per tile of a system: 512, or for a system of more than 512 rows per resident block, its
// rows split evenly over the resident blocks (rounded up to whole 32-row slices), so that it runs
// as one wave with no tail.  Depends only on the system and the grid, never on the other systems
// in a launch, so a system's sums are the same alone and in a mix.
int64_t cg_tile_rows(int64_t nrows, int grid) {
  if (nrows <= kCgTileRows * (int64_t)grid) return kCgTileRows;
  return ((nrows + grid - 1) / grid + 31) / 32 * 32;
}

enum CgStatusCode : int { CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAXIT = 2, CG_BREAKDOWN = 3 };

struct CgSys {
  const int64_t *rowptr;
  const int32_t *colidx;
  const double *vals;
  const double *b;
  double *x, *r, *z, *q, *dinv, *part, *p;
  // A in slices of 32 consecutive rows stored column by column (SELL-32): slice s holds
  // (sptr[s+1] - sptr[s]) columns of 32 entries from svals/scols + 32 sptr[s]; a row's entries in
  // CSR order, then zeros (column = the row itself) up to the slice width
  const int64_t *sptr;
  const double *svals;
  const int32_t *scols;
  int64_t nrows;
  int64_t tile_rows;  // rows per tile (whole SELL-32 slices)
  int ntiles;
  double rz, alpha, beta, bnorm2, rnorm2, rtol;
  int iters, maxit, active, status;
  unsigned cnt;
  int bad;
};

struct CgTile {
  int sys, tile;
};

struct CgStat {
  int status, iters;
  double rnorm2, bnorm2;
};

thread_local char g_smsg[512];

// Sum over the block, fixed association: xor butterfly within warps, then warp 0 over the warp sums.
// Result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
  }
  return t;
}

// Called by the whole block after thread 0 stored this tile's partials: true in the block that
// completed the system's last tile.  Never waits.
__device__ __forceinline__ bool last_tile(unsigned *cnt, int ntiles, int *sh_last) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(cnt, 1u);
    *sh_last = prev == (unsigned)(ntiles - 1);
  }
  __syncthreads();
  return *sh_last != 0;
}

// Sum of part[t * 3 + slot] over t = 0..ntiles-1 in a fixed association: thread k adds tiles
// k, k + blockDim, ... in order, then block_sum.  Called by the whole block; result in thread 0.
__device__ __forceinline__ double block_tiles_sum(const double *part, int slot, int ntiles, double *sh) {
  double s = 0.0;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) s += __ldcg(part + (int64_t)t * 3 + slot);
  return block_sum(s, sh);
}

// ---------------------------------------------------------------------------------- Dirichlet
__global__ void k_dirichlet(int64_t nrows, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                            double *__restrict__ vals, double *__restrict__ b, const uint8_t *__restrict__ is_bc,
                            const double *__restrict__ g) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  const int64_t k0 = rowptr[i], k1 = rowptr[i + 1];
  if (is_bc[i]) {
    for (int64_t k = k0; k < k1; k++) vals[k] = colidx[k] == i ? 1.0 : 0.0;
    b[i] = g ? g[i] : 0.0;
    return;
  }
  double bi = b[i];
  for (int64_t k = k0; k < k1; k++) {
    const int32_t j = colidx[k];
    if (!is_bc[j]) continue;
    if (g) bi -= vals[k] * g[j];
    vals[k] = 0.0;
  }
  b[i] = bi;
}

// ---------------------------------------------------------------------------------- CG kernels
// SELL-32 layout: width of each slice (the longest of its 32 rows).  One warp per slice.
__global__ void k_sell_width(const int64_t *__restrict__ rowptr, int64_t nrows, int64_t nslices,
                             int32_t *__restrict__ width) {
  const int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (sl >= nslices) return;  // warp-uniform
  const int64_t i = sl * 32 + lane;
  const int len = i < nrows ? (int)(rowptr[i + 1] - rowptr[i]) : 0;
  const int w = __reduce_max_sync(0xffffffffu, len);
  if (lane == 0) width[sl] = w;
}

// SELL-32 layout: copy of the values and columns, padded with zeros on the row's own column.
__global__ void k_sell_fill(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                            const double *__restrict__ vals, int64_t nrows, int64_t nslices,
                            const int64_t *__restrict__ sptr, double *__restrict__ svals, int32_t *__restrict__ scols) {
  const int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (sl >= nslices) return;
  const int64_t i = sl * 32 + lane;
  const int64_t e0 = i < nrows ? rowptr[i] : 0;
  const int len = i < nrows ? (int)(rowptr[i + 1] - e0) : 0;
  const int32_t pad = i < nrows ? (int32_t)i : 0;
  const int64_t k0 = sptr[sl], width = sptr[sl + 1] - k0;
  for (int64_t k = 0; k < width; k++) {
    const int64_t d = (k0 + k) * 32 + lane;
    svals[d] = k < len ? vals[e0 + k] : 0.0;
    scols[d] = k < len ? colidx[e0 + k] : pad;
  }
}

// Initial residual of one system (grid = its tiles): r = b - A x, z = r / diag, p_old = 0.
__global__ void __launch_bounds__(kCgThreads) k_cg_init(CgSys *S) {
  __shared__ double sh[kCgThreads / 32];
  __shared__ int sh_last;
  const int t = blockIdx.x;
  const int64_t r0 = (int64_t)t * S->tile_rows;
  const int64_t r1 = r0 + S->tile_rows < S->nrows ? r0 + S->tile_rows : S->nrows;
  double rz = 0.0, rr = 0.0, bb = 0.0;
  int bad = 0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kCgThreads) {
    double d = 0.0, ax = 0.0;
    for (int64_t e = S->rowptr[i]; e < S->rowptr[i + 1]; e++) {
      const int32_t j = S->colidx[e];
      const double a = S->vals[e];
      if (j == i) d = a;
      ax += a * S->x[j];
    }
    if (!(d > 0.0)) bad = 1;
    const double di = 1.0 / d, bi = S->b[i], ri = bi - ax, zi = di * ri;
    S->dinv[i] = di;
    S->r[i] = ri;
    S->z[i] = zi;
    S->p[i] = 0.0;
    S->q[i] = 0.0;
    rz += ri * zi;
    rr += ri * ri;
    bb += bi * bi;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&S->bad, 1);
  rz = block_sum(rz, sh);
  rr = block_sum(rr, sh);
  bb = block_sum(bb, sh);
  if (threadIdx.x == 0) {
    S->part[(int64_t)t * 3 + 0] = rz;
    S->part[(int64_t)t * 3 + 1] = rr;
    S->part[(int64_t)t * 3 + 2] = bb;
  }
  if (last_tile(&S->cnt, S->ntiles, &sh_last)) {
    const double srz = block_tiles_sum(S->part, 0, S->ntiles, sh);
    const double srr = block_tiles_sum(S->part, 1, S->ntiles, sh);
    const double sbb = block_tiles_sum(S->part, 2, S->ntiles, sh);
    if (threadIdx.x == 0) {
      S->rz = srz;
      S->rnorm2 = srr;
      S->bnorm2 = sbb;
      S->beta = 0.0;
      S->alpha = 0.0;
      S->iters = 0;
      if (atomicOr(&S->bad, 0)) S->status = CG_BREAKDOWN;
      else if (sqrt(srr) <= S->rtol * sqrt(sbb)) S->status = CG_CONVERGED;
      else if (S->maxit <= 0) S->status = CG_MAXIT;
      else S->status = CG_RUNNING;
      S->active = S->status == CG_RUNNING;
      S->cnt = 0;
    }
  }
}

// Launch A: w = A z, q = w + beta q, p = z + beta p, p.q; last tile: alpha.  A warp takes one
// SELL-32 slice at a time: lane l owns row 32 s + l, every load of values and columns is one
// coalesced 256-byte access, kSellBatch columns in flight, and the row sum runs in CSR order.
__global__ void __launch_bounds__(kCgThreads, 6) k_cg_direction_spmv(CgSys *sys, const CgTile *__restrict__ tiles,
                                                                     const int *ntiles_p) {
  __shared__ double sh[kCgThreads / 32];
  __shared__ int sh_last;
  const int ntiles = *ntiles_p;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const CgTile tl = tiles[t];
    CgSys *S = sys + tl.sys;
    if (!S->active) continue;
    const double beta = S->beta;
    double *__restrict__ p = S->p;
    double *__restrict__ q = S->q;
    const double *__restrict__ z = S->z;
    const int64_t *__restrict__ sptr = S->sptr;
    const double *__restrict__ svals = S->svals;
    const int32_t *__restrict__ scols = S->scols;
    const int64_t nrows = S->nrows;
    const int64_t nsl = (nrows + 31) / 32;
    const int64_t tsl = S->tile_rows / 32;
    const int64_t s0 = (int64_t)tl.tile * tsl;
    const int64_t s1 = s0 + tsl < nsl ? s0 + tsl : nsl;
    double pq = 0.0;
    for (int64_t sl = s0 + warp; sl < s1; sl += kCgThreads / 32) {
      const int64_t k0 = sptr[sl];
      const int width = (int)(sptr[sl + 1] - k0);
      const double *__restrict__ vv = svals + k0 * 32 + lane;
      const int32_t *__restrict__ cc = scols + k0 * 32 + lane;
      double w = 0.0;
      int k = 0;
      for (; k + kSellBatch <= width; k += kSellBatch) {
        int32_t c[kSellBatch];
        double v[kSellBatch];
#pragma unroll
        for (int u = 0; u < kSellBatch; u++) {
          c[u] = __ldcs(cc + (int64_t)(k + u) * 32);  // streamed once per iteration: evict first, so
          v[u] = __ldcs(vv + (int64_t)(k + u) * 32);  // the vectors stay in L2 across the launches
        }
#pragma unroll
        for (int u = 0; u < kSellBatch; u++) w = fma(v[u], z[c[u]], w);
      }
      for (; k < width; k++) w = fma(__ldcs(vv + (int64_t)k * 32), z[__ldcs(cc + (int64_t)k * 32)], w);
      const int64_t i = sl * 32 + lane;
      if (i < nrows) {
        const double qi = w + beta * q[i];
        const double pi = z[i] + beta * p[i];
        q[i] = qi;
        p[i] = pi;
        pq += pi * qi;
      }
    }
    pq = block_sum(pq, sh);
    if (threadIdx.x == 0) S->part[(int64_t)tl.tile * 3] = pq;
    if (last_tile(&S->cnt, S->ntiles, &sh_last)) {
      const double s = block_tiles_sum(S->part, 0, S->ntiles, sh);
      if (threadIdx.x == 0) {
        if (!(s > 0.0)) {
          S->status = CG_BREAKDOWN;
          S->active = 0;
        } else {
          S->alpha = S->rz / s;
        }
        S->cnt = 0;
      }
    }
    __syncthreads();
  }
}

// Launch B: x, r, z; r.z and r.r; last tile: beta and the convergence test.
__global__ void __launch_bounds__(kCgThreads, 6) k_cg_update(CgSys *sys, const CgTile *__restrict__ tiles,
                                                          const int *ntiles_p) {
  __shared__ double sh[kCgThreads / 32];
  __shared__ int sh_last;
  const int ntiles = *ntiles_p;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const CgTile tl = tiles[t];
    CgSys *S = sys + tl.sys;
    if (!S->active) continue;
    const double alpha = S->alpha;
    const double *__restrict__ p = S->p;
    const double *__restrict__ q = S->q;
    const double *__restrict__ dinv = S->dinv;
    double *__restrict__ x = S->x;
    double *__restrict__ r = S->r;
    double *__restrict__ z = S->z;
    const int64_t r0 = (int64_t)tl.tile * S->tile_rows;
    const int64_t r1 = r0 + S->tile_rows < S->nrows ? r0 + S->tile_rows : S->nrows;
    double rz = 0.0, rr = 0.0;
#pragma unroll 2
    for (int64_t i = r0 + threadIdx.x; i < r1; i += kCgThreads) {
      x[i] += alpha * p[i];
      const double ri = r[i] - alpha * q[i];
      const double zi = dinv[i] * ri;
      r[i] = ri;
      z[i] = zi;
      rz += ri * zi;
      rr += ri * ri;
    }
    rz = block_sum(rz, sh);
    rr = block_sum(rr, sh);
    if (threadIdx.x == 0) {
      S->part[(int64_t)tl.tile * 3 + 1] = rz;
      S->part[(int64_t)tl.tile * 3 + 2] = rr;
    }
    if (last_tile(&S->cnt, S->ntiles, &sh_last)) {
      const double srz = block_tiles_sum(S->part, 1, S->ntiles, sh);
      const double srr = block_tiles_sum(S->part, 2, S->ntiles, sh);
      if (threadIdx.x == 0) {
        S->beta = srz / S->rz;
        S->rz = srz;
        S->rnorm2 = srr;
        S->iters += 1;
        if (sqrt(srr) <= S->rtol * sqrt(S->bnorm2)) {
          S->status = CG_CONVERGED;
          S->active = 0;
        } else if (S->iters >= S->maxit) {
          S->status = CG_MAXIT;
          S->active = 0;
        }
        S->cnt = 0;
      }
    }
    __syncthreads();
  }
}

__global__ void k_cg_pack(const CgSys *sys, int n, CgStat *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i].status = sys[i].status;
  out[i].iters = sys[i].iters;
  out[i].rnorm2 = sys[i].rnorm2;
  out[i].bnorm2 = sys[i].bnorm2;
}

}  // namespace

const char *solve_message() { return g_smsg; }

cudaError_t launch_dirichlet(int64_t nrows, const int64_t *rowptr, const int32_t *colidx, double *vals, double *b,
                             const uint8_t *is_bc, const double *g, cudaStream_t s) {
  if (nrows > 0) k_dirichlet<<<(unsigned)((nrows + 255) / 256), 256, 0, s>>>(nrows, rowptr, colidx, vals, b, is_bc, g);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------- CG engine
struct CgEngine {
  fe_ctx *ctx;
  int cap;
  CgSys *d_sys;
  CgStat *d_stat, *h_stat;  // h_stat pinned
  std::vector<CgSys> h_sys;
  std::vector<char> used;
  CgTile *d_tiles;
  int *d_ntiles;
  int tile_cap;
  bool dirty;
  int grid;
  cudaStream_t capture;
  cudaGraphExec_t graph;
  int graph_iters;
  int64_t launches;  // kernels launched by the engine (graph replays counted per kernel)
};

}  // namespace fe

struct fe_cg {
  uint32_t magic;
  fe::CgEngine *e;
};

namespace fe {
namespace {
constexpr uint32_t kMagicCg = 0xFE0C6E11u;

void drop_graph(CgEngine *e) {
  if (e->graph) cudaGraphExecDestroy(e->graph);
  e->graph = nullptr;
}

cudaError_t upload_tiles(CgEngine *e) {
  std::vector<CgTile> t;
  for (int s = 0; s < e->cap; s++)
    if (e->used[s])
      for (int k = 0; k < e->h_sys[s].ntiles; k++) t.push_back({s, k});
  if ((int)t.size() > e->tile_cap) {
    int cap = e->tile_cap;
    while (cap < (int)t.size()) cap *= 2;
    CgTile *nt = (CgTile *)dev_alloc(e->ctx, sizeof(CgTile) * cap);
    if (!nt) return cudaErrorMemoryAllocation;
    cudaStreamSynchronize(e->ctx->stream);
    dev_free(e->ctx, e->d_tiles);
    e->d_tiles = nt;
    e->tile_cap = cap;
    drop_graph(e);  // the graph holds the old table's address
  }
  const int n = (int)t.size();
  // pageable source: the copy has taken the data when the call returns
  cudaError_t err = cudaSuccess;
  if (n > 0) err = cudaMemcpyAsync(e->d_tiles, t.data(), sizeof(CgTile) * n, cudaMemcpyHostToDevice, e->ctx->stream);
  if (err == cudaSuccess) err = cudaMemcpyAsync(e->d_ntiles, &n, sizeof(int), cudaMemcpyHostToDevice, e->ctx->stream);
  if (err == cudaSuccess) e->dirty = false;
  return err;
}

cudaError_t launch_iterations(CgEngine *e, int iters, cudaStream_t s) {
  for (int k = 0; k < iters; k++) {
    k_cg_direction_spmv<<<e->grid, kCgThreads, 0, s>>>(e->d_sys, e->d_tiles, e->d_ntiles);
    k_cg_update<<<e->grid, kCgThreads, 0, s>>>(e->d_sys, e->d_tiles, e->d_ntiles);
  }
  return cudaGetLastError();
}

void free_sys_vectors(CgEngine *e, CgSys &S) {
  dev_free(e->ctx, S.r);
  dev_free(e->ctx, S.z);
  dev_free(e->ctx, S.q);
  dev_free(e->ctx, S.dinv);
  dev_free(e->ctx, S.p);
  dev_free(e->ctx, (void *)S.sptr);
  dev_free(e->ctx, (void *)S.svals);
  dev_free(e->ctx, (void *)S.scols);
  dev_free(e->ctx, S.part);
  memset(&S, 0, sizeof S);
}
}  // namespace

bool cg_valid(const fe_cg *h) { return h && h->magic == kMagicCg && h->e; }
int64_t cg_launches(const fe_cg *h) { return h->e->launches; }
int64_t cg_one_wave_rows(const fe_cg *h) { return kCgTileRows * (int64_t)h->e->grid; }
int cg_grid(const fe_cg *h) { return h->e->grid; }

fe_status cg_limit_grid(fe_cg *h, int grid) {
  CgEngine *e = h->e;
  for (int s = 0; s < e->cap; s++)
    if (e->used[s]) {
      snprintf(g_smsg, sizeof g_smsg, "cg_limit_grid: systems are already tiled for %d blocks", e->grid);
      return FE_EINVAL;
    }
  if (grid >= 1 && grid < e->grid) {
    e->grid = grid;
    drop_graph(e);
  }
  return FE_OK;
}
fe_ctx *cg_ctx(const fe_cg *h) { return h->e->ctx; }

fe_status cg_create(fe_ctx *c, int max_systems, fe_cg **out) {
  g_smsg[0] = 0;
  CgEngine *e = new (std::nothrow) CgEngine();
  if (!e) return FE_ENOMEM;
  e->ctx = c;
  e->cap = max_systems;
  e->h_sys.assign(max_systems, CgSys{});
  e->used.assign(max_systems, 0);
  e->tile_cap = 1024;
  int sms = 152, per_a = 4, per_b = 4, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_a, k_cg_direction_spmv, kCgThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_b, k_cg_update, kCgThreads, 0);
  e->grid = sms * (per_a < per_b ? per_a : per_b);  // one wave of resident CTAs
  if (e->grid < 1) e->grid = 152;
  e->graph = nullptr;
  e->graph_iters = 0;
  e->launches = 0;
  e->dirty = true;
  e->d_sys = (CgSys *)dev_alloc(c, sizeof(CgSys) * max_systems);
  e->d_stat = (CgStat *)dev_alloc(c, sizeof(CgStat) * max_systems);
  e->d_tiles = (CgTile *)dev_alloc(c, sizeof(CgTile) * e->tile_cap);
  e->d_ntiles = (int *)dev_alloc(c, sizeof(int));
  e->h_stat = nullptr;
  e->capture = nullptr;
  cudaError_t err = cudaHostAlloc((void **)&e->h_stat, sizeof(CgStat) * max_systems, cudaHostAllocDefault);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->capture, cudaStreamNonBlocking);
  if (err == cudaSuccess && (!e->d_sys || !e->d_stat || !e->d_tiles || !e->d_ntiles)) err = cudaErrorMemoryAllocation;
  if (err == cudaSuccess) err = cudaMemsetAsync(e->d_sys, 0, sizeof(CgSys) * max_systems, c->stream);
  if (err == cudaSuccess) err = upload_tiles(e);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  fe_cg *h = err == cudaSuccess ? new (std::nothrow) fe_cg{kMagicCg, e} : nullptr;
  if (!h) {
    if (err != cudaSuccess) snprintf(g_smsg, sizeof g_smsg, "fe_cg_create: %s", cudaGetErrorString(err));
    cudaGetLastError();
    dev_free(c, e->d_sys);
    dev_free(c, e->d_stat);
    dev_free(c, e->d_tiles);
    dev_free(c, e->d_ntiles);
    if (e->h_stat) cudaFreeHost(e->h_stat);
    if (e->capture) cudaStreamDestroy(e->capture);
    delete e;
    return err == cudaErrorMemoryAllocation || err == cudaSuccess ? FE_ENOMEM : FE_ECUDA;
  }
  *out = h;
  return FE_OK;
}

fe_status cg_add(fe_cg *h, const int64_t *rowptr, const int32_t *colidx, const double *vals, int64_t nrows,
                 const double *b, double *x, double rtol, int maxit, int *slot, int maxrow) {
  CgEngine *e = h->e;
  g_smsg[0] = 0;
  int s = -1;
  for (int k = 0; k < e->cap; k++)
    if (!e->used[k]) {
      s = k;
      break;
    }
  if (s < 0) {
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_add: all %d slots are in use", e->cap);
    return FE_EINVAL;
  }
  const int64_t tile_rows = cg_tile_rows(nrows, e->grid);
  const int64_t ntiles = nrows > 0 ? (nrows + tile_rows - 1) / tile_rows : 0;
  if (ntiles > INT32_MAX / 2) {
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_add: %lld rows is too many", (long long)nrows);
    return FE_EUNSUPPORTED;
  }
  CgSys S;
  memset(&S, 0, sizeof S);
  S.rowptr = rowptr;
  S.colidx = colidx;
  S.vals = vals;
  S.b = b;
  S.x = x;
  S.nrows = nrows;
  S.tile_rows = tile_rows;
  S.ntiles = (int)ntiles;
  S.rtol = rtol;
  S.maxit = maxit;
  const size_t vb = sizeof(double) * (nrows > 0 ? nrows : 1);
  S.r = (double *)dev_alloc(e->ctx, vb);
  S.z = (double *)dev_alloc(e->ctx, vb);
  S.q = (double *)dev_alloc(e->ctx, vb);
  S.dinv = (double *)dev_alloc(e->ctx, vb);
  S.p = (double *)dev_alloc(e->ctx, vb);
  S.part = (double *)dev_alloc(e->ctx, sizeof(double) * 3 * (ntiles > 0 ? ntiles : 1));
  if (!S.r || !S.z || !S.q || !S.dinv || !S.p || !S.part) {
    free_sys_vectors(e, S);
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_add: device allocation failed");
    return FE_ENOMEM;
  }
  // SELL-32 copy of A: slice widths, their prefix sums, then the padded values and columns
  cudaStream_t st0 = e->ctx->stream;
  const int64_t nsl = (nrows + 31) / 32;
  int64_t *sptr = (int64_t *)dev_alloc(e->ctx, sizeof(int64_t) * (nsl + 1));
  int32_t *width = (int32_t *)dev_alloc(e->ctx, sizeof(int32_t) * (nsl > 0 ? nsl : 1));
  int64_t *tmp = (int64_t *)dev_alloc(e->ctx, sizeof(int64_t) * scan_tmp_elems(nsl));
  S.sptr = sptr;
  int64_t ncol = 0;
  cudaError_t err0 = (sptr && width && tmp) ? cudaSuccess : cudaErrorMemoryAllocation;
  if (err0 == cudaSuccess && nsl > 0) {
    k_sell_width<<<(unsigned)((nsl * 32 + 255) / 256), 256, 0, st0>>>(rowptr, nrows, nsl, width);
    err0 = cudaGetLastError();
  }
  if (err0 == cudaSuccess) err0 = exclusive_scan_i32_to_i64(width, sptr, nsl, tmp, st0);
  if (maxrow > 0) {
    // every slice is at most the longest row wide: size the copy for that and do not wait for
    // the exact total (no host synchronisation in the set-up)
    ncol = nsl * (int64_t)maxrow;
  } else {
    if (err0 == cudaSuccess) err0 = cudaMemcpyAsync(&ncol, sptr + nsl, sizeof(int64_t), cudaMemcpyDeviceToHost, st0);
    if (err0 == cudaSuccess) err0 = cudaStreamSynchronize(st0);
  }
  dev_free(e->ctx, width);
  dev_free(e->ctx, tmp);
  if (err0 == cudaSuccess) {
    S.svals = (double *)dev_alloc(e->ctx, sizeof(double) * 32 * (ncol > 0 ? ncol : 1));
    S.scols = (int32_t *)dev_alloc(e->ctx, sizeof(int32_t) * 32 * (ncol > 0 ? ncol : 1));
    if (!S.svals || !S.scols) err0 = cudaErrorMemoryAllocation;
  }
  if (err0 == cudaSuccess && nsl > 0) {
    k_sell_fill<<<(unsigned)((nsl * 32 + 255) / 256), 256, 0, st0>>>(rowptr, colidx, vals, nrows, nsl, sptr,
                                                                     (double *)S.svals, (int32_t *)S.scols);
    err0 = cudaGetLastError();
    e->launches += 5;  // width, three scan passes, fill
  }
  if (err0 != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(st0);
    free_sys_vectors(e, S);
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_add: sliced copy of A: %s", cudaGetErrorString(err0));
    return err0 == cudaErrorMemoryAllocation ? FE_ENOMEM : FE_ECUDA;
  }
  if (nrows == 0) S.status = CG_CONVERGED;  // nothing to solve
  cudaStream_t st = e->ctx->stream;
  cudaError_t err = cudaMemcpyAsync(e->d_sys + s, &S, sizeof S, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess && ntiles > 0) {
    k_cg_init<<<(unsigned)ntiles, kCgThreads, 0, st>>>(e->d_sys + s);
    err = cudaGetLastError();
    e->launches++;
  }
  if (err != cudaSuccess) {
    cudaStreamSynchronize(st);
    free_sys_vectors(e, S);
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_add: %s", cudaGetErrorString(err));
    return FE_ECUDA;
  }
  e->h_sys[s] = S;
  e->used[s] = 1;
  e->dirty = true;
  *slot = s;
  return FE_OK;
}

fe_status cg_iterate(fe_cg *h, int iters, int use_graph) {
  CgEngine *e = h->e;
  g_smsg[0] = 0;
  cudaStream_t st = e->ctx->stream;
  cudaError_t err = cudaSuccess;
  if (e->dirty) err = upload_tiles(e);
  if (err == cudaSuccess && iters > 0) {
    if (!use_graph) {
      err = launch_iterations(e, iters, st);
    } else {
      if (e->graph && e->graph_iters != iters) drop_graph(e);
      if (!e->graph) {
        cudaGraph_t g = nullptr;
        err = cudaStreamBeginCapture(e->capture, cudaStreamCaptureModeThreadLocal);
        if (err == cudaSuccess) {
          cudaError_t el = launch_iterations(e, iters, e->capture);
          err = cudaStreamEndCapture(e->capture, &g);
          if (err == cudaSuccess) err = el;
        }
        if (err == cudaSuccess) err = cudaGraphInstantiate(&e->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (err != cudaSuccess) e->graph = nullptr;
        else e->graph_iters = iters;
      }
      if (err == cudaSuccess) err = cudaGraphLaunch(e->graph, st);
    }
    if (err == cudaSuccess) e->launches += 2 * (int64_t)iters;
  }
  if (err != cudaSuccess) {
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_iterate: %s", cudaGetErrorString(err));
    return FE_ECUDA;
  }
  return FE_OK;
}

fe_status cg_poll(fe_cg *h, int n, int *status, int *iters, double *rnorm, double *bnorm) {
  CgEngine *e = h->e;
  g_smsg[0] = 0;
  if (n < 0 || n > e->cap) {
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_poll: %d slots asked, the engine has %d", n, e->cap);
    return FE_EINVAL;
  }
  cudaStream_t st = e->ctx->stream;
  k_cg_pack<<<(e->cap + 127) / 128, 128, 0, st>>>(e->d_sys, e->cap, e->d_stat);
  cudaError_t err = cudaGetLastError();
  e->launches++;
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(e->h_stat, e->d_stat, sizeof(CgStat) * e->cap, cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) {
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_poll: %s", cudaGetErrorString(err));
    return FE_ECUDA;
  }
  for (int s = 0; s < n; s++) {
    const bool u = e->used[s] != 0;
    if (status) status[s] = u ? e->h_stat[s].status : -1;
    if (iters) iters[s] = u ? e->h_stat[s].iters : 0;
    if (rnorm) rnorm[s] = u ? sqrt(e->h_stat[s].rnorm2) : 0.0;
    if (bnorm) bnorm[s] = u ? sqrt(e->h_stat[s].bnorm2) : 0.0;
  }
  return FE_OK;
}

fe_status cg_remove(fe_cg *h, int slot) {
  CgEngine *e = h->e;
  if (slot < 0 || slot >= e->cap || !e->used[slot]) {
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_remove: slot %d is not in use", slot);
    return FE_EINVAL;
  }
  cudaStream_t st = e->ctx->stream;
  cudaStreamSynchronize(st);  // no launch in flight may still read the system
  CgSys dead;
  memset(&dead, 0, sizeof dead);
  cudaError_t err = cudaMemcpyAsync(e->d_sys + slot, &dead, sizeof dead, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  free_sys_vectors(e, e->h_sys[slot]);
  e->used[slot] = 0;
  e->dirty = true;
  if (err != cudaSuccess) {
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_remove: %s", cudaGetErrorString(err));
    return FE_ECUDA;
  }
  return FE_OK;
}

void cg_destroy(fe_cg *h) {
  if (!h) return;
  CgEngine *e = h->e;
  cudaStreamSynchronize(e->ctx->stream);
  for (int s = 0; s < e->cap; s++)
    if (e->used[s]) free_sys_vectors(e, e->h_sys[s]);
  drop_graph(e);
  dev_free(e->ctx, e->d_sys);
  dev_free(e->ctx, e->d_stat);
  dev_free(e->ctx, e->d_tiles);
  dev_free(e->ctx, e->d_ntiles);
  cudaFreeHost(e->h_stat);
  cudaStreamDestroy(e->capture);
  delete e;
  h->magic = 0xDEADu;
  h->e = nullptr;
  delete h;
}

}  // namespace fe
