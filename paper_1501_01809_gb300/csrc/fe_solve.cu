// Strong Dirichlet conditions and a batched Jacobi-preconditioned CG engine.
//
// Dirichlet: symmetric elimination on the assembled CSR system, one thread per row (the row
// owner reads and rewrites only its own row, so the lift b_i -= A_ij g_j sees the assembled
// A_ij and no two threads touch the same entry).
//
// CG (Hestenes-Stiefel with M = diag(A), the solver of the Poisson experiment, Sec. 6.2): many
// independent systems advance together, two persistent launches per iteration for all of them.
// A system is cut into fixed tiles of kCgTileRows rows.  Dot products are Globals with SUM access
// (Sec. 4.4.2): every tile writes its partial sum to its own slot, and the tile that finishes
// last for that system (a device counter, no waiting) adds the slots in tile order.  So every
// system's arithmetic depends only on its own data and tiling: the iterates are bitwise the same
// whichever other systems share the launches.
//
//   launch A, per tile: p_new = z + beta p_old (rows of the tile, stored), q = A p_new (gathering
//            z_j + beta p_old_j for the columns), partial p_new.q; last tile: alpha = rz / p.q
//   launch B, per tile: x += alpha p_new, r -= alpha q, z = r / diag, partials r.z and r.r;
//            last tile: beta = rz' / rz, convergence test ||r|| <= rtol ||b||, swap p buffers
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "fe_internal.h"

namespace fe {
namespace {

constexpr int kCgThreads = 256;
constexpr int kCgRowsPerThread = 4;
constexpr int64_t kCgTileRows = kCgThreads * kCgRowsPerThread;

enum CgStatusCode : int { CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAXIT = 2, CG_BREAKDOWN = 3 };

struct CgSys {
  const int64_t *rowptr;
  const int32_t *colidx;
  const double *vals;
  const double *b;
  double *x, *r, *z, *q, *dinv, *part;
  double *p[2];
  int64_t nrows;
  int ntiles, cur;
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

// Sum of part[t * 3 + slot] over t = 0..ntiles-1 in a fixed association (warp 0; lane l takes
// t = l, l + 32, ... in order, then the xor butterfly).  Result valid in lane 0.
__device__ __forceinline__ double ordered_tiles_sum(const double *part, int slot, int ntiles) {
  const int l = threadIdx.x & 31;
  double s = 0.0;
  for (int t = l; t < ntiles; t += 32) s += __ldcg(part + (int64_t)t * 3 + slot);
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  return s;
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
// Initial residual of one system (grid = its tiles): r = b - A x, z = r / diag, p_old = 0.
__global__ void __launch_bounds__(kCgThreads) k_cg_init(CgSys *S) {
  __shared__ double sh[kCgThreads / 32];
  __shared__ int sh_last;
  const int t = blockIdx.x;
  const int64_t r0 = (int64_t)t * kCgTileRows;
  double rz = 0.0, rr = 0.0, bb = 0.0;
  int bad = 0;
  for (int k = 0; k < kCgRowsPerThread; k++) {
    const int64_t i = r0 + k * kCgThreads + threadIdx.x;
    if (i >= S->nrows) break;
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
    S->p[0][i] = 0.0;
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
  if (last_tile(&S->cnt, S->ntiles, &sh_last) && threadIdx.x < 32) {
    const double srz = ordered_tiles_sum(S->part, 0, S->ntiles);
    const double srr = ordered_tiles_sum(S->part, 1, S->ntiles);
    const double sbb = ordered_tiles_sum(S->part, 2, S->ntiles);
    if (threadIdx.x == 0) {
      S->rz = srz;
      S->rnorm2 = srr;
      S->bnorm2 = sbb;
      S->beta = 0.0;
      S->alpha = 0.0;
      S->cur = 0;
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

// Launch A: new direction, q = A p, p.q; last tile: alpha.
__global__ void __launch_bounds__(kCgThreads) k_cg_direction_spmv(CgSys *sys, const CgTile *__restrict__ tiles,
                                                                  const int *ntiles_p) {
  __shared__ double sh[kCgThreads / 32];
  __shared__ int sh_last;
  const int ntiles = *ntiles_p;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const CgTile tl = tiles[t];
    CgSys *S = sys + tl.sys;
    if (!S->active) continue;
    const double beta = S->beta;
    const int cur = S->cur;
    const double *__restrict__ pold = S->p[cur];
    double *__restrict__ pnew = S->p[cur ^ 1];
    const double *__restrict__ z = S->z;
    const int64_t *__restrict__ rowptr = S->rowptr;
    const int32_t *__restrict__ colidx = S->colidx;
    const double *__restrict__ vals = S->vals;
    const int64_t r0 = (int64_t)tl.tile * kCgTileRows, nrows = S->nrows;
    double pq = 0.0;
    for (int k = 0; k < kCgRowsPerThread; k++) {
      const int64_t i = r0 + k * kCgThreads + threadIdx.x;
      if (i >= nrows) break;
      double acc = 0.0;
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
        const int32_t j = colidx[e];
        acc += vals[e] * (z[j] + beta * pold[j]);
      }
      const double pn = z[i] + beta * pold[i];
      pnew[i] = pn;
      S->q[i] = acc;
      pq += pn * acc;
    }
    pq = block_sum(pq, sh);
    if (threadIdx.x == 0) S->part[(int64_t)tl.tile * 3] = pq;
    if (last_tile(&S->cnt, S->ntiles, &sh_last) && threadIdx.x < 32) {
      const double s = ordered_tiles_sum(S->part, 0, S->ntiles);
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

// Launch B: x, r, z; r.z and r.r; last tile: beta, convergence, buffer swap.
__global__ void __launch_bounds__(kCgThreads) k_cg_update(CgSys *sys, const CgTile *__restrict__ tiles,
                                                          const int *ntiles_p) {
  __shared__ double sh[kCgThreads / 32];
  __shared__ int sh_last;
  const int ntiles = *ntiles_p;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const CgTile tl = tiles[t];
    CgSys *S = sys + tl.sys;
    if (!S->active) continue;
    const double alpha = S->alpha;
    const double *__restrict__ pn = S->p[S->cur ^ 1];
    const int64_t r0 = (int64_t)tl.tile * kCgTileRows, nrows = S->nrows;
    double rz = 0.0, rr = 0.0;
    for (int k = 0; k < kCgRowsPerThread; k++) {
      const int64_t i = r0 + k * kCgThreads + threadIdx.x;
      if (i >= nrows) break;
      S->x[i] += alpha * pn[i];
      const double ri = S->r[i] - alpha * S->q[i];
      const double zi = S->dinv[i] * ri;
      S->r[i] = ri;
      S->z[i] = zi;
      rz += ri * zi;
      rr += ri * ri;
    }
    rz = block_sum(rz, sh);
    rr = block_sum(rr, sh);
    if (threadIdx.x == 0) {
      S->part[(int64_t)tl.tile * 3 + 1] = rz;
      S->part[(int64_t)tl.tile * 3 + 2] = rr;
    }
    if (last_tile(&S->cnt, S->ntiles, &sh_last) && threadIdx.x < 32) {
      const double srz = ordered_tiles_sum(S->part, 1, S->ntiles);
      const double srr = ordered_tiles_sum(S->part, 2, S->ntiles);
      if (threadIdx.x == 0) {
        S->beta = srz / S->rz;
        S->rz = srz;
        S->rnorm2 = srr;
        S->iters += 1;
        S->cur ^= 1;
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
  dev_free(e->ctx, S.p[0]);
  dev_free(e->ctx, S.p[1]);
  dev_free(e->ctx, S.part);
  memset(&S, 0, sizeof S);
}
}  // namespace

bool cg_valid(const fe_cg *h) { return h && h->magic == kMagicCg && h->e; }
int64_t cg_launches(const fe_cg *h) { return h->e->launches; }
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
  e->grid = 152 * 4;
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
                 const double *b, double *x, double rtol, int maxit, int *slot) {
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
  const int64_t ntiles = nrows > 0 ? (nrows + kCgTileRows - 1) / kCgTileRows : 0;
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
  S.ntiles = (int)ntiles;
  S.rtol = rtol;
  S.maxit = maxit;
  const size_t vb = sizeof(double) * (nrows > 0 ? nrows : 1);
  S.r = (double *)dev_alloc(e->ctx, vb);
  S.z = (double *)dev_alloc(e->ctx, vb);
  S.q = (double *)dev_alloc(e->ctx, vb);
  S.dinv = (double *)dev_alloc(e->ctx, vb);
  S.p[0] = (double *)dev_alloc(e->ctx, vb);
  S.p[1] = (double *)dev_alloc(e->ctx, vb);
  S.part = (double *)dev_alloc(e->ctx, sizeof(double) * 3 * (ntiles > 0 ? ntiles : 1));
  if (!S.r || !S.z || !S.q || !S.dinv || !S.p[0] || !S.p[1] || !S.part) {
    free_sys_vectors(e, S);
    snprintf(g_smsg, sizeof g_smsg, "fe_cg_add: device allocation failed");
    return FE_ENOMEM;
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
