// Batched assembly of many independent meshes in one persistent launch.
//
// The paper attributes the flattening of strong scaling to a fixed cost per field and par_loop of
// a few hundred microseconds (Sec. 6.4.2); on a GPU the analogue is the launch and tail cost of
// one kernel per mesh.  A batch concatenates the Mats and right-hand sides of all its problems in
// two contiguous buffers and assembles them with two launches (zero, then one persistent kernel
// whose CTAs take (problem, cell range) tiles from a device work counter and dispatch on the
// element type), optionally captured once into a CUDA graph and replayed.  Tile size and grid
// size are chosen by a small autotuner that times the candidates on the batch itself.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "fe_kernels.cuh"

namespace fe {
namespace {
using namespace kern;

// element/form variants compiled into the persistent kernel (FP64 and double-float, push)
enum BatchType : int {
  BT_P1_HELM = 0, BT_P2_HELM, BT_P1_MASS, BT_P2_MASS, BT_P1_LAP, BT_P2_LAP, BT_NTYPES
};

struct BatchItem {
  AsmArgs mat;  // vals -> this problem's slice of the batch values
  AsmArgs vec;  // y -> this problem's slice of the batch right-hand sides
  int type;
  int has_vec;
  int dd;       // element tensors in double-float
};

struct Tile {
  int item;
  int pad;
  int64_t begin, end;
};

template <int P, int FORM, class Ops>
__device__ __forceinline__ void batch_cell(const BatchItem &it, int64_t e) {
  mat_push_cell<2, P, FORM, Ops>(it.mat, e);
  if (it.has_vec) vec_push_cell<2, P, P, Ops>(it.vec, e);
}

template <class Ops>
__device__ __forceinline__ void batch_dispatch(const BatchItem &it, int64_t e) {
  switch (it.type) {
    case BT_P1_HELM: batch_cell<1, FE_FORM_HELMHOLTZ, Ops>(it, e); break;
    case BT_P2_HELM: batch_cell<2, FE_FORM_HELMHOLTZ, Ops>(it, e); break;
    case BT_P1_MASS: batch_cell<1, FE_FORM_MASS, Ops>(it, e); break;
    case BT_P2_MASS: batch_cell<2, FE_FORM_MASS, Ops>(it, e); break;
    case BT_P1_LAP: batch_cell<1, FE_FORM_LAPLACE, Ops>(it, e); break;
    case BT_P2_LAP: batch_cell<2, FE_FORM_LAPLACE, Ops>(it, e); break;
    default: break;
  }
}

// Zeroes the batch's values and right-hand sides and resets the work counter.
__global__ void k_batch_zero(double *__restrict__ vals, int64_t nv, double *__restrict__ rhs, int64_t nr,
                             int *counter) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  if (t == 0) *counter = 0;
  for (int64_t i = t; i < nv; i += st) vals[i] = 0.0;
  for (int64_t i = t; i < nr; i += st) rhs[i] = 0.0;
}

// Persistent: each CTA repeatedly takes the next tile; a tile is a cell range of one problem,
// one thread per cell.  Terminates when the tile counter passes the table (no waiting).
__global__ void __launch_bounds__(kPushThreads) k_batch_assemble(const BatchItem *__restrict__ items,
                                                                 const Tile *__restrict__ tiles, int ntiles,
                                                                 int *counter) {
  __shared__ int t_sh;
  while (true) {
    if (threadIdx.x == 0) t_sh = atomicAdd(counter, 1);
    __syncthreads();
    const int t = t_sh;
    __syncthreads();
    if (t >= ntiles) break;
    const Tile tl = tiles[t];
    const BatchItem &it = items[tl.item];
    for (int64_t e = tl.begin + threadIdx.x; e < tl.end; e += blockDim.x) {
      if (it.dd) batch_dispatch<OpsF32x2>(it, e);
      else batch_dispatch<OpsF64>(it, e);
    }
  }
}

int batch_type(const fe_form_desc &d) {
  if (d.dim != 2 || d.degree < 1 || d.degree > 2) return -1;
  const int p1 = d.degree == 1;
  switch (d.form) {
    case FE_FORM_HELMHOLTZ: return p1 ? BT_P1_HELM : BT_P2_HELM;
    case FE_FORM_MASS: return p1 ? BT_P1_MASS : BT_P2_MASS;
    case FE_FORM_LAPLACE: return p1 ? BT_P1_LAP : BT_P2_LAP;
    default: return -1;
  }
}

}  // namespace

struct BatchImpl {
  fe_ctx *ctx;
  int n;
  std::vector<BatchItem> items;
  std::vector<int64_t> val_off, rhs_off, nnz, nrows, ncell;
  int64_t total_vals, total_rhs, total_cells;
  double *vals, *rhs;
  BatchItem *d_items;
  Tile *d_tiles;
  int ntiles, tile_cap;
  int *d_counter;
  int tile_cells, grid;
  cudaGraphExec_t graph;
  int graph_tile_cells, graph_grid;
  cudaStream_t cap;  // private stream the graph is captured on (the context stream may be the legacy one)
};

}  // namespace fe

struct fe_batch {
  uint32_t magic;
  fe::BatchImpl *impl;
};

namespace fe {
namespace {
constexpr uint32_t kMagicBatch = 0xFE0BA7C4u;
thread_local char g_bmsg[512];

cudaError_t upload_tiles(BatchImpl *b, int tile_cells) {
  std::vector<Tile> t;
  for (int i = 0; i < b->n; i++)
    for (int64_t c = 0; c < b->ncell[i]; c += tile_cells) t.push_back({i, 0, c, c + tile_cells < b->ncell[i] ? c + tile_cells : b->ncell[i]});
  if ((int)t.size() > b->tile_cap) return cudaErrorInvalidValue;
  b->ntiles = (int)t.size();
  b->tile_cells = tile_cells;
  if (t.empty()) return cudaSuccess;
  return cudaMemcpyAsync(b->d_tiles, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice, b->ctx->stream);
}

cudaError_t launch_step(BatchImpl *b, cudaStream_t s) {
  k_batch_zero<<<152 * 8, 256, 0, s>>>(b->vals, b->total_vals, b->rhs, b->total_rhs, b->d_counter);
  if (b->ntiles > 0) k_batch_assemble<<<b->grid, kPushThreads, 0, s>>>(b->d_items, b->d_tiles, b->ntiles, b->d_counter);
  return cudaGetLastError();
}
}  // namespace

const char *batch_message() { return g_bmsg; }

// Host side of the C ABI (fe_api.cpp forwards).
static void free_impl(BatchImpl *b, void (*release)(fe_ctx *, void *)) {
  release(b->ctx, b->vals);
  release(b->ctx, b->rhs);
  release(b->ctx, b->d_items);
  release(b->ctx, b->d_tiles);
  release(b->ctx, b->d_counter);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

fe_status batch_create(fe_ctx *c, int n, const fe_batch_item *items, void *(*alloc)(fe_ctx *, size_t),
                       void (*release)(fe_ctx *, void *), fe_batch **out) {
  g_bmsg[0] = 0;
  BatchImpl *b = new (std::nothrow) BatchImpl();
  if (!b) return FE_ENOMEM;
  b->vals = b->rhs = nullptr;
  b->d_items = nullptr;
  b->d_tiles = nullptr;
  b->d_counter = nullptr;
  b->graph = nullptr;
  b->cap = nullptr;
  b->ctx = c;
  b->n = n;
  b->total_vals = b->total_rhs = b->total_cells = 0;
  for (int i = 0; i < n; i++) {
    const fe_batch_item &it = items[i];
    fe_kernel *k = it.kmat;
    const int type = batch_type(k->d);
    if (type < 0 || k->d.precision == FE_PREC_FP32) {
      snprintf(g_bmsg, sizeof g_bmsg, "fe_batch_create: item %d: only Mass/Laplace/Helmholtz on P1/P2 triangles, FP64 or "
               "double-float, are batched", i);
      delete b;
      return FE_EUNSUPPORTED;
    }
    fe_sparsity *sp = it.sp;
    if (sp->rmap != sp->cmap || sp->rmap->arity != k->nd || it.cells != sp->rmap->from || it.coord_map->from != it.cells ||
        it.coord_map->arity != 3 || it.coords->dim != 2 || it.coords->set != it.coord_map->to) {
      snprintf(g_bmsg, sizeof g_bmsg, "fe_batch_create: item %d: inconsistent sets, maps or sparsity", i);
      delete b;
      return FE_EINVAL;
    }
    BatchItem bi;
    memset(&bi, 0, sizeof bi);
    bi.type = type;
    bi.dd = k->d.precision == FE_PREC_F32X2;
    AsmArgs &a = bi.mat;
    a.ncell = it.cells->size;
    a.map = sp->rmap->values;
    a.coords = it.coords->data;
    a.cmapv = it.coord_map->values;
    a.nvert = it.coords->set->size;
    a.nrows = sp->nrows;
    a.rowptr = sp->rowptr;
    a.lut = sp->lut;
    a.err = c->d_err;
    a.checks = c->checks;
    bi.vec = a;
    if (it.kvec) {
      fe_kernel *kv = it.kvec;
      if (kv->d.form != FE_FORM_SOURCE || kv->d.coeff_degree != kv->d.degree || kv->d.degree != k->d.degree ||
          !it.f.dat || !it.f.map || it.f.map->arity != k->nd || it.f.map->from != it.cells) {
        snprintf(g_bmsg, sizeof g_bmsg, "fe_batch_create: item %d: the linear form must be f v dx with f in the same space", i);
        delete b;
        return FE_EUNSUPPORTED;
      }
      bi.has_vec = 1;
      bi.vec.coef = it.f.dat->data;
      bi.vec.coefmap = it.f.map->values;
      bi.vec.ncoef = it.f.dat->set->size;
    }
    b->items.push_back(bi);
    b->val_off.push_back(b->total_vals);
    b->rhs_off.push_back(b->total_rhs);
    b->nnz.push_back(sp->nnz);
    b->nrows.push_back(sp->nrows);
    b->ncell.push_back(it.cells->size);
    b->total_vals += sp->nnz;
    b->total_rhs += sp->nrows;
    b->total_cells += it.cells->size;
  }
  b->vals = (double *)alloc(c, sizeof(double) * (b->total_vals > 0 ? b->total_vals : 1));
  b->rhs = (double *)alloc(c, sizeof(double) * (b->total_rhs > 0 ? b->total_rhs : 1));
  b->d_items = (BatchItem *)alloc(c, sizeof(BatchItem) * (n > 0 ? n : 1));
  // tile table capacity for the smallest tile size the tuner tries (256 cells)
  int64_t cap = 0;
  for (int i = 0; i < n; i++) cap += (b->ncell[i] + 255) / 256;
  b->tile_cap = (int)(cap > 0 ? cap : 1);
  b->d_tiles = (Tile *)alloc(c, sizeof(Tile) * b->tile_cap);
  b->d_counter = (int *)alloc(c, 256);
  if (!b->vals || !b->rhs || !b->d_items || !b->d_tiles || !b->d_counter) {
    snprintf(g_bmsg, sizeof g_bmsg, "fe_batch_create: device allocation failed");
    free_impl(b, release);
    return FE_ENOMEM;
  }
  for (int i = 0; i < n; i++) {
    b->items[i].mat.vals = b->vals + b->val_off[i];
    b->items[i].vec.y = b->rhs + b->rhs_off[i];
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess && n > 0)
    e = cudaMemcpyAsync(b->d_items, b->items.data(), sizeof(BatchItem) * n, cudaMemcpyHostToDevice, c->stream);
  b->grid = 152 * 8;
  if (e == cudaSuccess) e = upload_tiles(b, 1024);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  b->graph = nullptr;
  if (e != cudaSuccess) {
    snprintf(g_bmsg, sizeof g_bmsg, "fe_batch_create: %s", cudaGetErrorString(e));
    free_impl(b, release);
    return FE_ECUDA;
  }
  fe_batch *h = new (std::nothrow) fe_batch{kMagicBatch, b};
  if (!h) {
    free_impl(b, release);
    return FE_ENOMEM;
  }
  *out = h;
  return FE_OK;
}

bool batch_valid(const fe_batch *h) { return h && h->magic == kMagicBatch && h->impl; }

fe_ctx *batch_ctx(const fe_batch *h) { return h->impl->ctx; }

fe_status batch_views(const fe_batch *h, int i, double **vals, int64_t *nnz, double **rhs, int64_t *nrows) {
  BatchImpl *b = h->impl;
  if (i < 0 || i >= b->n) return FE_EINVAL;
  if (vals) *vals = b->vals + b->val_off[i];
  if (nnz) *nnz = b->nnz[i];
  if (rhs) *rhs = b->rhs + b->rhs_off[i];
  if (nrows) *nrows = b->nrows[i];
  return FE_OK;
}

fe_status batch_assemble(fe_batch *h, int use_graph) {
  BatchImpl *b = h->impl;
  cudaStream_t s = b->ctx->stream;
  cudaError_t e;
  if (!use_graph) {
    e = launch_step(b, s);
  } else {
    if (b->graph && (b->graph_tile_cells != b->tile_cells || b->graph_grid != b->grid)) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    if (!b->graph) {
      // captured once on the private stream; the replays go to the context stream
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t el = launch_step(b, b->cap);
        e = cudaStreamEndCapture(b->cap, &g);
        if (e == cudaSuccess) e = el;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        snprintf(g_bmsg, sizeof g_bmsg, "fe_batch_assemble: graph capture: %s", cudaGetErrorString(e));
        return FE_ECUDA;
      }
      b->graph_tile_cells = b->tile_cells;
      b->graph_grid = b->grid;
    }
    e = cudaGraphLaunch(b->graph, s);
  }
  if (e != cudaSuccess) {
    snprintf(g_bmsg, sizeof g_bmsg, "fe_batch_assemble: %s", cudaGetErrorString(e));
    return FE_ECUDA;
  }
  return FE_OK;
}

// Autotuner: times every (tile cells, CTAs per SM) candidate `reps` times on the batch itself
// (CUDA events on the context stream, after one warm-up) and keeps the fastest.
fe_status batch_tune(fe_batch *h, int reps, int *best_tile, int *best_grid, float *best_ms) {
  BatchImpl *b = h->impl;
  cudaStream_t s = b->ctx->stream;
  const int tiles[] = {256, 1024, 4096, 16384};
  const int ctas[] = {4, 8, 16};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return FE_ECUDA;
  float best = 1e30f;
  int bt = b->tile_cells, bg = b->grid;
  cudaError_t e = cudaSuccess;
  for (int tc : tiles)
    for (int cs : ctas) {
      e = upload_tiles(b, tc);
      if (e != cudaSuccess) break;
      b->grid = 152 * cs;
      e = launch_step(b, s);
      if (e != cudaSuccess) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < (reps > 0 ? reps : 1); r++) launch_step(b, s);
      cudaEventRecord(e1, s);
      e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) break;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= (reps > 0 ? reps : 1);
      if (ms < best) {
        best = ms;
        bt = tc;
        bg = b->grid;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    snprintf(g_bmsg, sizeof g_bmsg, "fe_batch_tune: %s", cudaGetErrorString(e));
    return FE_ECUDA;
  }
  e = upload_tiles(b, bt);
  b->grid = bg;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return FE_ECUDA;
  if (best_tile) *best_tile = bt;
  if (best_grid) *best_grid = bg;
  if (best_ms) *best_ms = best;
  return FE_OK;
}

void batch_destroy(fe_batch *h, void (*release)(fe_ctx *, void *)) {
  BatchImpl *b = h->impl;
  cudaStreamSynchronize(b->ctx->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  free_impl(b, release);
  h->magic = 0xDEADu;
  h->impl = nullptr;
  delete h;
}

}  // namespace fe
