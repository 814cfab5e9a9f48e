// Request loop for assemble-and-solve requests: admission by device-memory budget, continuous
// batching of the Jacobi-CG iterations of every admitted system, retirement as each converges.
//
// Each request is a Poisson problem on its own mesh (the Poisson listing of Sec. 3.1 and the
// experiment of Sec. 6.2): a = inner(grad u, grad v) dx and L = f v dx assembled with the
// deterministic row-owner (pull) strategy, u = 0 on the flagged boundary nodes by symmetric
// elimination, then CG with M = diag(A).  Every step runs in this library's kernels; the loop
// itself is host code that decides what to launch.
//
// Loop, until every submitted request has finished or been refused:
//   1. if systems are iterating: launch one tick of `iters_per_tick` CG iterations for all of
//      them (a captured graph), without waiting for it.  Systems too large for one wave of
//      512-row tiles iterate in a second engine on a high-priority stream whose launches use
//      15/16 of the resident blocks: their blocks take the SMs first, and the smaller systems'
//      blocks run in the sixteenth kept free (sharing one launch instead, the small tiles would
//      add a second round on some blocks and slow the large system down; with all blocks taken
//      at high priority, the small systems would only run in the gaps between its launches);
//   2. meanwhile admit, in arrival order, requests that have arrived while a slot is free and the
//      request's worst-case device footprint fits in the budget beside what is held (a request
//      larger than the whole budget is refused; a request that does not fit yet waits, and so do
//      the ones behind it).  The requests admitted together form a round, built in three stages
//      with one host wait between stages whatever their number (admit_round), and assembled in
//      two launches for all of them (fe_serve_asm.cu).  Admission runs on a second stream, so the
//      systems already iterating are not paused by it; the server's stream waits for it before
//      the next tick;
//   3. poll the tick: converged systems copy their solution to the host and free everything they
//      held.  With nothing iterating and nothing admitted, sleep until the next arrival.
// Memory is accounted exactly: the server routes its allocations through a counting allocator that
// draws from its own stream-ordered CUDA memory pool (requests come and go too often for a
// synchronous allocator).
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fe_internal.h"

namespace fe {
namespace {

// Device objects of one mesh: the inputs that define it (cell-node and cell-vertex maps,
// coordinates, boundary flags) and its sparsity (pattern, lookup table, incidence).  Requests that
// carry the same non-zero mesh_key share one (the cache, kept across requests until evicted under
// the budget); a request without a key has a private one.
struct MeshEntry {
  uint64_t key = 0;
  fe_set *cells = nullptr, *nodes = nullptr, *verts = nullptr;
  fe_map *M = nullptr, *CM = nullptr;
  fe_dat *XY = nullptr;
  fe_sparsity *sp = nullptr;
  void *d_map = nullptr, *d_cv = nullptr, *d_xy = nullptr, *d_bc = nullptr;
  int refs = 0;           // admitted requests using it
  uint64_t last_use = 0;  // admission counter at the last use (least recently used is evicted first)
  bool ready = false;     // its sparsity is complete (false while the round that builds it runs)
};

struct Holding {  // device objects of one admitted request
  MeshEntry *mesh = nullptr;
  bool private_mesh = false;  // built for this request alone (no key): freed with it
  fe_dat *F = nullptr, *B = nullptr, *X = nullptr;
  fe_mat *A = nullptr;
  void *d_f = nullptr, *d_b = nullptr, *d_x = nullptr;
  int slot = -1;
  bool big = false;    // iterating in the large-system engine (high-priority stream)
  bool build = false;  // builds its mesh in its admission round
  void *mstage = nullptr, *vstage = nullptr;  // element tensors of the round's assembly (transient)
};

struct Req {
  fe_solve_request in;
  fe_solve_result res;
  size_t estimate;       // worst-case footprint, mesh included
  size_t mesh_estimate;  // its mesh part (maps, coordinates, flags, sparsity)
  Holding h;
};

thread_local char g_vmsg[512];

}  // namespace

struct Server {
  fe_ctx *parent;
  fe_ctx *ctx;  // same device and stream as the parent, counting allocator
  cudaStream_t main_stream = nullptr;  // the parent's stream: CG ticks, polls, retirement
  cudaStream_t adm = nullptr;          // admission (copies, sparsity, assembly, elimination, CG set-up)
  cudaEvent_t adm_done = nullptr;      // end of the last admissions, waited for by main_stream and hi
  cudaStream_t hi = nullptr;           // high priority: CG of the systems of more than one wave
  fe_cg *cgb = nullptr;                // engine of those systems
  cudaMemPool_t pool = nullptr;  // the server's own stream-ordered pool (requests come and go often)
  fe_server_config cfg;
  fe_kernel *klap[3] = {nullptr, nullptr, nullptr}, *ksrc[3] = {nullptr, nullptr, nullptr};
  fe_cg *cg = nullptr;
  std::vector<Req> reqs;
  std::vector<MeshEntry *> meshes;  // the cache: entries with a key (private ones are not listed)
  uint64_t admissions = 0;
  // pinned host slots for the staged sparsity builds of one admission round (one per request)
  int *h_maxcnt = nullptr, *h_maxrow = nullptr;
  int64_t *h_nnz = nullptr;
  // the table of the round's batched assembly: pinned host copy, device copy, and the event after
  // which the host copy may be rewritten
  ServeItem *h_items = nullptr, *d_items = nullptr;
  cudaEvent_t items_read = nullptr;
  int cache_hits = 0, cache_misses = 0, cache_evictions = 0, sparsity_builds = 0;
  // accounting
  // pointer -> (bytes, owner; kOwnerServer = server tables, kOwnerCache = cached meshes, else request)
  std::unordered_map<void *, std::pair<size_t, int64_t>> live;
  std::vector<size_t> owner_bytes;
  int64_t owner = -1;
  size_t base_bytes = 0, cache_bytes = 0, live_bytes = 0, peak_bytes = 0, reserved = 0;
  int estimate_misses = 0;
  double run_s = 0.0, admit_s = 0.0, tick_s = 0.0, retire_s = 0.0;
};

// The server context's stream for the duration of a scope: the engines and the library calls it
// makes run on the context's stream, which the loop points at the admission, main or high-priority
// stream; restored on every exit from the scope.
struct OnStream {
  fe_ctx *c;
  cudaStream_t prev;
  OnStream(Server *s, cudaStream_t st) : c(s->ctx), prev(s->ctx ? s->ctx->stream : nullptr) {
    if (c) c->stream = st;
  }
  ~OnStream() {
    if (c) c->stream = prev;
  }
  OnStream(const OnStream &) = delete;
  OnStream &operator=(const OnStream &) = delete;
};

}  // namespace fe

struct fe_server {
  uint32_t magic;
  fe::Server *s;
};

namespace fe {
namespace {
constexpr uint32_t kMagicServer = 0xFE05E2E5u;
constexpr int64_t kOwnerServer = -1, kOwnerCache = -2;

void *count_alloc(size_t bytes, void *user) {
  Server *s = static_cast<Server *>(user);
  void *ptr = nullptr;
  if (cudaMallocFromPoolAsync(&ptr, bytes, s->pool, s->ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
  }
  if (!ptr) return nullptr;
  s->live[ptr] = {bytes, s->owner};
  s->live_bytes += bytes;
  s->peak_bytes = std::max(s->peak_bytes, s->live_bytes);
  if (s->owner >= 0) s->owner_bytes[s->owner] += bytes;
  else if (s->owner == kOwnerCache) s->cache_bytes += bytes;
  else s->base_bytes += bytes;
  return ptr;
}

void count_free(void *ptr, void *user) {
  Server *s = static_cast<Server *>(user);
  auto it = s->live.find(ptr);
  if (it != s->live.end()) {
    const size_t b = it->second.first;
    const int64_t o = it->second.second;
    s->live_bytes -= b;
    if (o >= 0) s->owner_bytes[o] -= b;
    else if (o == kOwnerCache) s->cache_bytes -= b;
    else s->base_bytes -= b;
    s->live.erase(it);
  }
  cudaFreeAsync(ptr, s->ctx->stream);
}

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

int nodes_p(int p) { return (p + 1) * (p + 2) / 2; }

// Worst-case device bytes of one request (every allocation it makes, at its largest, while it
// is built; nnz bounded by the cell-node incidences times the arity, a row's length by the
// node's most frequent incidence times the arity).
size_t estimate_bytes(const fe_solve_request &r, size_t *mesh_part = nullptr) {
  const size_t nd = nodes_p(r.degree), ncell = r.ncell, nn = r.nnodes, nv = r.nvert;
  const size_t ninc = ncell * nd, nnz = ninc * nd;
  std::vector<int32_t> inc(nn, 0);
  int32_t maxinc = 0;
  for (size_t k = 0; k < ninc; k++) {
    const int32_t v = r.cell_node[k];
    if (v >= 0 && (size_t)v < nn) maxinc = std::max(maxinc, ++inc[v]);
  }
  const size_t nsl = (nn + 31) / 32, maxlen = std::min(nn, (size_t)maxinc * nd);
  const size_t sell = std::min(32 * nsl * maxlen, 32 * nsl * nn);
  auto a = [](size_t b) { return (std::max<size_t>(b, 16) + 255) & ~size_t(255); };
  size_t m = 0, t = 0;
  m += a(4 * ninc) + a(12 * ncell) + a(16 * nv) + a(nn);                                        // mesh inputs
  m += 2 * a(8 * (nn + 1)) + a(4 * ninc) + a(4 * nn) + a(4 * ninc * nd) + a(ninc * nd) +
       a(8 * scan_tmp_elems((int64_t)nn)) + a(4) + a(4 * nnz);                                  // sparsity
  if (mesh_part) *mesh_part = m;
  t += m + a(8 * nn) + a(8 * nn) + a(8 * nn);                                                   // f, b, x
  t += a(8 * nnz) + a(8 * ncell * nd * nd) + a(8 * ncell * nd);                                 // Mat, staging
  t += 5 * a(8 * nn) + a(24 * (nn / 512 + 1));  // CG vectors, tile partials (tiles of at least 512 rows)
  t += a(8 * (nsl + 1)) + a(4 * nsl) + a(8 * scan_tmp_elems((int64_t)nsl)) + a(8 * sell) + a(4 * sell);  // SELL
  return t;
}

#define SV_TRY(expr)                                   \
  do {                                                 \
    fe_status _st = (expr);                            \
    if (_st != FE_OK) return _st;                      \
  } while (0)

fe_status copy_in(Server *s, void **dst, const void *src, size_t bytes) {
  *dst = dev_alloc(s->ctx, bytes);
  if (!*dst) return FE_ENOMEM;
  if (bytes == 0) return FE_OK;
  return cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s->ctx->stream) == cudaSuccess ? FE_OK : FE_ECUDA;
}

// Frees a mesh entry's device objects (the caller has synchronised the streams that used them).
void mesh_free(Server *s, MeshEntry *m) {
  if (!m) return;
  if (m->sp) fe_sparsity_destroy(m->sp);
  if (m->XY) fe_dat_destroy(m->XY);
  for (fe_map *x : {m->M, m->CM})
    if (x) fe_map_destroy(x);
  for (fe_set *t : {m->cells, m->nodes, m->verts})
    if (t) fe_set_destroy(t);
  for (void *p : {m->d_map, m->d_cv, m->d_xy, m->d_bc}) dev_free(s->ctx, p);
  delete m;
}

void release(Server *s, Req &q) {
  Holding &h = q.h;
  const int64_t saved = s->owner;
  s->owner = &q - s->reqs.data();
  if (h.slot >= 0) fe_cg_remove(h.big ? s->cgb : s->cg, h.slot);
  cudaStreamSynchronize(s->ctx->stream);
  if (h.A) fe_mat_destroy(h.A);
  for (fe_dat *d : {h.F, h.B, h.X})
    if (d) fe_dat_destroy(d);
  for (void *p : {h.d_f, h.d_b, h.d_x, h.mstage, h.vstage}) dev_free(s->ctx, p);
  if (h.mesh) {
    if (h.private_mesh) mesh_free(s, h.mesh);
    else h.mesh->refs--;  // a cached mesh stays until evicted
  }
  h = Holding();
  s->owner = saved;
}

// Evicts unused cached meshes, least recently used first, until `need` more bytes fit in the
// budget beside what is held; returns whether they fit.  Nothing waits: an entry without
// references has no work in flight.  Its last users have retired, each after a wait on the stream
// it iterated on, whose ticks had waited for their admission; its frees are stream-ordered on the
// admission stream (the context's stream while the loop admits).
bool make_room(Server *s, size_t held, size_t need) {
  auto fits = [&]() { return s->base_bytes + s->cache_bytes + held + need <= s->cfg.hbm_budget; };
  while (!fits()) {
    MeshEntry *victim = nullptr;
    for (MeshEntry *m : s->meshes)
      if (m->refs == 0 && (!victim || m->last_use < victim->last_use)) victim = m;
    if (!victim) return false;
    s->meshes.erase(std::find(s->meshes.begin(), s->meshes.end(), victim));
    const int64_t saved = s->owner;
    s->owner = kOwnerCache;
    mesh_free(s, victim);
    s->owner = saved;
    s->cache_evictions++;
  }
  return true;
}

MeshEntry *find_mesh(Server *s, const fe_solve_request &r) {
  if (r.mesh_key == 0) return nullptr;
  for (MeshEntry *m : s->meshes)
    if (m->key == r.mesh_key) return m;
  return nullptr;
}

// Starts a mesh entry on the device: copies of the maps, coordinates and boundary flags, its sets,
// maps and coordinate Dat, and the first stage of its sparsity build (the longest incidence list
// read back into the server's pinned slot k); admit_round finishes it.
fe_status mesh_begin(Server *s, const fe_solve_request &r, MeshEntry *m, int k) {
  fe_ctx *c = s->ctx;
  const int nd = nodes_p(r.degree);
  SV_TRY(copy_in(s, &m->d_map, r.cell_node, sizeof(int32_t) * r.ncell * nd));
  SV_TRY(copy_in(s, &m->d_cv, r.cell_vertex, sizeof(int32_t) * r.ncell * 3));
  SV_TRY(copy_in(s, &m->d_xy, r.coords, sizeof(double) * r.nvert * 2));
  SV_TRY(copy_in(s, &m->d_bc, r.is_bc, r.nnodes));
  SV_TRY(fe_set_create(c, r.ncell, &m->cells));
  SV_TRY(fe_set_create(c, r.nnodes, &m->nodes));
  SV_TRY(fe_set_create(c, r.nvert, &m->verts));
  // the range checks are launched without waiting: the flags are read once per stage of the round,
  // before any kernel indexes through the maps (the sparsity build checks the cell-node map)
  SV_TRY(fe_map_create(c, m->cells, m->nodes, nd, (const int32_t *)m->d_map, 0, &m->M));
  SV_TRY(fe_map_create(c, m->cells, m->verts, 3, (const int32_t *)m->d_cv, 0, &m->CM));
  if (r.ncell > 0 && launch_map_validate((const int32_t *)m->d_cv, r.ncell * 3, r.nvert, c->d_err, c->stream) != cudaSuccess)
    return FE_ECUDA;
  SV_TRY(fe_dat_create(c, m->verts, 2, (double *)m->d_xy, &m->XY));
  SV_TRY(sparsity_build_begin(c, m->M, m->M, &m->sp, &s->h_maxcnt[k]));
  return FE_OK;
}

// The request at fault when a stage's range check failed (the device flags are the context's, so
// they do not say whose map it was): the first new mesh of the round with a map value outside
// its target set, read from the request's host arrays.
int64_t culprit(const Server *s, const std::vector<int64_t> &ids) {
  for (int64_t id : ids) {
    const fe_solve_request &r = s->reqs[id].in;
    if (!s->reqs[id].h.build) continue;
    const int64_t nc = r.ncell * nodes_p(r.degree), nv = r.ncell * 3;
    for (int64_t k = 0; k < nc; k++)
      if (r.cell_node[k] < 0 || r.cell_node[k] >= r.nnodes) return id;
    for (int64_t k = 0; k < nv; k++)
      if (r.cell_vertex[k] < 0 || r.cell_vertex[k] >= r.nvert) return id;
  }
  return ids[0];
}

// Builds the systems of one admission round on the device and hands them to the CG engines.  The
// loop has planned the round: each request fits in the budget, its mesh entry is referenced (a
// cached one, or a new one that the request builds: h.build), so that no later request of the
// round evicts it.  Stages, each only launching work on the admission stream:
//   1. the new meshes' copies and range checks and the first stage of their sparsity builds (the
//      longest incidence list read back into a pinned slot); every request's vectors;
//   2. after one wait for all of them, the row pass of every new pattern (nnz and the longest
//      row read back);
//   3. after a second wait, the column compaction, every request's Mat and staging, then ONE
//      element-tensor launch and ONE row launch for the whole round (Laplace Mat with the
//      boundary rows and columns eliminated, source right-hand side), then each system's CG
//      set-up.
// A round without new meshes does not wait at all.  On failure *failed is the request at fault.
fe_status admit_round(Server *s, const std::vector<int64_t> &ids, int64_t *failed) {
  fe_ctx *c = s->ctx;
  cudaStream_t st = c->stream;
  const int n = (int)ids.size();
  std::vector<int> slot(n, -1);  // pinned slot of each mesh built in the round
  auto mesh_owner = [&](int k) { return s->reqs[ids[k]].h.private_mesh ? ids[k] : kOwnerCache; };
  int nb = 0;
  for (int k = 0; k < n; k++) {  // stage 1
    Req &q = s->reqs[ids[k]];
    const fe_solve_request &r = q.in;
    Holding &h = q.h;
    *failed = ids[k];
    if (h.build) {
      slot[k] = nb++;
      s->owner = mesh_owner(k);
      const fe_status bs = mesh_begin(s, r, h.mesh, slot[k]);
      s->owner = ids[k];
      if (bs != FE_OK) return bs;
    }
    s->owner = ids[k];
    MeshEntry *m = h.mesh;
    SV_TRY(copy_in(s, &h.d_f, r.f, sizeof(double) * r.nnodes));
    h.d_b = dev_alloc(c, sizeof(double) * (r.nnodes > 0 ? r.nnodes : 1));
    h.d_x = dev_alloc(c, sizeof(double) * (r.nnodes > 0 ? r.nnodes : 1));
    if (!h.d_b || !h.d_x) return FE_ENOMEM;
    if (cudaMemsetAsync(h.d_x, 0, sizeof(double) * r.nnodes, st) != cudaSuccess) return FE_ECUDA;
    SV_TRY(fe_dat_create(c, m->nodes, 1, (double *)h.d_f, &h.F));
    SV_TRY(fe_dat_create(c, m->nodes, 1, (double *)h.d_b, &h.B));
    SV_TRY(fe_dat_create(c, m->nodes, 1, (double *)h.d_x, &h.X));
  }
  if (nb > 0) {
    fe_status fs = sparsity_check_flags(c, "fe_server_run");  // the one wait of stage 1
    if (fs != FE_OK) {
      *failed = culprit(s, ids);
      return fs;
    }
    for (int k = 0; k < n; k++) {                        // stage 2
      if (slot[k] < 0) continue;
      *failed = ids[k];
      SV_TRY(sparsity_build_rows(s->reqs[ids[k]].h.mesh->sp, s->h_maxcnt[slot[k]], &s->h_nnz[slot[k]],
                                 &s->h_maxrow[slot[k]]));
    }
    fs = sparsity_check_flags(c, "fe_server_run");  // the one wait of stage 2
    if (fs != FE_OK) {
      *failed = culprit(s, ids);
      return fs;
    }
    for (int k = 0; k < n; k++) {
      if (slot[k] < 0) continue;
      MeshEntry *m = s->reqs[ids[k]].h.mesh;
      *failed = ids[k];
      s->owner = mesh_owner(k);
      fs = sparsity_build_finish(m->sp, s->h_nnz[slot[k]], s->h_maxrow[slot[k]]);
      s->owner = ids[k];
      if (fs != FE_OK) return fs;
      m->ready = true;
      s->sparsity_builds++;
    }
  }
  // stage 3: the round's table (the host copy is rewritten once the previous round's copy has
  // been read), the Mats and the transient element staging
  if (cudaEventSynchronize(s->items_read) != cudaSuccess) return FE_ECUDA;
  int64_t cell_tiles = 0, row_tiles = 0;
  size_t row_smem = 0;
  for (int k = 0; k < n; k++) {
    Req &q = s->reqs[ids[k]];
    const fe_solve_request &r = q.in;
    Holding &h = q.h;
    MeshEntry *m = h.mesh;
    *failed = ids[k];
    s->owner = ids[k];
    if (sparsity_canonical(m->sp, st) != cudaSuccess) return FE_ECUDA;  // the row owners sum in incidence order
    SV_TRY(fe_mat_create(c, m->sp, &h.A));
    const fe_form_desc d{FE_FORM_LAPLACE, 2, r.degree, 0, s->cfg.precision, FE_STRATEGY_PULL};
    const int nd = nodes_p(r.degree);
    h.mstage = dev_alloc(c, std::max<size_t>(stage_bytes_mat(d, r.ncell), 16));
    h.vstage = dev_alloc(c, std::max<size_t>(stage_bytes_vec(d, r.ncell, nd), 16));
    if (!h.mstage || !h.vstage) return FE_ENOMEM;
    const size_t smem = serve_row_smem(r.degree, m->sp->maxrow, s->cfg.precision);
    if (smem > 227 * 1024) {
      snprintf(g_vmsg, sizeof g_vmsg, "a row of %d entries is too long for the batched assembly", m->sp->maxrow);
      return FE_EUNSUPPORTED;
    }
    row_smem = std::max(row_smem, smem);
    ServeItem &it = s->h_items[k];
    memset(&it, 0, sizeof it);
    AsmArgs &a = it.mat;
    a.ncell = r.ncell;
    a.map = (const int32_t *)m->d_map;
    a.coords = (const double *)m->d_xy;
    a.cmapv = (const int32_t *)m->d_cv;
    a.nvert = r.nvert;
    a.nrows = r.nnodes;
    a.rowptr = m->sp->rowptr;
    a.lut = m->sp->lut;
    a.vals = h.A->values;
    a.adjptr = m->sp->adjptr;
    a.adj = m->sp->adj;
    a.err = c->d_err;
    a.checks = c->checks;
    a.rowcap = m->sp->maxrow;
    a.zero_first = 1;
    it.vec = a;
    it.vec.rowptr = nullptr;
    it.vec.lut = nullptr;
    it.vec.vals = nullptr;
    it.vec.coef = (const double *)h.d_f;  // f in the same space: its map is the cell-node map
    it.vec.coefmap = (const int32_t *)m->d_map;
    it.vec.ncoef = r.nnodes;
    it.vec.y = (double *)h.d_b;
    it.mstage = h.mstage;
    it.vstage = h.vstage;
    it.colidx = m->sp->colidx;
    it.is_bc = (const uint8_t *)m->d_bc;
    it.p = r.degree;
    it.cell_tile0 = cell_tiles;
    it.row_tile0 = row_tiles;
    cell_tiles += (r.ncell + kServeCellTile - 1) / kServeCellTile;
    row_tiles += (r.nnodes + kServeRowTile - 1) / kServeRowTile;
  }
  *failed = ids[0];
  if (cudaMemcpyAsync(s->d_items, s->h_items, sizeof(ServeItem) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaEventRecord(s->items_read, st) != cudaSuccess ||
      launch_serve_assembly(s->d_items, n, cell_tiles, row_tiles, row_smem, s->cfg.precision, st) != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_vmsg, sizeof g_vmsg, "launching the batched assembly of %d systems", n);
    return FE_ECUDA;
  }
  for (int k = 0; k < n; k++) {  // the staging is read by the launches above alone (frees are stream-ordered)
    Holding &h = s->reqs[ids[k]].h;
    dev_free(c, h.mstage);
    dev_free(c, h.vstage);
    h.mstage = h.vstage = nullptr;
  }
  for (int k = 0; k < n; k++) {  // CG set-up
    Req &q = s->reqs[ids[k]];
    Holding &h = q.h;
    *failed = ids[k];
    s->owner = ids[k];
    h.big = q.in.nnodes > cg_one_wave_rows(s->cg);
    SV_TRY(fe_cg_add(h.big ? s->cgb : s->cg, h.A, h.B, h.X, s->cfg.rtol, s->cfg.maxit, &h.slot));
  }
  return FE_OK;
}

// Undoes a failed round (the admission stream idle): requests that reference a mesh which the
// round did not finish drop that reference, the partly built entries leave the cache and go
// with the request that built them, then every request of the round releases what it holds.
void fail_round(Server *s, const std::vector<int64_t> &ids) {
  for (int64_t id : ids) {
    Holding &h = s->reqs[id].h;
    if (h.mesh && !h.mesh->ready && !h.build) {
      h.mesh->refs--;
      h.mesh = nullptr;
    }
  }
  for (int64_t id : ids) {
    Holding &h = s->reqs[id].h;
    if (h.build && !h.mesh->ready && !h.private_mesh) {
      s->meshes.erase(std::find(s->meshes.begin(), s->meshes.end(), h.mesh));
      h.private_mesh = true;
    }
  }
  for (int64_t id : ids) release(s, s->reqs[id]);
}

void server_free(Server *s) {
  if (!s) return;
  // nothing may be in flight on any of the server's streams while its objects are freed
  if (s->adm) cudaStreamSynchronize(s->adm);
  if (s->hi) cudaStreamSynchronize(s->hi);
  if (s->ctx) {
    if (s->main_stream) s->ctx->stream = s->main_stream;
    cudaStreamSynchronize(s->ctx->stream);
  }
  for (Req &q : s->reqs) release(s, q);
  s->owner = kOwnerCache;
  for (MeshEntry *m : s->meshes) mesh_free(s, m);
  s->meshes.clear();
  s->owner = kOwnerServer;
  if (s->cg) fe_cg_destroy(s->cg);
  if (s->cgb) {
    OnStream on(s, s->hi);
    fe_cg_destroy(s->cgb);
  }
  for (int p = 1; p <= 2; p++) {
    if (s->klap[p]) fe_kernel_destroy(s->klap[p]);
    if (s->ksrc[p]) fe_kernel_destroy(s->ksrc[p]);
  }
  if (s->hi) cudaStreamSynchronize(s->hi);
  if (s->ctx) {
    s->ctx->stream = s->main_stream ? s->main_stream : s->ctx->stream;
    if (s->d_items) dev_free(s->ctx, s->d_items);
    cudaStreamSynchronize(s->ctx->stream);
    fe_ctx_destroy(s->ctx);
  }
  for (void *p : {(void *)s->h_maxcnt, (void *)s->h_maxrow, (void *)s->h_nnz, (void *)s->h_items})
    if (p) cudaFreeHost(p);
  if (s->items_read) cudaEventDestroy(s->items_read);
  if (s->adm_done) cudaEventDestroy(s->adm_done);
  if (s->adm) cudaStreamDestroy(s->adm);
  if (s->hi) cudaStreamDestroy(s->hi);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  delete s;
}
}  // namespace

const char *server_message() { return g_vmsg; }

fe_status server_create(fe_ctx *parent, const fe_server_config *cfg, fe_server **out) {
  g_vmsg[0] = 0;
  if (cfg->max_active < 1 || cfg->iters_per_tick < 1 || !(cfg->rtol > 0.0) || cfg->maxit < 1 ||
      (cfg->precision != FE_PREC_FP64 && cfg->precision != FE_PREC_F32X2)) {
    snprintf(g_vmsg, sizeof g_vmsg, "fe_server_create: bad configuration");
    return FE_EINVAL;
  }
  Server *s = new (std::nothrow) Server();
  if (!s) return FE_ENOMEM;
  s->parent = parent;
  s->cfg = *cfg;
  // a private pool on the device: allocations are stream-ordered and cached across requests (the
  // budget is enforced by the server's own accounting, not by the pool)
  cudaMemPoolProps props;
  memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = parent->device;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_vmsg, sizeof g_vmsg, "fe_server_create: cannot create a memory pool");
    delete s;
    return FE_ECUDA;
  }
  uint64_t keep = cfg->hbm_budget;
  cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  fe_status st = fe_ctx_create(parent->device, parent->stream, &s->ctx);
  if (st == FE_OK) {
    s->main_stream = s->ctx->stream;
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (cudaStreamCreateWithFlags(&s->adm, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s->hi, cudaStreamNonBlocking, hi_prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->adm_done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      st = FE_ECUDA;
    }
  }
  if (st == FE_OK) st = fe_ctx_set_allocator(s->ctx, count_alloc, count_free, s);
  if (st == FE_OK) {  // the admission rounds' read-back slots and assembly table
    const size_t na = (size_t)cfg->max_active;
    if (cudaHostAlloc((void **)&s->h_maxcnt, sizeof(int) * na, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&s->h_maxrow, sizeof(int) * na, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&s->h_nnz, sizeof(int64_t) * na, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&s->h_items, sizeof(ServeItem) * na, cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->items_read, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      st = FE_ECUDA;
    }
    if (st == FE_OK) {
      s->d_items = (ServeItem *)dev_alloc(s->ctx, sizeof(ServeItem) * na);
      if (!s->d_items) st = FE_ENOMEM;
    }
  }
  for (int p = 1; p <= 2 && st == FE_OK; p++) {
    fe_form_desc d{FE_FORM_LAPLACE, 2, p, 0, cfg->precision, FE_STRATEGY_PULL};
    st = fe_kernel_create(s->ctx, &d, &s->klap[p]);
    fe_form_desc v{FE_FORM_SOURCE, 2, p, p, cfg->precision, FE_STRATEGY_PULL};
    if (st == FE_OK) st = fe_kernel_create(s->ctx, &v, &s->ksrc[p]);
  }
  if (st == FE_OK) st = fe_cg_create(s->ctx, cfg->max_active, &s->cg);
  if (st == FE_OK) {
    OnStream on(s, s->hi);
    st = fe_cg_create(s->ctx, cfg->max_active, &s->cgb);
  }
  if (st == FE_OK) {
    const int g = cg_grid(s->cgb);
    st = cg_limit_grid(s->cgb, g - g / 16);
  }
  if (st != FE_OK) {
    snprintf(g_vmsg, sizeof g_vmsg, "fe_server_create: %s", fe_last_error());
    server_free(s);
    return st;
  }
  fe_server *h = new (std::nothrow) fe_server{kMagicServer, s};
  if (!h) {
    server_free(s);
    return FE_ENOMEM;
  }
  *out = h;
  return FE_OK;
}

bool server_valid(const fe_server *h) { return h && h->magic == kMagicServer && h->s; }
fe_ctx *server_ctx(const fe_server *h) { return h->s->parent; }

fe_status server_submit(fe_server *h, const fe_solve_request *r, int64_t *id) {
  Server *s = h->s;
  g_vmsg[0] = 0;
  if ((r->degree != 1 && r->degree != 2) || r->ncell < 0 || r->nnodes < 0 || r->nvert < 0 ||
      (r->ncell > 0 && (!r->cell_node || !r->cell_vertex || !r->coords)) ||
      (r->nnodes > 0 && (!r->f || !r->is_bc || !r->x_out)) || !(r->arrival_s >= 0.0)) {
    snprintf(g_vmsg, sizeof g_vmsg, "fe_server_submit: bad request");
    return FE_EINVAL;
  }
  Req q;
  memset(&q.res, 0, sizeof q.res);
  q.in = *r;
  q.estimate = estimate_bytes(*r, &q.mesh_estimate);
  q.res.estimate = q.estimate;
  q.res.status = FE_SOLVE_PENDING;
  s->reqs.push_back(q);
  s->owner_bytes.push_back(0);
  if (id) *id = (int64_t)s->reqs.size() - 1;
  return FE_OK;
}

fe_status server_run(fe_server *h) {
  Server *s = h->s;
  g_vmsg[0] = 0;
  const fe_server_config &cfg = s->cfg;
  std::vector<int64_t> order;
  for (int64_t i = 0; i < (int64_t)s->reqs.size(); i++)
    if (s->reqs[i].res.status == FE_SOLVE_PENDING) order.push_back(i);
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t a, int64_t b) { return s->reqs[a].in.arrival_s < s->reqs[b].in.arrival_s; });
  size_t next = 0;
  std::vector<int64_t> active;            // request ids iterating
  // per engine (0: the systems of one wave or less, 1: the larger ones): status of every slot
  std::vector<int> st_status[2], st_iters[2];
  std::vector<double> st_r[2], st_b[2];
  for (int k = 0; k < 2; k++) {
    st_status[k].assign(cfg.max_active, 0);
    st_iters[k].assign(cfg.max_active, 0);
    st_r[k].assign(cfg.max_active, 0.0);
    st_b[k].assign(cfg.max_active, 0.0);
  }
  fe_cg *engines[2] = {s->cg, s->cgb};
  cudaStream_t streams[2] = {s->main_stream, s->hi};
  auto has = [&](int k) {
    for (int64_t id : active)
      if ((int)s->reqs[id].h.big == k) return true;
    return false;
  };
  const auto t0 = std::chrono::steady_clock::now();
  size_t held = 0;  // sum of charges of the admitted requests
  while (next < order.size() || !active.empty()) {
    // 1. one tick of CG for every admitted system, launched without waiting
    const double tt0 = now_s(t0);
    const bool ticked = !active.empty();
    const bool ran[2] = {has(0), has(1)};
    for (int k = 1; k >= 0; k--) {  // the large systems' tick first, on the high-priority stream
      if (!ran[k]) continue;
      fe_status st;
      {
        OnStream on(s, streams[k]);
        st = fe_cg_iterate(engines[k], cfg.iters_per_tick, 1);
      }
      if (st != FE_OK) {
        snprintf(g_vmsg, sizeof g_vmsg, "fe_server_run: %s", fe_last_error());
        return st;
      }
    }
    s->tick_s += now_s(t0) - tt0;
    // 2. admission, in arrival order, on the admission stream while the tick runs: plan a round
    //    of every request that has arrived and fits, then build the round together
    bool admitted = false;
    {
      OnStream on(s, s->adm);
      std::vector<int64_t> round;
      size_t pending = 0;  // planned bytes of the round (a new mesh counted in its request's)
      while (next < order.size() && (int)(active.size() + round.size()) < cfg.max_active) {
        Req &q = s->reqs[order[next]];
        if (q.in.arrival_s > now_s(t0)) break;
        MeshEntry *m = find_mesh(s, q.in);
        // a cached mesh is not charged again: the request needs only its own part
        const size_t need = m ? q.estimate - q.mesh_estimate : q.estimate;
        if (s->base_bytes + need > cfg.hbm_budget) {
          q.res.status = FE_SOLVE_REFUSED;
          q.res.admitted_s = q.res.finished_s = now_s(t0);
          next++;
          continue;
        }
        if (!make_room(s, held + pending, need)) break;  // wait for memory (unused cached meshes are evicted first)
        Holding &h = q.h;
        if (m) {
          s->cache_hits++;
        } else {
          m = new (std::nothrow) MeshEntry();
          if (!m) break;  // admitted later, if ever (the round so far goes ahead)
          m->key = q.in.mesh_key;
          h.build = true;
          if (m->key != 0) {  // cached from now on: later requests of the round with its key share it
            s->cache_misses++;
            s->meshes.push_back(m);
          } else {
            h.private_mesh = true;
          }
        }
        h.mesh = m;
        m->refs++;
        m->last_use = ++s->admissions;
        q.res.admitted_s = now_s(t0);
        pending += need;
        round.push_back(order[next]);
        next++;
      }
      if (!round.empty()) {
        const double tr0 = now_s(t0);
        int64_t failed = round[0];
        g_vmsg[0] = 0;
        const fe_status st = admit_round(s, round, &failed);
        s->owner = -1;
        s->admit_s += now_s(t0) - tr0;
        if (st != FE_OK) {
          char why[384];
          snprintf(why, sizeof why, "%s", g_vmsg[0] ? g_vmsg : fe_last_error());
          snprintf(g_vmsg, sizeof g_vmsg, "fe_server_run: request %lld: %s", (long long)failed, why);
          cudaStreamSynchronize(s->adm);  // the round's work on the admission stream has ended
          fail_round(s, round);
          return st;
        }
        for (int64_t id : round) {
          Req &q = s->reqs[id];
          if (s->owner_bytes[id] > q.estimate) s->estimate_misses++;
          q.res.bytes = s->owner_bytes[id];
          held += q.res.bytes;
          active.push_back(id);
        }
        admitted = true;
      }
    }
    if (admitted && (cudaEventRecord(s->adm_done, s->adm) != cudaSuccess ||
                     cudaStreamWaitEvent(s->main_stream, s->adm_done, 0) != cudaSuccess ||
                     cudaStreamWaitEvent(s->hi, s->adm_done, 0) != cudaSuccess)) {
      snprintf(g_vmsg, sizeof g_vmsg, "fe_server_run: ordering admission before the next tick");
      return FE_ECUDA;
    }
    if (!ticked) {
      if (!admitted && next < order.size()) {
        const double wait = s->reqs[order[next]].in.arrival_s - now_s(t0);
        if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
      }
      continue;
    }
    // 3. poll the tick, then retire the finished systems
    const double tp0 = now_s(t0);
    fe_status st = FE_OK;
    for (int k = 0; k < 2 && st == FE_OK; k++) {
      if (!ran[k] && !has(k)) continue;  // nothing of this engine iterating or just admitted
      OnStream on(s, streams[k]);
      st = fe_cg_poll(engines[k], cfg.max_active, st_status[k].data(), st_iters[k].data(), st_r[k].data(),
                      st_b[k].data());
    }
    const double tt1 = now_s(t0);
    s->tick_s += tt1 - tp0;
    if (st != FE_OK) {
      snprintf(g_vmsg, sizeof g_vmsg, "fe_server_run: %s", fe_last_error());
      return st;
    }
    for (size_t k = 0; k < active.size();) {
      const int64_t id = active[k];
      Req &q = s->reqs[id];
      const int sl = q.h.slot, e = q.h.big ? 1 : 0;
      if (st_status[e][sl] == 0) {
        k++;
        continue;
      }
      q.res.status = st_status[e][sl];
      q.res.iters = st_iters[e][sl];
      q.res.rnorm = st_r[e][sl];
      q.res.bnorm = st_b[e][sl];
      {
        // the solution and the frees are ordered on the stream the system iterated on
        OnStream on(s, streams[e]);
        cudaError_t ce = cudaSuccess;
        if (q.in.nnodes > 0)
          ce = cudaMemcpyAsync(q.in.x_out, q.h.d_x, sizeof(double) * q.in.nnodes, cudaMemcpyDeviceToHost,
                               s->ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->ctx->stream);
        if (ce != cudaSuccess) {
          snprintf(g_vmsg, sizeof g_vmsg, "fe_server_run: copying the solution of request %lld", (long long)id);
          return FE_ECUDA;
        }
        q.res.finished_s = now_s(t0);
        held -= q.res.bytes;
        release(s, q);
      }
      active.erase(active.begin() + k);
    }
    s->retire_s += now_s(t0) - tt1;
  }
  s->run_s = now_s(t0);
  return FE_OK;
}

fe_status server_result(const fe_server *h, int64_t id, fe_solve_result *out) {
  const Server *s = h->s;
  if (id < 0 || id >= (int64_t)s->reqs.size()) return FE_EINVAL;
  *out = s->reqs[id].res;
  return FE_OK;
}

fe_status server_stats(const fe_server *h, fe_server_stats *out) {
  const Server *s = h->s;
  memset(out, 0, sizeof *out);
  out->peak_bytes = s->peak_bytes;
  out->live_bytes = s->live_bytes;
  out->base_bytes = s->base_bytes;
  out->estimate_misses = s->estimate_misses;
  out->run_s = s->run_s;
  out->cg_launches = (s->cg ? cg_launches(s->cg) : 0) + (s->cgb ? cg_launches(s->cgb) : 0);
  out->admit_s = s->admit_s;
  out->tick_s = s->tick_s;
  out->retire_s = s->retire_s;
  out->cache_hits = s->cache_hits;
  out->cache_misses = s->cache_misses;
  out->cache_evictions = s->cache_evictions;
  out->sparsity_builds = s->sparsity_builds;
  out->cache_bytes = s->cache_bytes;
  for (const Req &q : s->reqs) {
    out->submitted++;
    if (q.res.status == FE_SOLVE_CONVERGED) out->converged++;
    if (q.res.status == FE_SOLVE_REFUSED) out->refused++;
  }
  return FE_OK;
}

void server_destroy(fe_server *h) {
  server_free(h->s);
  h->magic = 0xDEADu;
  h->s = nullptr;
  delete h;
}

}  // namespace fe
