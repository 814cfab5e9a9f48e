// C ABI of libfe (declared in include/fe.h): handle management, argument validation, the
// allocator, and the host-side sequencing of the sparsity and assembly kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "fe_internal.h"

namespace fe {
// Device memory through the context's allocator (cudaMalloc when none is set), 256-byte granules.
void *dev_alloc(fe_ctx *c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (c->alloc) return c->alloc(bytes, c->user);
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(fe_ctx *c, void *p) {
  if (!p) return;
  if (c->free_fn) c->free_fn(p, c->user);
  else cudaFree(p);
}
}  // namespace fe
using fe::dev_alloc;
using fe::dev_free;

namespace {

thread_local std::string g_err;

fe_status fail(fe_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

fe_status ok() { return FE_OK; }

fe_status cuda_fail(cudaError_t e, const char *where) {
  return fail(FE_ECUDA, "%s: CUDA error %d (%s)", where, (int)e, cudaGetErrorString(e));
}

#define FE_CHECK_CUDA(call, where)            \
  do {                                        \
    cudaError_t _e = (call);                  \
    if (_e != cudaSuccess) return cuda_fail(_e, where); \
  } while (0)

bool valid(const fe_ctx *c) { return c && c->magic == fe::kMagicCtx; }
bool valid(const fe_set *s) { return s && s->magic == fe::kMagicSet && valid(s->ctx); }
bool valid(const fe_map *m) { return m && m->magic == fe::kMagicMap && valid(m->ctx); }
bool valid(const fe_dat *d) { return d && d->magic == fe::kMagicDat && valid(d->ctx); }
bool valid(const fe_sparsity *s) { return s && s->magic == fe::kMagicSp && valid(s->ctx); }
bool valid(const fe_mat *m) { return m && m->magic == fe::kMagicMat && valid(m->ctx); }
bool valid(const fe_kernel *k) { return k && k->magic == fe::kMagicKer && valid(k->ctx); }
bool valid(const fe_global *g) { return g && g->magic == fe::kMagicGlobal && valid(g->ctx); }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};


// An NVTX range around one compute call of the C ABI, so that profilers can group its launches by
// call (header-only NVTX; without an attached tool a call costs a pointer test).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

// Reads and clears the device error flags (synchronises the stream).
fe_status check_device_flags(fe_ctx *c, const char *where) {
  int h[2] = {0, 0};
  FE_CHECK_CUDA(cudaMemcpyAsync(h, c->d_err, sizeof h, cudaMemcpyDeviceToHost, c->stream), where);
  FE_CHECK_CUDA(cudaStreamSynchronize(c->stream), where);
  if (h[0]) {
    int z[2] = {0, 0};
    FE_CHECK_CUDA(cudaMemcpyAsync(c->d_err, z, sizeof z, cudaMemcpyHostToDevice, c->stream), where);
    FE_CHECK_CUDA(cudaStreamSynchronize(c->stream), where);
    if (h[0] & fe::ERR_RANGE) return fail(FE_ERANGE, "%s: a map value lies outside its target set (first index %d)", where, h[1]);
    if (h[0] & fe::ERR_LUT)
      return fail(FE_ERANGE, "%s: a lookup-table entry lies beyond its CSR row (cell %d); the entry was skipped", where,
                  h[1]);
    if (h[0] & fe::ERR_NNZ_CHANGED) return fail(FE_EINVAL, "%s: the rebuilt pattern has a different nnz", where);
    if (h[0] & fe::ERR_TC_TIMEOUT)
      return fail(FE_ETIMEOUT, "%s: a tensor-core product did not complete in time (block %d)", where, h[1]);
    if (h[0] & fe::ERR_ROW_TOO_LONG)
      return fail(FE_EUNSUPPORTED, "%s: a row has more than %d columns (row %d)", where, fe::kMaxRowLen, h[1]);
    if (h[0] & fe::ERR_CAND_OVERFLOW)
      return fail(FE_EUNSUPPORTED, "%s: a row has more than %d candidate entries (row %d)", where, fe::kMaxCand, h[1]);
    return fail(FE_ECUDA, "%s: device error flags 0x%x", where, h[0]);
  }
  return FE_OK;
}

}  // namespace

extern "C" {

const char *fe_last_error(void) { return g_err.c_str(); }
const char *fe_version(void) { return "libfe 0.1 (sm_103a)"; }

// ------------------------------------------------------------------------------------ context
fe_status fe_ctx_create(int device, void *cuda_stream, fe_ctx **out) {
  if (!out) return fail(FE_EINVAL, "fe_ctx_create: out is NULL");
  *out = nullptr;
  int n = 0;
  FE_CHECK_CUDA(cudaGetDeviceCount(&n), "fe_ctx_create");
  if (device < 0 || device >= n) return fail(FE_EINVAL, "fe_ctx_create: device %d of %d", device, n);
  DeviceGuard g(device);
  FE_CHECK_CUDA(cudaSetDevice(device), "fe_ctx_create");
  fe_ctx *c = new (std::nothrow) fe_ctx();
  if (!c) return fail(FE_ENOMEM, "fe_ctx_create: host allocation");
  c->magic = fe::kMagicCtx;
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  c->checks = 0;
  if (cudaMalloc(&c->d_err, 4 * sizeof(int)) != cudaSuccess) {
    delete c;
    return fail(FE_ENOMEM, "fe_ctx_create: device error flags");
  }
  int z[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpy(c->d_err, z, sizeof z, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(c->d_err);
    delete c;
    return cuda_fail(e, "fe_ctx_create");
  }
  *out = c;
  return ok();
}

fe_status fe_ctx_set_stream(fe_ctx *c, void *s) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_ctx_set_stream: invalid context");
  c->stream = (cudaStream_t)s;
  return ok();
}

fe_status fe_ctx_set_allocator(fe_ctx *c, fe_alloc_fn a, fe_free_fn f, void *user) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_ctx_set_allocator: invalid context");
  if ((a == nullptr) != (f == nullptr)) return fail(FE_EINVAL, "fe_ctx_set_allocator: give both or neither");
  c->alloc = a;
  c->free_fn = f;
  c->user = user;
  return ok();
}

fe_status fe_ctx_set_checks(fe_ctx *c, int checks) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_ctx_set_checks: invalid context");
  c->checks = checks != 0;
  return ok();
}

fe_status fe_sync(fe_ctx *c) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_sync: invalid context");
  DeviceGuard g(c->device);
  return check_device_flags(c, "fe_sync");
}

fe_status fe_ctx_destroy(fe_ctx *c) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_ctx_destroy: invalid context");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_err);
  c->magic = fe::kDead;
  delete c;
  return ok();
}

// ------------------------------------------------------------------------------------ Set
fe_status fe_set_create(fe_ctx *c, int64_t size, fe_set **out) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_set_create: invalid context");
  if (!out || size < 0) return fail(FE_EINVAL, "fe_set_create: bad arguments (size %lld)", (long long)size);
  fe_set *s = new (std::nothrow) fe_set{fe::kMagicSet, c, size};
  if (!s) return fail(FE_ENOMEM, "fe_set_create: host allocation");
  *out = s;
  return ok();
}

fe_status fe_set_size(const fe_set *s, int64_t *size) {
  if (!valid(s) || !size) return fail(FE_EHANDLE, "fe_set_size: invalid set");
  *size = s->size;
  return ok();
}

fe_status fe_set_destroy(fe_set *s) {
  if (!valid(s)) return fail(FE_EHANDLE, "fe_set_destroy: invalid set");
  s->magic = fe::kDead;
  delete s;
  return ok();
}

// ------------------------------------------------------------------------------------ Map
fe_status fe_map_create(fe_ctx *c, fe_set *from, fe_set *to, int arity, const int32_t *values, int validate,
                        fe_map **out) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_map_create: invalid context");
  if (!valid(from) || !valid(to) || from->ctx != c || to->ctx != c)
    return fail(FE_EHANDLE, "fe_map_create: sets belong to another context");
  if (!out || arity < 1 || (from->size > 0 && !values))
    return fail(FE_EINVAL, "fe_map_create: bad arguments (arity %d)", arity);
  if (to->size > INT32_MAX) return fail(FE_EUNSUPPORTED, "fe_map_create: target set larger than int32");
  if (validate && from->size > 0) {
    DeviceGuard g(c->device);
    FE_CHECK_CUDA(fe::launch_map_validate(values, from->size * arity, to->size, c->d_err, c->stream), "fe_map_create");
    fe_status st = check_device_flags(c, "fe_map_create");
    if (st != FE_OK) return st;
  }
  fe_map *m = new (std::nothrow) fe_map{fe::kMagicMap, c, from, to, arity, values};
  if (!m) return fail(FE_ENOMEM, "fe_map_create: host allocation");
  *out = m;
  return ok();
}

fe_status fe_map_destroy(fe_map *m) {
  if (!valid(m)) return fail(FE_EHANDLE, "fe_map_destroy: invalid map");
  m->magic = fe::kDead;
  delete m;
  return ok();
}

// ------------------------------------------------------------------------------------ Dat
fe_status fe_dat_create(fe_ctx *c, fe_set *set, int dim, void *ptr, fe_dat **out) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_dat_create: invalid context");
  if (!valid(set) || set->ctx != c) return fail(FE_EHANDLE, "fe_dat_create: set belongs to another context");
  if (!out || dim < 1 || (set->size > 0 && !ptr)) return fail(FE_EINVAL, "fe_dat_create: bad arguments");
  fe_dat *d = new (std::nothrow) fe_dat{fe::kMagicDat, c, set, dim, (double *)ptr};
  if (!d) return fail(FE_ENOMEM, "fe_dat_create: host allocation");
  *out = d;
  return ok();
}

fe_status fe_dat_destroy(fe_dat *d) {
  if (!valid(d)) return fail(FE_EHANDLE, "fe_dat_destroy: invalid dat");
  d->magic = fe::kDead;
  delete d;
  return ok();
}

// ------------------------------------------------------------------------------------ Sparsity
static void sparsity_free(fe_sparsity *sp) {
  fe_ctx *c = sp->ctx;
  dev_free(c, sp->rowptr);
  dev_free(c, sp->colidx);
  dev_free(c, sp->lut);
  dev_free(c, sp->adjptr);
  dev_free(c, sp->adj);
  dev_free(c, sp->rowcnt);
  dev_free(c, sp->coltmp);
  dev_free(c, sp->scan_tmp);
  dev_free(c, sp->d_maxcnt);
  dev_free(c, sp->d_changed);
  dev_free(c, sp->vstage);
}

}  // extern "C"

namespace fe {

// The sparsity build in three stages, each only launching work and asynchronous read-backs into
// the caller's host slots (pinned ones keep every stage free of host synchronisation), so that a
// caller building several patterns waits once per stage for all of them: begin (buffers,
// incidence, the maps' range checks, the longest incidence list), rows (sort, ranks, row
// lengths, rowptr; nnz and the longest row), finish (colidx and its compaction).  The caller
// reads the device flags (check_device_flags) between the stages and discards a failed build.
fe_status sparsity_build_begin(fe_ctx *c, fe_map *rmap, fe_map *cmap, fe_sparsity **out, int *h_maxcnt) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_sparsity_build: invalid context");
  if (!valid(rmap) || !valid(cmap) || rmap->ctx != c || cmap->ctx != c)
    return fail(FE_EHANDLE, "fe_sparsity_build: maps belong to another context");
  if (!out) return fail(FE_EINVAL, "fe_sparsity_build: out is NULL");
  if (rmap->from != cmap->from) return fail(FE_EINVAL, "fe_sparsity_build: row and column maps need the same source set");
  const int64_t ncell = rmap->from->size;
  if (ncell * (int64_t)rmap->arity >= INT32_MAX)
    return fail(FE_EUNSUPPORTED, "fe_sparsity_build: more than 2^31 cell-node incidences");
  if (rmap->arity > 64 || cmap->arity > 64) return fail(FE_EUNSUPPORTED, "fe_sparsity_build: arity above 64");
  DeviceGuard g(c->device);
  fe_sparsity *sp = new (std::nothrow) fe_sparsity();
  if (!sp) return fail(FE_ENOMEM, "fe_sparsity_build: host allocation");
  sp->magic = fe::kMagicSp;
  sp->ctx = c;
  sp->rmap = rmap;
  sp->cmap = cmap;
  sp->nrows = rmap->to->size;
  sp->ncols = cmap->to->size;
  sp->ncell = ncell;
  sp->ndr = rmap->arity;
  sp->ndc = cmap->arity;
  const int64_t ninc = ncell * sp->ndr;
  sp->scan_tmp_elems = fe::scan_tmp_elems(sp->nrows);
  sp->rowptr = (int64_t *)dev_alloc(c, sizeof(int64_t) * (sp->nrows + 1));
  sp->adjptr = (int64_t *)dev_alloc(c, sizeof(int64_t) * (sp->nrows + 1));
  sp->adj = (int32_t *)dev_alloc(c, sizeof(int32_t) * ninc);
  sp->rowcnt = (int32_t *)dev_alloc(c, sizeof(int32_t) * sp->nrows);
  sp->coltmp = (int32_t *)dev_alloc(c, sizeof(int32_t) * ninc * sp->ndc);
  sp->lut = (uint8_t *)dev_alloc(c, (size_t)ninc * sp->ndc);
  sp->scan_tmp = (int64_t *)dev_alloc(c, sizeof(int64_t) * sp->scan_tmp_elems);
  sp->d_maxcnt = (int *)dev_alloc(c, sizeof(int));
  sp->d_changed = (int *)dev_alloc(c, 2 * sizeof(int));  // [0] a row changed length, [1] a column changed
  if (!sp->rowptr || !sp->adjptr || !sp->adj || !sp->rowcnt || !sp->coltmp || !sp->lut || !sp->scan_tmp || !sp->d_maxcnt ||
      !sp->d_changed) {
    sparsity_free(sp);
    delete sp;
    return fail(FE_ENOMEM, "fe_sparsity_build: device allocation failed");
  }
  // the rebuild flags read zero until a rebuild writes them
  cudaError_t e = cudaMemsetAsync(sp->d_changed, 0, 2 * sizeof(int), c->stream);
  // incidence (validates the row map), the column map's range check, the longest incidence list
  if (e == cudaSuccess) e = fe::sparsity_incidence(sp, c->stream, c->d_err);
  if (e == cudaSuccess && cmap->to->size > 0 && ncell > 0)
    e = fe::launch_map_validate(cmap->values, ncell * cmap->arity, cmap->to->size, c->d_err, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_maxcnt, sp->d_maxcnt, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) {
    sparsity_free(sp);
    delete sp;
    return cuda_fail(e, "fe_sparsity_build");
  }
  *out = sp;
  return FE_OK;
}

fe_status sparsity_build_rows(fe_sparsity *sp, int maxcnt, int64_t *h_nnz, int *h_maxrow) {
  fe_ctx *c = sp->ctx;
  DeviceGuard g(c->device);
  const int64_t maxcand = (int64_t)maxcnt * sp->ndc;
  if (maxcand > fe::kMaxCand)
    return fail(FE_EUNSUPPORTED, "fe_sparsity_build: a row has %lld candidate entries (limit %d)", (long long)maxcand,
                fe::kMaxCand);
  sp->cap = 32;
  while (sp->cap < maxcand) sp->cap <<= 1;
  sp->acap = 4;
  while (sp->acap < maxcnt) sp->acap += 4;
  cudaError_t e = fe::sparsity_rows(sp, c->stream, c->d_err);
  if (e == cudaSuccess) e = fe::launch_max_i32(sp->rowcnt, sp->nrows, sp->d_maxcnt, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_nnz, sp->rowptr + sp->nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_maxrow, sp->d_maxcnt, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  return e != cudaSuccess ? cuda_fail(e, "fe_sparsity_build") : FE_OK;
}

fe_status sparsity_build_finish(fe_sparsity *sp, int64_t nnz, int maxrow) {
  fe_ctx *c = sp->ctx;
  DeviceGuard g(c->device);
  sp->nnz = nnz;
  sp->maxrow = maxrow;
  sp->colidx = (int32_t *)dev_alloc(c, sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  if (!sp->colidx) return fail(FE_ENOMEM, "fe_sparsity_build: colidx allocation");
  // stream-ordered: the compaction raises no flag, so nothing waits for it
  cudaError_t e = fe::sparsity_compact(sp, c->stream, c->d_err, 0);
  return e != cudaSuccess ? cuda_fail(e, "fe_sparsity_build") : FE_OK;
}

fe_status sparsity_check_flags(fe_ctx *c, const char *where) { return check_device_flags(c, where); }

void sparsity_discard(fe_sparsity *sp) {
  if (!sp) return;
  sparsity_free(sp);
  delete sp;
}

}  // namespace fe

extern "C" {

fe_status fe_sparsity_build(fe_ctx *c, fe_map *rmap, fe_map *cmap, fe_sparsity **out) {
  Range nvtx_range("fe_sparsity_build");
  fe_sparsity *sp = nullptr;
  int maxcnt = 0, mr = 0;
  int64_t nnz = 0;
  fe_status st = fe::sparsity_build_begin(c, rmap, cmap, &sp, &maxcnt);
  if (st != FE_OK) return st;
  st = check_device_flags(c, "fe_sparsity_build");  // waits for the incidence and the checks
  if (st == FE_OK) st = fe::sparsity_build_rows(sp, maxcnt, &nnz, &mr);
  if (st == FE_OK) st = check_device_flags(c, "fe_sparsity_build");  // waits for the row pass
  if (st == FE_OK) st = fe::sparsity_build_finish(sp, nnz, mr);
  if (st != FE_OK) {
    fe::sparsity_discard(sp);
    return st;
  }
  *out = sp;
  return ok();
}

fe_status fe_sparsity_rebuild(fe_sparsity *sp) {
  Range nvtx_range("fe_sparsity_rebuild");
  if (!valid(sp)) return fail(FE_EHANDLE, "fe_sparsity_rebuild: invalid sparsity");
  fe_ctx *c = sp->ctx;
  DeviceGuard g(c->device);
  if (!sp->coltmp) return fail(FE_EINVAL, "fe_sparsity_rebuild: the pattern's build scratch was released");
  // In-place pass first: rows that keep their lengths go straight to colidx.  Only when a row's
  // length changed do the full row pass, its scan and the compaction run (gated on the device).
  // The incidence is filled against the previous row offsets first; the in-place pass checks each
  // row's count, and a changed count sends the rebuild through the full incidence too.
  FE_CHECK_CUDA(cudaMemsetAsync(sp->d_changed, 0, 2 * sizeof(int), c->stream), "fe_sparsity_rebuild");
  FE_CHECK_CUDA(fe::sparsity_incidence_reuse(sp, c->stream, c->d_err), "fe_sparsity_rebuild");
  FE_CHECK_CUDA(fe::sparsity_rows_inplace(sp, c->stream, c->d_err, sp->d_changed), "fe_sparsity_rebuild");
  FE_CHECK_CUDA(fe::sparsity_incidence_gated(sp, c->stream, c->d_err, sp->d_changed), "fe_sparsity_rebuild");
  FE_CHECK_CUDA(fe::sparsity_rows(sp, c->stream, c->d_err, sp->d_changed), "fe_sparsity_rebuild");
  FE_CHECK_CUDA(fe::sparsity_compact(sp, c->stream, c->d_err, 1, sp->d_changed), "fe_sparsity_rebuild");
  return ok();
}

fe_status fe_sparsity_build_noalloc(const int32_t *rmap, int arity_r, const int32_t *cmap, int arity_c, int64_t ncell,
                                    int64_t nrows, int64_t ncols, int64_t *rowptr, int32_t *colidx,
                                    int64_t colidx_capacity, uint8_t *lut, int64_t *nnz, void *cuda_stream) {
  Range nvtx_range("fe_sparsity_build_noalloc");
  fe_status st = fe::sparsity_build_noalloc(rmap, arity_r, cmap, arity_c, ncell, nrows, ncols, rowptr, colidx,
                                            colidx_capacity, lut, nnz, (cudaStream_t)cuda_stream);
  if (st != FE_OK) return fail(st, "%s", fe::noalloc_message());
  return ok();
}

fe_status fe_sparsity_csr(const fe_sparsity *sp, int64_t *nrows, int64_t *ncols, int64_t *nnz, const int64_t **rowptr,
                          const int32_t **colidx) {
  if (!valid(sp)) return fail(FE_EHANDLE, "fe_sparsity_csr: invalid sparsity");
  if (nrows) *nrows = sp->nrows;
  if (ncols) *ncols = sp->ncols;
  if (nnz) *nnz = sp->nnz;
  if (rowptr) *rowptr = sp->rowptr;
  if (colidx) *colidx = sp->colidx;
  return ok();
}

fe_status fe_sparsity_track_columns(fe_sparsity *sp, int on) {
  if (!valid(sp)) return fail(FE_EHANDLE, "fe_sparsity_track_columns: invalid sparsity");
  sp->track_cols = on != 0;
  return ok();
}

fe_status fe_sparsity_changed(const fe_sparsity *sp, const int **flags) {
  if (!valid(sp)) return fail(FE_EHANDLE, "fe_sparsity_changed: invalid sparsity");
  if (!flags) return fail(FE_EINVAL, "fe_sparsity_changed: flags == NULL");
  *flags = sp->d_changed;
  return ok();
}

fe_status fe_sparsity_lut(const fe_sparsity *sp, const uint8_t **lut) {
  if (!valid(sp) || !lut) return fail(FE_EHANDLE, "fe_sparsity_lut: invalid sparsity");
  *lut = sp->lut;
  return ok();
}

fe_status fe_sparsity_destroy(fe_sparsity *sp) {
  if (!valid(sp)) return fail(FE_EHANDLE, "fe_sparsity_destroy: invalid sparsity");
  DeviceGuard g(sp->ctx->device);
  cudaStreamSynchronize(sp->ctx->stream);
  sparsity_free(sp);
  sp->magic = fe::kDead;
  delete sp;
  return ok();
}

// ------------------------------------------------------------------------------------ Mat
fe_status fe_mat_create(fe_ctx *c, fe_sparsity *sp, fe_mat **out) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_mat_create: invalid context");
  if (!valid(sp) || sp->ctx != c) return fail(FE_EHANDLE, "fe_mat_create: sparsity belongs to another context");
  if (!out) return fail(FE_EINVAL, "fe_mat_create: out is NULL");
  DeviceGuard g(c->device);
  double *v = (double *)dev_alloc(c, sizeof(double) * (sp->nnz > 0 ? sp->nnz : 1));
  if (!v) return fail(FE_ENOMEM, "fe_mat_create: values allocation (%lld entries)", (long long)sp->nnz);
  fe_mat *m = new (std::nothrow) fe_mat{fe::kMagicMat, c, sp, v, nullptr, 0};
  if (!m) {
    dev_free(c, v);
    return fail(FE_ENOMEM, "fe_mat_create: host allocation");
  }
  FE_CHECK_CUDA(fe::launch_zero_f64(v, sp->nnz, c->stream), "fe_mat_create");
  *out = m;
  return ok();
}

fe_status fe_mat_values(const fe_mat *m, double **values) {
  if (!valid(m) || !values) return fail(FE_EHANDLE, "fe_mat_values: invalid mat");
  *values = m->values;
  return ok();
}

fe_status fe_mat_zero(fe_mat *m) {
  Range nvtx_range("fe_mat_zero");
  if (!valid(m)) return fail(FE_EHANDLE, "fe_mat_zero: invalid mat");
  DeviceGuard g(m->ctx->device);
  FE_CHECK_CUDA(fe::launch_zero_f64(m->values, m->sp->nnz, m->ctx->stream), "fe_mat_zero");
  return ok();
}

fe_status fe_mat_destroy(fe_mat *m) {
  if (!valid(m)) return fail(FE_EHANDLE, "fe_mat_destroy: invalid mat");
  DeviceGuard g(m->ctx->device);
  cudaStreamSynchronize(m->ctx->stream);
  dev_free(m->ctx, m->values);
  dev_free(m->ctx, m->stage);
  m->magic = fe::kDead;
  delete m;
  return ok();
}

// ------------------------------------------------------------------------------------ Kernel
static int num_nodes(int dim, int p) {
  if (dim == 2) return (p + 1) * (p + 2) / 2;
  if (dim == 3) return (p + 1) * (p + 2) * (p + 3) / 6;
  return -1;
}

fe_status fe_kernel_create(fe_ctx *c, const fe_form_desc *d, fe_kernel **out) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_kernel_create: invalid context");
  if (!d || !out) return fail(FE_EINVAL, "fe_kernel_create: NULL argument");
  if (d->dim < 2 || d->dim > 3 || d->degree < 1) return fail(FE_EINVAL, "fe_kernel_create: dim %d degree %d", d->dim, d->degree);
  if (!fe::kernel_supported(*d))
    return fail(FE_EUNSUPPORTED, "fe_kernel_create: form %d on P%d (dim %d, coefficient P%d, precision %d) is not built in",
                d->form, d->degree, d->dim, d->coeff_degree, d->precision);
  fe_kernel *k = new (std::nothrow) fe_kernel();
  if (!k) return fail(FE_ENOMEM, "fe_kernel_create: host allocation");
  k->magic = fe::kMagicKer;
  k->ctx = c;
  k->d = *d;
  k->nd = num_nodes(d->dim, d->degree);
  k->nf = d->form == FE_FORM_SOURCE ? num_nodes(d->dim, d->coeff_degree) : d->dim + 1;
  *out = k;
  return ok();
}

fe_status fe_kernel_destroy(fe_kernel *k) {
  if (!valid(k)) return fail(FE_EHANDLE, "fe_kernel_destroy: invalid kernel");
  k->magic = fe::kDead;
  delete k;
  return ok();
}

// ------------------------------------------------------------------------------------ par_loops
static fe_status common_args(const char *who, fe_ctx *c, fe_kernel *k, fe_set *cells, fe_map *map, fe_dat *coords,
                             fe_map *coord_map, fe::AsmArgs &a) {
  if (!valid(c)) return fail(FE_EHANDLE, "%s: invalid context", who);
  if (!valid(k) || k->ctx != c) return fail(FE_EHANDLE, "%s: invalid kernel", who);
  if (!valid(cells) || cells->ctx != c) return fail(FE_EHANDLE, "%s: invalid cell set", who);
  if (!valid(map) || map->ctx != c) return fail(FE_EHANDLE, "%s: invalid map", who);
  if (!valid(coords) || coords->ctx != c) return fail(FE_EHANDLE, "%s: invalid coordinate dat", who);
  if (!valid(coord_map) || coord_map->ctx != c) return fail(FE_EHANDLE, "%s: invalid coordinate map", who);
  if (map->from != cells || coord_map->from != cells) return fail(FE_EINVAL, "%s: maps must start from the iteration set", who);
  if (map->arity != k->nd) return fail(FE_EARITY, "%s: map arity %d, element has %d nodes", who, map->arity, k->nd);
  if (coord_map->arity != k->d.dim + 1) return fail(FE_EARITY, "%s: coordinate map arity %d", who, coord_map->arity);
  if (coords->dim != k->d.dim || coords->set != coord_map->to)
    return fail(FE_EINVAL, "%s: coordinates must be a dim-%d Dat on the coordinate map's target", who, k->d.dim);
  memset(&a, 0, sizeof a);
  a.ncell = cells->size;
  a.map = map->values;
  a.coords = coords->data;
  a.cmapv = coord_map->values;
  a.nvert = coords->set->size;
  a.nrows = map->to->size;
  a.err = c->d_err;
  a.checks = c->checks;
  return FE_OK;
}

static fe_status kappa_arg(const char *who, fe_ctx *c, fe_kernel *k, fe_set *cells, const fe_arg *coeffs, int ncoeffs,
                           fe::AsmArgs &a) {
  if (k->d.form != FE_FORM_KAPPA_DIFFUSION) return FE_OK;
  if (ncoeffs < 1 || !coeffs || !valid(coeffs[0].dat) || !valid(coeffs[0].map) || coeffs[0].dat->ctx != c)
    return fail(FE_EINVAL, "%s: kappa-diffusion needs one coefficient", who);
  if (coeffs[0].map->from != cells || coeffs[0].map->arity != k->d.dim + 1 || coeffs[0].dat->set != coeffs[0].map->to ||
      coeffs[0].dat->dim != 1)
    return fail(FE_EARITY, "%s: kappa must be a scalar P1 Dat with a map of arity dim+1", who);
  a.coef = coeffs[0].dat->data;
  a.coefmap = coeffs[0].map->values;
  a.ncoef = coeffs[0].dat->set->size;
  return FE_OK;
}

// Staging buffers of the pull strategy, allocated on first use and kept with their owner.
static fe_status ensure_stage(fe_ctx *c, void **buf, size_t *have, size_t need, const char *who) {
  if (*buf && *have >= need) return FE_OK;
  dev_free(c, *buf);
  *buf = dev_alloc(c, need);
  *have = *buf ? need : 0;
  if (!*buf) return fail(FE_ENOMEM, "%s: staging buffer of %zu bytes", who, need);
  return FE_OK;
}

fe_status fe_assemble_mat(fe_ctx *c, fe_kernel *k, fe_set *cells, fe_mat *A, int zero_first, fe_dat *coords,
                          fe_map *coord_map, const fe_arg *coeffs, int ncoeffs) {
  Range nvtx_range("fe_assemble_mat");
  const char *who = "fe_assemble_mat";
  if (!valid(A) || A->ctx != c) return fail(FE_EHANDLE, "%s: invalid mat", who);
  fe::AsmArgs a;
  fe_status st = common_args(who, c, k, cells, A->sp->rmap, coords, coord_map, a);
  if (st != FE_OK) return st;
  if (A->sp->rmap != A->sp->cmap) return fail(FE_EUNSUPPORTED, "%s: only square forms (same test and trial map)", who);
  if (k->d.form == FE_FORM_SOURCE) return fail(FE_EINVAL, "%s: a linear form assembles into a Dat", who);
  st = kappa_arg(who, c, k, cells, coeffs, ncoeffs, a);
  if (st != FE_OK) return st;
  a.rowptr = A->sp->rowptr;
  a.lut = A->sp->lut;
  a.vals = A->values;
  a.adjptr = A->sp->adjptr;
  a.adj = A->sp->adj;
  a.rowcap = A->sp->maxrow;
  a.zero_first = zero_first;
  DeviceGuard g(c->device);
  const bool pull = fe::resolve_strategy(k->d, true) == FE_STRATEGY_PULL;
  if (pull) {
    FE_CHECK_CUDA(fe::sparsity_canonical(A->sp, c->stream), who);  // row owners sum in incidence order
    st = ensure_stage(c, &A->stage, &A->stage_bytes, fe::stage_bytes_mat(k->d, cells->size), who);
    if (st != FE_OK) return st;
    a.stage = A->stage;
  } else if (zero_first) {
    FE_CHECK_CUDA(fe::launch_zero_f64(A->values, A->sp->nnz, c->stream), who);
  }
  int unsup = 0;
  FE_CHECK_CUDA(fe::launch_assemble_mat(k->d, a, c->stream, &unsup), who);
  if (unsup) return fail(FE_EUNSUPPORTED, "%s: no kernel for this form/strategy", who);
  return ok();
}

// The row incidence used by the pull strategy of a vector par_loop: that of a sparsity built from
// (map, map).  AUTO uses it when given; PULL requires it.
static fe_status pull_incidence(const char *who, fe_ctx *c, fe_kernel *k, fe_set *cells, fe_map *map,
                                const fe_sparsity *sp, fe::AsmArgs &a) {
  const bool have = sp && valid(sp) && sp->ctx == c;
  if (have && (sp->rmap != map || sp->ncell != cells->size))
    return fail(FE_EINVAL, "%s: the sparsity was not built from this map", who);
  if (fe::resolve_strategy(k->d, have) != FE_STRATEGY_PULL) return FE_OK;
  if (!have) return fail(FE_EINVAL, "%s: the pull strategy needs the sparsity built from (map, map)", who);
  a.adjptr = sp->adjptr;
  a.adj = sp->adj;
  DeviceGuard g(c->device);  // the row owners sum in incidence order: canonical, once per build
  FE_CHECK_CUDA(fe::sparsity_canonical(const_cast<fe_sparsity *>(sp), c->stream), who);
  return FE_OK;
}

fe_status fe_assemble_vec(fe_ctx *c, fe_kernel *k, fe_set *cells, fe_dat *b, fe_map *test_map, int zero_first,
                          fe_dat *coords, fe_map *coord_map, const fe_arg *coeffs, int ncoeffs, const fe_sparsity *sp) {
  Range nvtx_range("fe_assemble_vec");
  const char *who = "fe_assemble_vec";
  fe::AsmArgs a;
  fe_status st = common_args(who, c, k, cells, test_map, coords, coord_map, a);
  if (st != FE_OK) return st;
  if (k->d.form != FE_FORM_SOURCE) return fail(FE_EINVAL, "%s: kernel is not a linear form", who);
  if (!valid(b) || b->ctx != c || b->set != test_map->to || b->dim != 1)
    return fail(FE_EINVAL, "%s: b must be a scalar Dat on the test map's target", who);
  if (ncoeffs < 1 || !coeffs || !valid(coeffs[0].dat) || !valid(coeffs[0].map) || coeffs[0].map->from != cells ||
      coeffs[0].map->arity != k->nf || coeffs[0].dat->set != coeffs[0].map->to || coeffs[0].dat->dim != 1)
    return fail(FE_EARITY, "%s: f must be a scalar Dat with a map of arity %d", who, k->nf);
  a.coef = coeffs[0].dat->data;
  a.coefmap = coeffs[0].map->values;
  a.ncoef = coeffs[0].dat->set->size;
  a.y = b->data;
  a.zero_first = zero_first;
  st = pull_incidence(who, c, k, cells, test_map, sp, a);
  if (st != FE_OK) return st;
  DeviceGuard g(c->device);
  if (a.adj) {
    fe_sparsity *msp = const_cast<fe_sparsity *>(sp);
    st = ensure_stage(c, &msp->vstage, &msp->vstage_bytes, fe::stage_bytes_vec(k->d, cells->size, k->nd), who);
    if (st != FE_OK) return st;
    a.stage = msp->vstage;
  } else if (zero_first) {
    FE_CHECK_CUDA(fe::launch_zero_f64(b->data, b->set->size, c->stream), who);
  }
  int unsup = 0;
  FE_CHECK_CUDA(fe::launch_assemble_vec(k->d, a, c->stream, &unsup), who);
  if (unsup) return fail(FE_EUNSUPPORTED, "%s: no kernel for this form/strategy", who);
  return ok();
}

fe_status fe_action(fe_ctx *c, fe_kernel *k, fe_set *cells, fe_dat *x, fe_dat *y, fe_map *map, int zero_first,
                    fe_dat *coords, fe_map *coord_map, const fe_arg *coeffs, int ncoeffs, const fe_sparsity *sp) {
  Range nvtx_range("fe_action");
  const char *who = "fe_action";
  fe::AsmArgs a;
  fe_status st = common_args(who, c, k, cells, map, coords, coord_map, a);
  if (st != FE_OK) return st;
  if (k->d.form == FE_FORM_SOURCE) return fail(FE_EINVAL, "%s: the action needs a bilinear form", who);
  if (!valid(x) || !valid(y) || x->ctx != c || y->ctx != c || x->set != map->to || y->set != map->to || x->dim != 1 ||
      y->dim != 1)
    return fail(FE_EINVAL, "%s: x and y must be scalar Dats on the map's target", who);
  if (x->data == y->data) return fail(FE_EINVAL, "%s: x and y must not alias", who);
  st = kappa_arg(who, c, k, cells, coeffs, ncoeffs, a);
  if (st != FE_OK) return st;
  a.x = x->data;
  a.y = y->data;
  a.zero_first = zero_first;
  st = pull_incidence(who, c, k, cells, map, sp, a);
  if (st != FE_OK) return st;
  DeviceGuard g(c->device);
  if (a.adj) {
    fe_sparsity *msp = const_cast<fe_sparsity *>(sp);
    st = ensure_stage(c, &msp->vstage, &msp->vstage_bytes, fe::stage_bytes_vec(k->d, cells->size, k->nd), who);
    if (st != FE_OK) return st;
    a.stage = msp->vstage;
  } else if (zero_first) {
    FE_CHECK_CUDA(fe::launch_zero_f64(y->data, y->set->size, c->stream), who);
  }
  int unsup = 0;
  FE_CHECK_CUDA(fe::launch_action(k->d, a, c->stream, &unsup), who);
  if (unsup) return fail(FE_EUNSUPPORTED, "%s: no kernel for this form/strategy", who);
  return ok();
}

fe_status fe_assemble_mat_action(fe_ctx *c, fe_kernel *k, fe_set *cells, fe_mat *A, fe_dat *x, fe_dat *y,
                                 fe_map *map, int zero_first, fe_dat *coords, fe_map *coord_map, const fe_arg *coeffs,
                                 int ncoeffs) {
  Range nvtx_range("fe_assemble_mat_action");
  const char *who = "fe_assemble_mat_action";
  if (!valid(A) || A->ctx != c) return fail(FE_EHANDLE, "%s: invalid mat", who);
  fe::AsmArgs a;
  fe_status st = common_args(who, c, k, cells, map, coords, coord_map, a);
  if (st != FE_OK) return st;
  if (A->sp->rmap != map || A->sp->cmap != map)
    return fail(FE_EINVAL, "%s: the Mat's sparsity must be built from (map, map)", who);
  if (k->d.form == FE_FORM_SOURCE) return fail(FE_EINVAL, "%s: the kernel must be a bilinear form", who);
  if (!valid(x) || !valid(y) || x->ctx != c || y->ctx != c || x->set != map->to || y->set != map->to || x->dim != 1 ||
      y->dim != 1)
    return fail(FE_EINVAL, "%s: x and y must be scalar Dats on the map's target", who);
  if (x->data == y->data) return fail(FE_EINVAL, "%s: x and y must not alias", who);
  st = kappa_arg(who, c, k, cells, coeffs, ncoeffs, a);
  if (st != FE_OK) return st;
  a.rowptr = A->sp->rowptr;
  a.lut = A->sp->lut;
  a.vals = A->values;
  a.x = x->data;
  a.y = y->data;
  DeviceGuard g(c->device);
  if (zero_first) {
    FE_CHECK_CUDA(fe::launch_zero_f64(A->values, A->sp->nnz, c->stream), who);
    FE_CHECK_CUDA(fe::launch_zero_f64(y->data, y->set->size, c->stream), who);
  }
  int unsup = 0;
  FE_CHECK_CUDA(fe::launch_mat_action(k->d, a, c->stream, &unsup), who);
  if (unsup) return fail(FE_EUNSUPPORTED, "%s: no fused kernel for this form, precision or strategy", who);
  return ok();
}

// ------------------------------------------------------------------------------------ Global
fe_status fe_global_create(fe_ctx *c, int dim, fe_global **out) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_global_create: invalid context");
  if (!out || dim < 1) return fail(FE_EINVAL, "fe_global_create: bad arguments (dim %d)", dim);
  DeviceGuard g(c->device);
  double *v = (double *)dev_alloc(c, sizeof(double) * dim);
  if (!v) return fail(FE_ENOMEM, "fe_global_create: device allocation failed");
  FE_CHECK_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * dim, c->stream), "fe_global_create");
  fe_global *h = new (std::nothrow) fe_global{fe::kMagicGlobal, c, dim, v, nullptr, 0, nullptr, 0};
  if (!h) {
    dev_free(c, v);
    return fail(FE_ENOMEM, "fe_global_create: host allocation");
  }
  *out = h;
  return ok();
}

fe_status fe_global_data(const fe_global *g, double **values) {
  if (!valid(g)) return fail(FE_EHANDLE, "fe_global_data: invalid global");
  if (!values) return fail(FE_EINVAL, "fe_global_data: values == NULL");
  *values = g->data;
  return ok();
}

fe_status fe_global_destroy(fe_global *g) {
  if (!valid(g)) return fail(FE_EHANDLE, "fe_global_destroy: invalid global");
  DeviceGuard dg(g->ctx->device);
  cudaStreamSynchronize(g->ctx->stream);
  dev_free(g->ctx, g->data);
  dev_free(g->ctx, g->stage);
  dev_free(g->ctx, g->part);
  g->magic = fe::kDead;
  delete g;
  return ok();
}

// Rank-0 forms: the element stage of the pull kernels (K_e x_e, or b_e for the linear form), then
// the deterministic sum of x_e . stage_e over the cells.
fe_status fe_assemble_global(fe_ctx *c, fe_kernel *k, fe_set *cells, fe_global *g, int zero_first, fe_dat *x,
                             fe_map *map, fe_dat *coords, fe_map *coord_map, const fe_arg *coeffs, int ncoeffs) {
  Range nvtx_range("fe_assemble_global");
  const char *who = "fe_assemble_global";
  fe::AsmArgs a;
  fe_status st = common_args(who, c, k, cells, map, coords, coord_map, a);
  if (st != FE_OK) return st;
  if (!valid(g) || g->ctx != c) return fail(FE_EHANDLE, "%s: invalid global", who);
  if (!valid(x) || x->ctx != c || x->set != map->to || x->dim != 1)
    return fail(FE_EINVAL, "%s: x must be a scalar Dat on the map's target", who);
  if (k->d.form == FE_FORM_SOURCE) {
    if (ncoeffs < 1 || !coeffs || !valid(coeffs[0].dat) || !valid(coeffs[0].map) || coeffs[0].map->from != cells ||
        coeffs[0].map->arity != k->nf || coeffs[0].dat->set != coeffs[0].map->to || coeffs[0].dat->dim != 1)
      return fail(FE_EARITY, "%s: f must be a scalar Dat with a map of arity %d", who, k->nf);
    a.coef = coeffs[0].dat->data;
    a.coefmap = coeffs[0].map->values;
    a.ncoef = coeffs[0].dat->set->size;
  } else {
    st = kappa_arg(who, c, k, cells, coeffs, ncoeffs, a);
    if (st != FE_OK) return st;
    a.x = x->data;
  }
  DeviceGuard dg(c->device);
  st = ensure_stage(c, &g->stage, &g->stage_bytes,
                    std::max<size_t>(fe::stage_bytes_vec(k->d, cells->size, k->nd), 16), who);
  if (st != FE_OK) return st;
  void *part = g->part;
  st = ensure_stage(c, &part, &g->part_bytes, sizeof(double) * (size_t)fe::global_parts(cells->size), who);
  g->part = static_cast<double *>(part);
  if (st != FE_OK) return st;
  a.stage = g->stage;
  int unsup = 0;
  FE_CHECK_CUDA(fe::launch_elem_stage(k->d, a, c->stream, &unsup), who);
  if (unsup) return fail(FE_EUNSUPPORTED, "%s: no element kernel for this form and precision", who);
  FE_CHECK_CUDA(fe::launch_global_dot(k->d.precision, cells->size, k->nd, map->values, g->stage, x->data,
                                      x->set->size, g->part, g->data, zero_first, c->checks, c->d_err, c->stream),
                who);
  return ok();
}

fe_status fe_reduce_cell_volume(fe_ctx *c, fe_set *cells, fe_global *g, int op, int zero_first, fe_dat *coords,
                                fe_map *coord_map) {
  Range nvtx_range("fe_reduce_cell_volume");
  const char *who = "fe_reduce_cell_volume";
  if (!valid(c)) return fail(FE_EHANDLE, "%s: invalid context", who);
  if (!valid(cells) || cells->ctx != c) return fail(FE_EHANDLE, "%s: invalid cell set", who);
  if (!valid(g) || g->ctx != c) return fail(FE_EHANDLE, "%s: invalid global", who);
  if (!valid(coords) || coords->ctx != c) return fail(FE_EHANDLE, "%s: invalid coordinate dat", who);
  if (!valid(coord_map) || coord_map->ctx != c) return fail(FE_EHANDLE, "%s: invalid coordinate map", who);
  if (op != FE_REDUCE_SUM && op != FE_REDUCE_MIN && op != FE_REDUCE_MAX) return fail(FE_EINVAL, "%s: op %d", who, op);
  const int dim = coords->dim;
  if (dim != 2 && dim != 3) return fail(FE_EINVAL, "%s: coordinates of dimension %d", who, dim);
  if (coord_map->from != cells || coords->set != coord_map->to)
    return fail(FE_EINVAL, "%s: the coordinate map must go from the cells to the coordinates' set", who);
  if (coord_map->arity != dim + 1) return fail(FE_EARITY, "%s: coordinate map arity %d", who, coord_map->arity);
  DeviceGuard dg(c->device);
  void *part = g->part;
  fe_status st = ensure_stage(c, &part, &g->part_bytes, sizeof(double) * (size_t)fe::global_parts(cells->size), who);
  g->part = static_cast<double *>(part);
  if (st != FE_OK) return st;
  FE_CHECK_CUDA(fe::launch_cell_volume_reduce(dim, op, cells->size, coord_map->values, coords->data, coords->set->size,
                                              g->part, g->data, zero_first, c->checks, c->d_err, c->stream),
                who);
  return ok();
}

// ------------------------------------------------------------------------------------ stored element matrices
fe_status fe_elem_matrices(fe_ctx *c, fe_kernel *k, fe_set *cells, double *Ke, fe_dat *coords, fe_map *coord_map,
                           const fe_arg *coeffs, int ncoeffs) {
  Range nvtx_range("fe_elem_matrices");
  const char *who = "fe_elem_matrices";
  if (!valid(c)) return fail(FE_EHANDLE, "%s: invalid context", who);
  if (!valid(k) || k->ctx != c) return fail(FE_EHANDLE, "%s: invalid kernel", who);
  if (!valid(cells) || cells->ctx != c) return fail(FE_EHANDLE, "%s: invalid cell set", who);
  if (!valid(coords) || coords->ctx != c) return fail(FE_EHANDLE, "%s: invalid coordinate dat", who);
  if (!valid(coord_map) || coord_map->ctx != c) return fail(FE_EHANDLE, "%s: invalid coordinate map", who);
  if (coord_map->from != cells) return fail(FE_EINVAL, "%s: the coordinate map must start from the iteration set", who);
  if (coord_map->arity != k->d.dim + 1) return fail(FE_EARITY, "%s: coordinate map arity %d", who, coord_map->arity);
  if (coords->dim != k->d.dim || coords->set != coord_map->to)
    return fail(FE_EINVAL, "%s: coordinates must be a dim-%d Dat on the coordinate map's target", who, k->d.dim);
  if (k->d.form == FE_FORM_SOURCE) return fail(FE_EUNSUPPORTED, "%s: element matrices need a bilinear form", who);
  if (!Ke && cells->size > 0) return fail(FE_EINVAL, "%s: Ke is NULL", who);
  fe::AsmArgs a;
  memset(&a, 0, sizeof a);
  a.ncell = cells->size;
  a.coords = coords->data;
  a.cmapv = coord_map->values;
  a.nvert = coords->set->size;
  a.err = c->d_err;
  a.checks = c->checks;
  fe_status st = kappa_arg(who, c, k, cells, coeffs, ncoeffs, a);
  if (st != FE_OK) return st;
  DeviceGuard g(c->device);
  int unsup = 0;
  FE_CHECK_CUDA(fe::launch_elem_store(k->d, a, Ke, c->stream, &unsup), who);
  if (unsup) return fail(FE_EUNSUPPORTED, "%s: no stored-matrix kernel for this form/element/precision", who);
  return ok();
}

fe_status fe_action_stored(fe_ctx *c, fe_kernel *k, fe_set *cells, const double *Ke, fe_dat *x, fe_dat *y, fe_map *map,
                           int zero_first) {
  Range nvtx_range("fe_action_stored");
  const char *who = "fe_action_stored";
  if (!valid(c)) return fail(FE_EHANDLE, "%s: invalid context", who);
  if (!valid(k) || k->ctx != c) return fail(FE_EHANDLE, "%s: invalid kernel", who);
  if (!valid(cells) || cells->ctx != c) return fail(FE_EHANDLE, "%s: invalid cell set", who);
  if (!valid(map) || map->ctx != c) return fail(FE_EHANDLE, "%s: invalid map", who);
  if (map->from != cells) return fail(FE_EINVAL, "%s: the map must start from the iteration set", who);
  if (map->arity != k->nd) return fail(FE_EARITY, "%s: map arity %d, element has %d nodes", who, map->arity, k->nd);
  if (k->d.form == FE_FORM_SOURCE) return fail(FE_EUNSUPPORTED, "%s: the action needs a bilinear form", who);
  if (!valid(x) || !valid(y) || x->ctx != c || y->ctx != c || x->set != map->to || y->set != map->to || x->dim != 1 ||
      y->dim != 1)
    return fail(FE_EINVAL, "%s: x and y must be scalar Dats on the map's target", who);
  if (x->data == y->data) return fail(FE_EINVAL, "%s: x and y must not alias", who);
  if (!Ke && cells->size > 0) return fail(FE_EINVAL, "%s: Ke is NULL", who);
  fe::AsmArgs a;
  memset(&a, 0, sizeof a);
  a.ncell = cells->size;
  a.map = map->values;
  a.nrows = map->to->size;
  a.x = x->data;
  a.y = y->data;
  a.err = c->d_err;
  a.checks = c->checks;
  DeviceGuard g(c->device);
  if (zero_first) FE_CHECK_CUDA(fe::launch_zero_f64(y->data, y->set->size, c->stream), who);
  int unsup = 0;
  FE_CHECK_CUDA(fe::launch_action_stored(k->d, k->nd, a, Ke, c->stream, &unsup), who);
  if (unsup) return fail(FE_EUNSUPPORTED, "%s: no stored-matrix kernel for this form/element/precision", who);
  return ok();
}

// ------------------------------------------------------------------------------------ batches
static void *batch_alloc(fe_ctx *c, size_t n) { return dev_alloc(c, n); }
static void batch_release(fe_ctx *c, void *p) { dev_free(c, p); }

fe_status fe_batch_create(fe_ctx *c, int n, const fe_batch_item *items, fe_batch **out) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_batch_create: invalid context");
  if (n < 0 || (n > 0 && !items) || !out) return fail(FE_EINVAL, "fe_batch_create: bad arguments");
  for (int i = 0; i < n; i++) {
    const fe_batch_item &it = items[i];
    if (!valid(it.kmat) || it.kmat->ctx != c || (it.kvec && (!valid(it.kvec) || it.kvec->ctx != c)) ||
        !valid(it.cells) || it.cells->ctx != c || !valid(it.sp) || it.sp->ctx != c || !valid(it.coords) ||
        it.coords->ctx != c || !valid(it.coord_map) || it.coord_map->ctx != c ||
        (it.kvec && (!valid(it.f.dat) || !valid(it.f.map) || it.f.dat->ctx != c || it.f.map->ctx != c)))
      return fail(FE_EHANDLE, "fe_batch_create: item %d has an invalid handle", i);
  }
  DeviceGuard g(c->device);
  fe_status st = fe::batch_create(c, n, items, batch_alloc, batch_release, out);
  if (st != FE_OK) return fail(st, "%s", fe::batch_message()[0] ? fe::batch_message() : "fe_batch_create failed");
  return ok();
}

fe_status fe_batch_values(const fe_batch *b, int item, double **values, int64_t *nnz, double **rhs, int64_t *nrows) {
  if (!fe::batch_valid(b)) return fail(FE_EHANDLE, "fe_batch_values: invalid batch");
  if (fe::batch_views(b, item, values, nnz, rhs, nrows) != FE_OK) return fail(FE_EINVAL, "fe_batch_values: item %d", item);
  return ok();
}

fe_status fe_batch_tune(fe_batch *b, int reps, int *tile_cells, int *grid, float *ms) {
  Range nvtx_range("fe_batch_tune");
  if (!fe::batch_valid(b)) return fail(FE_EHANDLE, "fe_batch_tune: invalid batch");
  DeviceGuard g(fe::batch_ctx(b)->device);
  fe_status st = fe::batch_tune(b, reps, tile_cells, grid, ms);
  if (st != FE_OK) return fail(st, "%s", fe::batch_message());
  return ok();
}

fe_status fe_batch_assemble(fe_batch *b, int use_graph) {
  Range nvtx_range("fe_batch_assemble");
  if (!fe::batch_valid(b)) return fail(FE_EHANDLE, "fe_batch_assemble: invalid batch");
  DeviceGuard g(fe::batch_ctx(b)->device);
  fe_status st = fe::batch_assemble(b, use_graph);
  if (st != FE_OK) return fail(st, "%s", fe::batch_message());
  return ok();
}

fe_status fe_batch_destroy(fe_batch *b) {
  if (!fe::batch_valid(b)) return fail(FE_EHANDLE, "fe_batch_destroy: invalid batch");
  DeviceGuard g(fe::batch_ctx(b)->device);
  fe::batch_destroy(b, batch_release);
  return ok();
}

// ------------------------------------------------------------------------------------ wave steps
static double wave_bc_value(double t) {
  constexpr double kPi = 3.14159265358979323846;
  return sin(10.0 * kPi * t);
}

fe_status fe_wave_steps(fe_ctx *c, fe_kernel *k, fe_set *cells, fe_dat *phi, fe_dat *p, const double *mass,
                        const uint8_t *is_bc, fe_map *map, fe_dat *coords, fe_map *coord_map, const fe_sparsity *sp,
                        double t0, double dt, int nsteps) {
  Range nvtx_range("fe_wave_steps");
  const char *who = "fe_wave_steps";
  fe::AsmArgs a;
  fe_status st = common_args(who, c, k, cells, map, coords, coord_map, a);
  if (st != FE_OK) return st;
  if (k->d.form != FE_FORM_LAPLACE || k->d.degree != 1 ||
      (k->d.precision != FE_PREC_FP64 && k->d.precision != FE_PREC_F32X2))
    return fail(FE_EUNSUPPORTED, "%s: P1 Laplace kernels in FP64 or double-float only", who);
  if (!valid(phi) || !valid(p) || phi->ctx != c || p->ctx != c || phi->set != map->to || p->set != map->to ||
      phi->dim != 1 || p->dim != 1 || phi->data == p->data)
    return fail(FE_EINVAL, "%s: phi and p must be distinct scalar Dats on the map's target", who);
  if (nsteps < 0 || !(dt == dt) || (map->to->size > 0 && !mass)) return fail(FE_EINVAL, "%s: bad nsteps, dt or mass", who);
  if (!sp || !valid(sp) || sp->ctx != c || sp->rmap != map || sp->ncell != cells->size)
    return fail(FE_EINVAL, "%s: sp must be the sparsity built from (map, map)", who);
  a.x = phi->data;
  a.y = phi->data;
  a.adjptr = sp->adjptr;
  a.adj = sp->adj;
  DeviceGuard g(c->device);
  fe_sparsity *msp = const_cast<fe_sparsity *>(sp);
  FE_CHECK_CUDA(fe::sparsity_canonical(msp, c->stream), who);  // rows sum in incidence order
  st = ensure_stage(c, &msp->vstage, &msp->vstage_bytes, fe::wave_stage_bytes(k->d.dim, k->d.precision, cells->size),
                    who);
  if (st != FE_OK) return st;
  FE_CHECK_CUDA(fe::launch_wave(k->d, a, msp->vstage, mass, is_bc, p->data, t0, dt, nsteps, wave_bc_value, c->stream),
                who);
  return ok();
}

// ------------------------------------------------------------------------------------ Dirichlet
fe_status fe_dirichlet_apply(fe_ctx *c, fe_mat *A, fe_dat *b, const uint8_t *is_bc, const double *g) {
  Range nvtx_range("fe_dirichlet_apply");
  const char *who = "fe_dirichlet_apply";
  if (!valid(c)) return fail(FE_EHANDLE, "%s: invalid context", who);
  if (!valid(A) || A->ctx != c || !valid(b) || b->ctx != c) return fail(FE_EHANDLE, "%s: invalid mat or dat", who);
  const fe_sparsity *sp = A->sp;
  if (sp->rmap != sp->cmap || sp->nrows != sp->ncols) return fail(FE_EINVAL, "%s: A must be square", who);
  if (b->set != sp->rmap->to || b->dim != 1) return fail(FE_EINVAL, "%s: b must be a scalar Dat on A's rows", who);
  if (sp->nrows > 0 && !is_bc) return fail(FE_EINVAL, "%s: is_bc is NULL", who);
  DeviceGuard gd(c->device);
  FE_CHECK_CUDA(fe::launch_dirichlet(sp->nrows, sp->rowptr, sp->colidx, A->values, b->data, is_bc, g, c->stream), who);
  return ok();
}

// ------------------------------------------------------------------------------------ CG
fe_status fe_cg_create(fe_ctx *c, int max_systems, fe_cg **out) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_cg_create: invalid context");
  if (max_systems < 1 || max_systems > (1 << 20) || !out) return fail(FE_EINVAL, "fe_cg_create: bad arguments");
  DeviceGuard g(c->device);
  fe_status st = fe::cg_create(c, max_systems, out);
  if (st != FE_OK) return fail(st, "%s", fe::solve_message()[0] ? fe::solve_message() : "fe_cg_create failed");
  return ok();
}

fe_status fe_cg_add(fe_cg *cg, fe_mat *A, fe_dat *b, fe_dat *x, double rtol, int maxit, int *slot) {
  Range nvtx_range("fe_cg_add");
  const char *who = "fe_cg_add";
  if (!fe::cg_valid(cg)) return fail(FE_EHANDLE, "%s: invalid engine", who);
  fe_ctx *c = fe::cg_ctx(cg);
  if (!valid(A) || A->ctx != c || !valid(b) || b->ctx != c || !valid(x) || x->ctx != c)
    return fail(FE_EHANDLE, "%s: A, b and x must belong to the engine's context", who);
  const fe_sparsity *sp = A->sp;
  if (sp->rmap != sp->cmap || sp->nrows != sp->ncols) return fail(FE_EINVAL, "%s: A must be square", who);
  if (b->set != sp->rmap->to || x->set != sp->rmap->to || b->dim != 1 || x->dim != 1 || b->data == x->data)
    return fail(FE_EINVAL, "%s: b and x must be distinct scalar Dats on A's rows", who);
  if (!(rtol >= 0.0) || maxit < 0 || !slot) return fail(FE_EINVAL, "%s: bad rtol, maxit or slot", who);
  DeviceGuard g(c->device);
  fe_status st =
      fe::cg_add(cg, sp->rowptr, sp->colidx, A->values, sp->nrows, b->data, x->data, rtol, maxit, slot, sp->maxrow);
  if (st != FE_OK) return fail(st, "%s", fe::solve_message());
  return ok();
}

fe_status fe_cg_iterate(fe_cg *cg, int iters, int use_graph) {
  Range nvtx_range("fe_cg_iterate");
  if (!fe::cg_valid(cg)) return fail(FE_EHANDLE, "fe_cg_iterate: invalid engine");
  if (iters < 0) return fail(FE_EINVAL, "fe_cg_iterate: iters < 0");
  DeviceGuard g(fe::cg_ctx(cg)->device);
  fe_status st = fe::cg_iterate(cg, iters, use_graph);
  if (st != FE_OK) return fail(st, "%s", fe::solve_message());
  return ok();
}

fe_status fe_cg_poll(fe_cg *cg, int nslots, int *status, int *iters, double *rnorm, double *bnorm) {
  if (!fe::cg_valid(cg)) return fail(FE_EHANDLE, "fe_cg_poll: invalid engine");
  DeviceGuard g(fe::cg_ctx(cg)->device);
  fe_status st = fe::cg_poll(cg, nslots, status, iters, rnorm, bnorm);
  if (st != FE_OK) return fail(st, "%s", fe::solve_message());
  return ok();
}

fe_status fe_cg_remove(fe_cg *cg, int slot) {
  if (!fe::cg_valid(cg)) return fail(FE_EHANDLE, "fe_cg_remove: invalid engine");
  DeviceGuard g(fe::cg_ctx(cg)->device);
  fe_status st = fe::cg_remove(cg, slot);
  if (st != FE_OK) return fail(st, "%s", fe::solve_message());
  return ok();
}

fe_status fe_cg_destroy(fe_cg *cg) {
  if (!fe::cg_valid(cg)) return fail(FE_EHANDLE, "fe_cg_destroy: invalid engine");
  DeviceGuard g(fe::cg_ctx(cg)->device);
  fe::cg_destroy(cg);
  return ok();
}

// ------------------------------------------------------------------------------------ serving
fe_status fe_server_create(fe_ctx *c, const fe_server_config *cfg, fe_server **out) {
  if (!valid(c)) return fail(FE_EHANDLE, "fe_server_create: invalid context");
  if (!cfg || !out) return fail(FE_EINVAL, "fe_server_create: bad arguments");
  DeviceGuard g(c->device);
  fe_status st = fe::server_create(c, cfg, out);
  if (st != FE_OK) return fail(st, "%s", fe::server_message());
  return ok();
}

fe_status fe_server_submit(fe_server *srv, const fe_solve_request *req, int64_t *id) {
  if (!fe::server_valid(srv)) return fail(FE_EHANDLE, "fe_server_submit: invalid server");
  if (!req) return fail(FE_EINVAL, "fe_server_submit: req is NULL");
  fe_status st = fe::server_submit(srv, req, id);
  if (st != FE_OK) return fail(st, "%s", fe::server_message());
  return ok();
}

fe_status fe_server_run(fe_server *srv) {
  Range nvtx_range("fe_server_run");
  if (!fe::server_valid(srv)) return fail(FE_EHANDLE, "fe_server_run: invalid server");
  DeviceGuard g(fe::server_ctx(srv)->device);
  fe_status st = fe::server_run(srv);
  if (st != FE_OK) return fail(st, "%s", fe::server_message());
  return ok();
}

fe_status fe_server_result(const fe_server *srv, int64_t id, fe_solve_result *out) {
  if (!fe::server_valid(srv)) return fail(FE_EHANDLE, "fe_server_result: invalid server");
  if (!out || fe::server_result(srv, id, out) != FE_OK) return fail(FE_EINVAL, "fe_server_result: no request %lld", (long long)id);
  return ok();
}

fe_status fe_server_stats_get(const fe_server *srv, fe_server_stats *out) {
  if (!fe::server_valid(srv)) return fail(FE_EHANDLE, "fe_server_stats_get: invalid server");
  if (!out) return fail(FE_EINVAL, "fe_server_stats_get: out is NULL");
  return fe::server_stats(srv, out) == FE_OK ? ok() : fail(FE_EINVAL, "fe_server_stats_get failed");
}

fe_status fe_server_destroy(fe_server *srv) {
  if (!fe::server_valid(srv)) return fail(FE_EHANDLE, "fe_server_destroy: invalid server");
  DeviceGuard g(fe::server_ctx(srv)->device);
  fe::server_destroy(srv);
  return ok();
}

}  // extern "C"
