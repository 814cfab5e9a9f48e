// Internal declarations of libfe: handle layouts and the launch functions of the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fe.h"

namespace fe {

constexpr uint32_t kMagicCtx = 0xFE0C7A11u, kMagicSet = 0xFE05E7u, kMagicMap = 0xFE0AA9u,
                   kMagicDat = 0xFE0DA7u, kMagicSp = 0xFE05BA25u, kMagicMat = 0xFE0AA7u,
                   kMagicKer = 0xFE0CE2u, kMagicGlobal = 0xFE061Bu, kDead = 0xDEADu;

// device error-flag bits (ctx->d_err[0]); d_err[1] keeps the first offending index (low 32 bits)
enum : int { ERR_RANGE = 1, ERR_ROW_TOO_LONG = 2, ERR_NNZ_CHANGED = 4, ERR_CAND_OVERFLOW = 8, ERR_TC_TIMEOUT = 16,
              ERR_LUT = 32 };

// Rows of the CSR pattern are limited to 256 entries so the lookup table fits a byte.
constexpr int kMaxRowLen = 256;
// Per-row candidate capacity of the warp-per-row sparsity kernel (incidence x arity).
constexpr int kMaxCand = 4096;

}  // namespace fe

struct fe_ctx {
  uint32_t magic;
  int device;
  cudaStream_t stream;
  fe_alloc_fn alloc;
  fe_free_fn free_fn;
  void *user;
  int checks;
  int *d_err;  // [4] device ints
};

struct fe_set {
  uint32_t magic;
  fe_ctx *ctx;
  int64_t size;
};

struct fe_map {
  uint32_t magic;
  fe_ctx *ctx;
  fe_set *from, *to;
  int arity;
  const int32_t *values;
};

struct fe_dat {
  uint32_t magic;
  fe_ctx *ctx;
  fe_set *set;
  int dim;
  double *data;
};

struct fe_sparsity {
  uint32_t magic;
  fe_ctx *ctx;
  fe_map *rmap, *cmap;
  int64_t nrows, ncols, ncell;
  int ndr, ndc;
  int64_t nnz;       // known after build
  int cap;           // candidate capacity per row of the row kernel (hash table size, power of two)
  int acap;          // incidence capacity per row (multiple of 4 >= longest incidence list)
  int64_t *rowptr;   // [nrows+1]
  int32_t *colidx;   // [nnz]
  uint8_t *lut;      // [ncell*ndr*ndc]
  int64_t *adjptr;   // [nrows+1]  row -> incidence range
  int32_t *adj;      // [ncell*ndr] e*ndr+i, sorted within each row
  int32_t *rowcnt;   // [nrows] scratch: incidence counts / cursors / unique counts
  int32_t *coltmp;   // [ncell*ndr*ndc] scratch: unique columns at incidence-based offsets
  int64_t *scan_tmp; // scan block sums
  int64_t scan_tmp_elems;
  int *d_maxcnt;     // [1] max incidence count
  int *d_changed;    // [2] rebuild: [0] some row changed its length (the in-place pass is not enough),
                     // [1] some row kept its length but a column changed (nonzero when not tracked)
  int track_cols;    // rebuilds compare each column written in place (fe_sparsity_track_columns)
  int adj_canonical; // each row's incidence list is in ascending order (sparsity_canonical)
  int maxrow;        // longest row (entries), known after build
  void *vstage;      // staging of element vectors for pull action / linear form (lazily allocated)
  size_t vstage_bytes;
};

struct fe_mat {
  uint32_t magic;
  fe_ctx *ctx;
  fe_sparsity *sp;
  double *values;
  void *stage;  // staging of element matrices for pull assembly (lazily allocated)
  size_t stage_bytes;
};

struct fe_global {
  uint32_t magic;
  fe_ctx *ctx;
  int dim;
  double *data;  // dim values (library-owned)
  void *stage;   // element stage of a rank-0 form (lazily allocated)
  size_t stage_bytes;
  double *part;  // per-block partial reductions (lazily allocated)
  size_t part_bytes;
};

struct fe_kernel {
  uint32_t magic;
  fe_ctx *ctx;
  fe_form_desc d;
  int nd;  // nodes of the test/trial element
  int nf;  // nodes of the coefficient element (SOURCE) or dim+1 (kappa)
};

namespace fe {

// ---- scan ----
int64_t scan_tmp_elems(int64_t n);
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.  tmp: scan_tmp_elems(n) int64.
// gate: NULL, or a device flag; when it holds 0 the launches return without work.
cudaError_t exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp,
                                      cudaStream_t s, const int *gate = nullptr);

// ---- maps / sparsity ----
cudaError_t launch_map_validate(const int32_t *v, int64_t n, int64_t limit, int *err, cudaStream_t s);
// incidence: counts -> adjptr (scan) -> adj fill; with_max: also the longest incidence list
// (d_maxcnt, needed to size the row kernel at build time only)
// the sparsity build in stages (fe_api.cpp): asynchronous read-backs into the caller's host slots;
// the caller checks the device flags between stages and discards a failed build
fe_status sparsity_build_begin(fe_ctx *c, fe_map *rmap, fe_map *cmap, fe_sparsity **out, int *h_maxcnt);
fe_status sparsity_build_rows(fe_sparsity *sp, int maxcnt, int64_t *h_nnz, int *h_maxrow);
fe_status sparsity_build_finish(fe_sparsity *sp, int64_t nnz, int maxrow);
fe_status sparsity_check_flags(fe_ctx *c, const char *where);
void sparsity_discard(fe_sparsity *sp);
cudaError_t sparsity_incidence(fe_sparsity *sp, cudaStream_t s, int *err, int with_max = 1);
// rebuild: fill against the previous row offsets (counts checked by the in-place row pass), and
// the full incidence gated on the device flag that pass sets
cudaError_t sparsity_incidence_reuse(fe_sparsity *sp, cudaStream_t s, int *err);
cudaError_t sparsity_incidence_gated(fe_sparsity *sp, cudaStream_t s, int *err, const int *gate);
// sort rows, write lut, unique columns (coltmp at incidence-based offsets), row lengths -> rowptr
// (scan).  gate as for the scan.
cudaError_t sparsity_rows(fe_sparsity *sp, cudaStream_t s, int *err, const int *gate = nullptr);
// rebuild fast pass: as sparsity_rows, but every row whose length equals its length in rowptr
// writes its columns straight to colidx; rowptr is not rewritten.  *changed = 1 when a row's
// length differs or rowptr[nrows] != nnz (then sparsity_rows, its scan and the compaction must
// run, gated on changed).
cudaError_t sparsity_rows_inplace(fe_sparsity *sp, cudaStream_t s, int *err, int *changed);
// Each row's incidence list in ascending order, once per build: the order the row-owner (pull)
// kernels and the wave step sum in.  The row kernel leaves the lists in the fill kernel's order
// (its atomics make that order run-dependent); no-op when already done.
cudaError_t sparsity_canonical(fe_sparsity *sp, cudaStream_t s);
// colidx[rowptr[r] + k] = coltmp[adjptr[r] ndc + k]; check_nnz: flags ERR_NNZ_CHANGED if
// rowptr[nrows] != nnz.  gate as for the scan.
cudaError_t sparsity_compact(fe_sparsity *sp, cudaStream_t s, int *err, int check_nnz,
                             const int *gate = nullptr);
cudaError_t launch_max_i32(const int32_t *v, int64_t n, int *out, cudaStream_t s);

// ---- fills ----
cudaError_t launch_zero_f64(double *p, int64_t n, cudaStream_t s);
cudaError_t launch_zero_i32(int32_t *p, int64_t n, cudaStream_t s);

// ---- sparsity without device allocation (static scratch, fe_noalloc.cu) ----
fe_status sparsity_build_noalloc(const int32_t *rmap, int ndr, const int32_t *cmap, int ndc, int64_t ncell,
                                 int64_t nrows, int64_t ncols, int64_t *rowptr, int32_t *colidx,
                                 int64_t colidx_capacity, uint8_t *lut, int64_t *nnz_out, cudaStream_t s);
const char *noalloc_message();

// ---- device memory through the context's allocator (fe_api.cpp) ----
void *dev_alloc(fe_ctx *c, size_t bytes);
void dev_free(fe_ctx *c, void *p);

// ---- batches (fe_batch.cu) ----
fe_status batch_create(fe_ctx *c, int n, const fe_batch_item *items, void *(*alloc)(fe_ctx *, size_t),
                       void (*release)(fe_ctx *, void *), fe_batch **out);
bool batch_valid(const fe_batch *b);
fe_status batch_views(const fe_batch *b, int i, double **vals, int64_t *nnz, double **rhs, int64_t *nrows);
fe_status batch_assemble(fe_batch *b, int use_graph);
fe_status batch_tune(fe_batch *b, int reps, int *best_tile, int *best_grid, float *best_ms);
void batch_destroy(fe_batch *b, void (*release)(fe_ctx *, void *));
const char *batch_message();
fe_ctx *batch_ctx(const fe_batch *b);

// ---- Dirichlet and CG (fe_solve.cu) ----
cudaError_t launch_dirichlet(int64_t nrows, const int64_t *rowptr, const int32_t *colidx, double *vals, double *b,
                             const uint8_t *is_bc, const double *g, cudaStream_t s);
fe_status cg_create(fe_ctx *c, int max_systems, fe_cg **out);
bool cg_valid(const fe_cg *h);
int64_t cg_launches(const fe_cg *h);
// Rows above which a system is cut into one tile per resident block (one wave of the launch).
int64_t cg_one_wave_rows(const fe_cg *h);
// Blocks the engine launches (one wave of resident blocks by default); cg_limit_grid lowers it,
// before any system is added (the tiling of a system depends on it).
int cg_grid(const fe_cg *h);
fe_status cg_limit_grid(fe_cg *h, int grid);
fe_ctx *cg_ctx(const fe_cg *h);
fe_status cg_add(fe_cg *h, const int64_t *rowptr, const int32_t *colidx, const double *vals, int64_t nrows,
                 const double *b, double *x, double rtol, int maxit, int *slot,
                 int maxrow = 0);
fe_status cg_iterate(fe_cg *h, int iters, int use_graph);
fe_status cg_poll(fe_cg *h, int n, int *status, int *iters, double *rnorm, double *bnorm);
fe_status cg_remove(fe_cg *h, int slot);
void cg_destroy(fe_cg *h);
const char *solve_message();

// ---- request loop (fe_serve.cpp) ----
fe_status server_create(fe_ctx *parent, const fe_server_config *cfg, fe_server **out);
bool server_valid(const fe_server *h);
fe_ctx *server_ctx(const fe_server *h);
fe_status server_submit(fe_server *h, const fe_solve_request *r, int64_t *id);
fe_status server_run(fe_server *h);
fe_status server_result(const fe_server *h, int64_t id, fe_solve_result *out);
fe_status server_stats(const fe_server *h, fe_server_stats *out);
void server_destroy(fe_server *h);
const char *server_message();
size_t noalloc_scratch_bytes();

// ---- assembly ----
struct AsmArgs {
  int64_t ncell;
  const int32_t *map;     // [ncell][nd] test (= trial) map
  const double *coords;   // [nvert][dim]
  const int32_t *cmapv;   // [ncell][dim+1] coordinate map
  int64_t nvert;          // coordinate set size
  int64_t nrows;          // target set size of map
  const double *coef;     // kappa (P1) or f values, may be null
  const int32_t *coefmap; // its map
  int64_t ncoef;          // size of the coefficient's set
  // Mat output
  const int64_t *rowptr;
  const uint8_t *lut;
  double *vals;
  // incidence (pull)
  const int64_t *adjptr;
  const int32_t *adj;
  // vector input/output
  const double *x;
  double *y;
  int *err;
  int checks;
  // staged pull
  void *stage;     // ncell * NUP (Mat) or ncell * ND (action, vector) element values
  int rowcap;      // longest row of the pattern (shared-memory accumulators per row owner)
  int zero_first;  // row kernels overwrite instead of adding
};
using LaunchFn = cudaError_t (*)(const AsmArgs &, cudaStream_t);
// strategy resolved for a call (AUTO -> PULL when the row incidence is available)
int resolve_strategy(const fe_form_desc &d, bool have_incidence);
// bytes of the staging buffer for a pull Mat (ncell * NUP) or vector (ncell * ND) of this kernel
size_t stage_bytes_mat(const fe_form_desc &d, int64_t ncell);
size_t stage_bytes_vec(const fe_form_desc &d, int64_t ncell, int nd);
cudaError_t launch_assemble_mat(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported);
cudaError_t launch_assemble_vec(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported);
cudaError_t launch_action(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported);
// assembly and matrix-free action in one pass (push strategy; FP64 and double-float)
cudaError_t launch_mat_action(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported);
bool kernel_supported(const fe_form_desc &d);

// ---- assembly of the systems a request loop admits together (fe_serve_asm.cu) ----
// One system: a P1 or P2 Laplace Mat on its pattern (mat: staged pull arguments, zero_first) with
// the flagged rows and columns eliminated, and its source right-hand side (vec: f in the same
// space, y = b).  Tiles are numbered across the systems: cells in tiles of kServeCellTile, rows in
// tiles of kServeRowTile; cell_tile0 / row_tile0 are a system's first tiles (non-decreasing).
constexpr int kServeCellTile = 128, kServeRowTile = 256;
struct ServeItem {
  AsmArgs mat, vec;
  void *mstage, *vstage;  // element matrices (full rows) and element vectors, arithmetic type
  const int32_t *colidx;
  const uint8_t *is_bc;
  int p;
  int64_t cell_tile0, row_tile0;
};
// Shared memory of the row launch for a system (rowcap accumulators per row group).
size_t serve_row_smem(int p, int rowcap, int precision);
// Two launches on s: element tensors of every cell, then every row (Mat, elimination, RHS).
cudaError_t launch_serve_assembly(const ServeItem *d_items, int nitems, int64_t cell_tiles, int64_t row_tiles,
                                  size_t row_smem, int precision, cudaStream_t s);

// ---- Globals (fe_global.cu): reductions over cells in a fixed order ----
// element stage of a rank-0 form: K_e x_e (bilinear) or b_e (linear) into a.stage, ND per cell
cudaError_t launch_elem_stage(const fe_form_desc &d, const AsmArgs &a, cudaStream_t s, int *unsupported);
int64_t global_parts(int64_t ncell);  // partial sums of a cell reduction (one per block of cells)
// *g (+)= sum over cells e of sum_i x[map(e)[i]] stage[e nd + i] (stage in the precision's type)
cudaError_t launch_global_dot(int precision, int64_t ncell, int nd, const int32_t *map, const void *stage,
                              const double *x, int64_t nx, double *part, double *g, int zero_first, int checks,
                              int *err, cudaStream_t s);
// *g (op)= reduction (FE_REDUCE_SUM/MIN/MAX) of the cells' volumes |det J| / dim!
cudaError_t launch_cell_volume_reduce(int dim, int op, int64_t ncell, const int32_t *cmapv, const double *coords,
                                      int64_t nvert, double *part, double *g, int zero_first, int checks, int *err,
                                      cudaStream_t s);

// ---- stored element matrices (fe_stored_f64.cu, fe_stored_dd.cu) ----
// Ke: [nd(nd+1)/2][ncell] FP64, entry-major (see fe_stored.cuh)
using StoreFn = cudaError_t (*)(const AsmArgs &, double *, cudaStream_t);
using StoredActionFn = cudaError_t (*)(const AsmArgs &, const double *, cudaStream_t);
cudaError_t launch_elem_store(const fe_form_desc &d, const AsmArgs &a, double *Ke, cudaStream_t s, int *unsupported);
cudaError_t launch_action_stored(const fe_form_desc &d, int nd, const AsmArgs &a, const double *Ke, cudaStream_t s,
                                 int *unsupported);

// ---- explicit wave steps (fe_wave.cu) ----
size_t wave_stage_bytes(int dim, int precision, int64_t ncell);
cudaError_t launch_wave(const fe_form_desc &d, const AsmArgs &a, void *stage, const double *mass,
                        const uint8_t *is_bc, double *p, double t0, double dt, int nsteps,
                        double (*bc_value)(double), cudaStream_t s);

}  // namespace fe
