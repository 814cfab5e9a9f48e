/*
 * fe.h -- C ABI of libfe, GB300-native cell-wise finite element assembly.
 *
 * The calls follow the data model and execution model of PyOP2 as described in
 * Rathgeber et al., "Firedrake: automating the finite element method by composing
 * abstractions" (ACM TOMS), Sec. 4:
 *   Sets (Sec. 4.1), Maps of constant arity (Sec. 4.2), Dats and Mats (Sec. 4.3),
 *   parallel loops with access descriptors READ / INC (Sec. 4.4, 4.4.1), Mats assembled
 *   through a pair of Maps (Sec. 4.4.3), and the form-assembly argument order of the
 *   Firedrake layer (Sec. 5.1.3: output tensor, then coordinates, then coefficients).
 *
 * General conventions
 *  - Every function returns an fe_status; 0 (FE_OK) on success, a negative code otherwise,
 *    with a message available from fe_last_error() on the calling thread.  No call aborts.
 *  - Device buffers passed in (map values, coordinates, coefficient and output vectors) are
 *    BORROWED: the caller owns them and keeps them alive while any handle refers to them.
 *    Buffers the library creates (CSR pattern, lookup tables, Mat values, scratch) are
 *    OWNED by the returned handle and freed by its destroy call; they are allocated through
 *    the context's allocator (fe_ctx_set_allocator), by default cudaMalloc.
 *  - Compute calls are asynchronous on the context's CUDA stream.  Errors that only the
 *    device can detect (map values out of range when checks are on) are reported by the
 *    next fe_sync() as FE_ERANGE.
 *  - Cells are simplices: triangles (dim 2) or tetrahedra (dim 3), affine (P1 coordinates).
 *  - Lagrange P_p local node order (the column order of a cell-node Map): nodes are the
 *    lattice points sum_m alpha_m x_m / p of the cell (x_m its vertices, |alpha| = p):
 *    the vertices 0..dim; then each edge (a, b), a < b, in lexicographic order, walked from
 *    a to b (alpha_a = p - t, alpha_b = t, t = 1..p-1); then each face (a, b, c), a < b < c,
 *    lexicographic, interior points by descending alpha_a, then alpha_b; then (3D) the cell
 *    interior by descending alpha_0, alpha_1, alpha_2.
 *  - Index types: map values int32; CSR rowptr int64, colidx int32 (columns sorted per row).
 */
#ifndef FE_H
#define FE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int fe_status;
#define FE_OK 0
#define FE_EINVAL (-1)        /* bad argument (null pointer, size, mismatched sets)          */
#define FE_EHANDLE (-2)       /* handle belongs to another context or was destroyed           */
#define FE_ERANGE (-3)        /* a map value lies outside its target set                      */
#define FE_EARITY (-4)        /* map arity does not match the element of the kernel           */
#define FE_ENOMEM (-5)        /* the allocator failed                                         */
#define FE_ECUDA (-6)         /* a CUDA runtime call failed (message has the CUDA error)      */
#define FE_ETIMEOUT (-7)      /* a bounded device wait gave up                                */
#define FE_EUNSUPPORTED (-8)  /* form/element/size combination not built into this library   */

typedef struct fe_ctx fe_ctx;
typedef struct fe_set fe_set;
typedef struct fe_map fe_map;
typedef struct fe_dat fe_dat;
typedef struct fe_sparsity fe_sparsity;
typedef struct fe_mat fe_mat;
typedef struct fe_kernel fe_kernel;

/* Forms (Sec. 3.1, Listing 1: a = inner(grad u, grad v) dx, L = f v dx; plus mass and
 * kappa-weighted diffusion with kappa a P1 Function). */
typedef enum {
  FE_FORM_MASS = 1,             /* u v dx                                    */
  FE_FORM_LAPLACE = 2,          /* inner(grad u, grad v) dx                  */
  FE_FORM_HELMHOLTZ = 3,        /* inner(grad u, grad v) dx + u v dx         */
  FE_FORM_KAPPA_DIFFUSION = 4,  /* kappa inner(grad u, grad v) dx, kappa P1  */
  FE_FORM_SOURCE = 5            /* linear: f v dx, f in P_q                  */
} fe_form;

/* Arithmetic of the element tensor.  Accumulation into the global Mat/Dat is FP64 always. */
typedef enum {
  FE_PREC_FP64 = 0,   /* native IEEE double                                               */
  FE_PREC_F32X2 = 1,  /* pairs of FP32 (error-free transformations), ~2^-46 relative     */
  FE_PREC_TF32X3 = 3, /* tensor cores (tcgen05): three TF32 products of hi/lo splits, FP32
                         accumulation in TMEM, FP64 global accumulation; P4 kappa-diffusion Mat on
                         triangles, push only                                            */
  FE_PREC_FP32 = 2    /* single FP32 (triangles, push): the precision study of high-order
                         elements, ~1e-7 relative element error                           */
} fe_precision;

/* How the INC into the global Mat/Dat is executed. */
typedef enum {
  FE_STRATEGY_AUTO = 0,  /* the library's faster choice on this hardware: currently PUSH       */
  FE_STRATEGY_PUSH = 1,  /* one thread per cell, FP64 atomic adds through the lookup table */
  FE_STRATEGY_PULL = 2   /* staged: element tensors stored per cell, then one owner per row
                            sums its cells' contributions in the fixed incidence order --
                            no atomics, bitwise reproducible results; uses a staging buffer
                            (ncell x upper triangle, or ncell x nodes, values) per Mat or
                            sparsity, allocated on first use                                 */
} fe_strategy;

typedef struct {
  int form;          /* fe_form                                                           */
  int dim;           /* 2 (triangles) or 3 (tetrahedra)                                   */
  int degree;        /* Lagrange degree p of the test (= trial) space                     */
  int coeff_degree;  /* degree of the coefficient f (FE_FORM_SOURCE); kappa is always P1  */
  int precision;     /* fe_precision                                                      */
  int strategy;      /* fe_strategy                                                       */
} fe_form_desc;

/* A coefficient argument (READ through its own map), Sec. 5.1.3. */
typedef struct {
  fe_dat *dat;
  fe_map *map;
} fe_arg;

/* Device allocator hooks: alloc(bytes, user) returns a device pointer or NULL. */
typedef void *(*fe_alloc_fn)(size_t bytes, void *user);
typedef void (*fe_free_fn)(void *ptr, void *user);

/* Message of the last failing call on this thread ("" if none).  Never NULL. */
const char *fe_last_error(void);

/* Library version string. */
const char *fe_version(void);

/* ---------------------------------------------------------------- context
 * fe_ctx_create: binds a device and a CUDA stream (cudaStream_t passed as void*, borrowed;
 * NULL = the legacy default stream).  Allocates a small device error-flag buffer.
 * Errors: FE_EINVAL (out == NULL), FE_ECUDA (bad device). */
fe_status fe_ctx_create(int device, void *cuda_stream, fe_ctx **out);
fe_status fe_ctx_set_stream(fe_ctx *ctx, void *cuda_stream);
/* Replace the allocator for buffers created after this call (NULL, NULL = cudaMalloc). */
fe_status fe_ctx_set_allocator(fe_ctx *ctx, fe_alloc_fn alloc, fe_free_fn free_fn, void *user);
/* checks != 0: kernels verify every map value against its target set and flag FE_ERANGE. */
fe_status fe_ctx_set_checks(fe_ctx *ctx, int checks);
/* Waits for the context stream, then reports (and clears) any device-side error flag. */
fe_status fe_sync(fe_ctx *ctx);
fe_status fe_ctx_destroy(fe_ctx *ctx);

/* ---------------------------------------------------------------- Set (Sec. 4.1)
 * An abstract entity count; stores no data.  Errors: FE_EINVAL (size < 0). */
fe_status fe_set_create(fe_ctx *ctx, int64_t size, fe_set **out);
fe_status fe_set_size(const fe_set *set, int64_t *size);
fe_status fe_set_destroy(fe_set *set);

/* ---------------------------------------------------------------- Map (Sec. 4.2)
 * Constant-arity map from -> to.  dev_values: device int32 [from.size][arity], row-major,
 * borrowed.  validate != 0 runs a range-check kernel and synchronises: FE_ERANGE if any value
 * lies outside [0, to.size).  Errors: FE_EINVAL (arity < 1, null values with from.size > 0). */
fe_status fe_map_create(fe_ctx *ctx, fe_set *from, fe_set *to, int arity, const int32_t *dev_values,
                        int validate, fe_map **out);
fe_status fe_map_destroy(fe_map *map);

/* ---------------------------------------------------------------- Dat (Sec. 4.3)
 * A vector of dim float64 values per set element: device [set.size][dim], borrowed. */
fe_status fe_dat_create(fe_ctx *ctx, fe_set *set, int dim, void *dev_ptr, fe_dat **out);
fe_status fe_dat_destroy(fe_dat *dat);

/* ---------------------------------------------------------------- Sparsity (Sec. 4.4.3)
 * Builds on the device the CSR pattern of the union over cells e of
 * {(rmap(e)[i], cmap(e)[j])}: rows = rmap target set, columns = cmap target set, columns
 * sorted ascending, no duplicates (bitwise deterministic).  Also builds the per-cell lookup
 * table giving, for each (e, i, j), the position of cmap(e)[j] within row rmap(e)[i], and the
 * row -> (cell, local index) incidence used by the row-owner (pull) kernels (put into ascending
 * order by the first pull or wave call after each build, which is what makes their sums
 * bitwise reproducible; push calls never need it).  rmap and cmap
 * must share their source set (the cells).  Owned buffers.  Synchronises the stream twice (the
 * longest incidence list and the maps' range checks, then nnz and the longest row); the last
 * kernel, the colidx compaction, is still in flight on the stream when it returns.  Errors: FE_EINVAL (different source sets), FE_ERANGE (map value out of range),
 * FE_EUNSUPPORTED (a row with more than 256 columns or more than 4096 candidate entries). */
fe_status fe_sparsity_build(fe_ctx *ctx, fe_map *rmap, fe_map *cmap, fe_sparsity **out);
/* Recomputes pattern, lookup table and incidence from the (possibly rewritten) map values into
 * the existing buffers, asynchronously (no host synchronisation).  The caller guarantees the
 * pattern size is unchanged; a changed nnz is flagged on the device and reported by fe_sync as
 * FE_EINVAL.  This is the per-step sparsity build of the benchmark.  The incidence is filled
 * against the previous row offsets, and a first row pass checks every row's incidence count and
 * writes every row whose length is unchanged straight into colidx; only when some count or row
 * length changed (e.g. relabelled nodes) do the full incidence (count, scan, fill), the full row
 * pass, the row-pointer scan and the colidx compaction run (their launches are gated on a device
 * flag, so the call stays asynchronous).  The result is the same either way. */
fe_status fe_sparsity_rebuild(fe_sparsity *sp);
/* Device pointer to two ints written by each fe_sparsity_rebuild (zero after fe_sparsity_build):
 * flags[0] != 0 when some row changed length (the rebuild ran its full path); flags[1] != 0 when
 * some row kept its length but its columns changed, or when the sparsity does not track columns
 * (then every rebuild sets it).  With column tracking on, rowptr and colidx equal those before the
 * rebuild exactly when both flags are 0, so a caller holding a copy of the pattern needs to read
 * it again only when a flag is set.  Read them after the rebuild's work on the stream (a
 * stream-ordered copy, or fe_sync). */
fe_status fe_sparsity_changed(const fe_sparsity *sp, const int **flags);
/* Column tracking (off after fe_sparsity_build; on != 0 turns it on, 0 off) for the rebuilds that
 * follow: the in-place row pass compares each column it would write with the one already there,
 * writes only a different one and reports it in flags[1] of fe_sparsity_changed.  The compares
 * add about an eighth to the row pass's instructions.  Host call, no device work; FE_EHANDLE for
 * an invalid handle. */
fe_status fe_sparsity_track_columns(fe_sparsity *sp, int on);
/* Read-only views of the CSR pattern (device pointers owned by sp). */
fe_status fe_sparsity_csr(const fe_sparsity *sp, int64_t *nrows, int64_t *ncols, int64_t *nnz,
                          const int64_t **rowptr, const int32_t **colidx);
/* Device pointer to the uint8 lookup table [ncell][arity_r][arity_c] (rank within the row). */
fe_status fe_sparsity_lut(const fe_sparsity *sp, const uint8_t **lut);
fe_status fe_sparsity_destroy(fe_sparsity *sp);

/* ---------------------------------------------------------------- Sparsity without allocation
 * The paper has no counterpart to this call.  It computes exactly what fe_sparsity_build
 * computes (same kernels, bitwise identical pattern and lookup table) for callers that must not
 * allocate device memory: code whose device memory is a budget owned by another runtime (an
 * arena or pool that stray cudaMalloc calls would bypass or overrun), and code that cannot
 * afford cudaMalloc's latency and device-wide synchronisation where it builds patterns.
 * There is no context or handle: inputs and outputs are the caller's device buffers, and the
 * kernels' scratch is one static device array of about 23 MB that every GPU loading the library
 * holds until the process exits.  Limits (FE_EUNSUPPORTED beyond them): nrows <= 262144,
 * ncell * arity_r <= 1048576, ncell * arity_r * arity_c <= 4194304, per-row limits as for
 * fe_sparsity_build.
 *   rmap, cmap  device int32 [ncell][arity_r], [ncell][arity_c] (read)
 *   rowptr      device int64 [nrows + 1] (written)
 *   colidx      device int32 [colidx_capacity] (written); NULL = size query: rowptr and lut are
 *               written, *nnz is set, colidx is not touched
 *   lut         device uint8 [ncell][arity_r][arity_c] (written), rank of cmap(e)[j] in row rmap(e)[i]
 *   nnz         host, set to the number of entries of the pattern
 * Errors: FE_EINVAL (bad argument, or colidx_capacity < nnz -- nnz is still reported),
 * FE_ERANGE (a map value outside its target set), FE_EUNSUPPORTED, FE_ECUDA.
 * Synchronises cuda_stream (it reads nnz).  The first call on a device looks up the array's
 * device address with that device current; make it before any stream capture on that device.
 * The address is kept for the life of the process: after cudaDeviceReset on that device (which
 * unloads the module and its array) this entry point must not be called again.
 * All calls share the array and it keeps the last call's contents (each call clears what must
 * start at zero); calls that overlap on the GPU race on it, so serialise them. */
fe_status fe_sparsity_build_noalloc(const int32_t *rmap, int arity_r, const int32_t *cmap, int arity_c, int64_t ncell,
                                    int64_t nrows, int64_t ncols, int64_t *rowptr, int32_t *colidx,
                                    int64_t colidx_capacity, uint8_t *lut, int64_t *nnz, void *cuda_stream);

/* ---------------------------------------------------------------- Mat (Sec. 4.3, 4.4.3)
 * FP64 values over a sparsity (owned, [nnz]), write-only to par_loops (INC). */
fe_status fe_mat_create(fe_ctx *ctx, fe_sparsity *sp, fe_mat **out);
fe_status fe_mat_values(const fe_mat *mat, double **values);
fe_status fe_mat_zero(fe_mat *mat);
fe_status fe_mat_destroy(fe_mat *mat);

/* ---------------------------------------------------------------- Kernel (Sec. 5.2)
 * Selects the generated local kernel for (form, dim, degree[, coeff_degree], precision,
 * strategy).  Errors: FE_EUNSUPPORTED if the combination is not compiled in. */
fe_status fe_kernel_create(fe_ctx *ctx, const fe_form_desc *desc, fe_kernel **out);
fe_status fe_kernel_destroy(fe_kernel *k);

/* ---------------------------------------------------------------- par_loops (Sec. 4.4, 5.1.3)
 * fe_assemble_mat: A(INC, (map, map)) over the cells; coords (a Dat of dim float64 per vertex)
 * READ through coord_map (arity dim+1); coefficients READ through their maps (kappa for
 * FE_FORM_KAPPA_DIFFUSION: one P1 coefficient).  A's sparsity must have been built from
 * (map, map).  zero_first != 0 clears A first (MatZeroEntries).
 * Errors: FE_EINVAL, FE_EARITY, FE_EHANDLE, FE_EUNSUPPORTED. */
fe_status fe_assemble_mat(fe_ctx *ctx, fe_kernel *k, fe_set *cells, fe_mat *A, int zero_first,
                          fe_dat *coords, fe_map *coord_map, const fe_arg *coeffs, int ncoeffs);
/* fe_assemble_vec: b(INC, test_map) for FE_FORM_SOURCE; coeffs[0] = f (P_q through its map).
 * For the pull strategy sp must be the sparsity built from (test_map, test_map) (its
 * incidence is reused); it may be NULL for push. */
fe_status fe_assemble_vec(fe_ctx *ctx, fe_kernel *k, fe_set *cells, fe_dat *b, fe_map *test_map,
                          int zero_first, fe_dat *coords, fe_map *coord_map, const fe_arg *coeffs,
                          int ncoeffs, const fe_sparsity *sp);
/* fe_action: y(INC, map) = A(x) cell by cell without forming A (the bilinear form with its
 * trial argument replaced by the Function x, as the paper's wave step assembles
 * inner(grad v, grad phi) dx each step, Sec. 6.3); x READ through map.  sp as for
 * fe_assemble_vec. */
fe_status fe_action(fe_ctx *ctx, fe_kernel *k, fe_set *cells, fe_dat *x, fe_dat *y, fe_map *map,
                    int zero_first, fe_dat *coords, fe_map *coord_map, const fe_arg *coeffs,
                    int ncoeffs, const fe_sparsity *sp);

/* fe_assemble_mat_action: fe_assemble_mat and fe_action of the same bilinear kernel in one pass
 * over the cells.  A(INC, (map, map)) += K_e and y(INC, map) += K_e x_e, x READ through map:
 * each cell's element matrix is computed once, in registers, for both outputs, and no assembled
 * matrix is read for y (the action stays matrix-free, Sec. 6.3).  zero_first != 0 clears A and y
 * first.  The push strategy only (AUTO or PUSH), FE_PREC_FP64 (every compiled element) or
 * FE_PREC_F32X2 (P1, P2); the results equal the two separate calls' within rounding (y's products
 * are summed in another order).
 * Errors: FE_EINVAL (x and y alias, sets), FE_EARITY, FE_EHANDLE, FE_EUNSUPPORTED. */
fe_status fe_assemble_mat_action(fe_ctx *ctx, fe_kernel *k, fe_set *cells, fe_mat *A, fe_dat *x, fe_dat *y,
                                 fe_map *map, int zero_first, fe_dat *coords, fe_map *coord_map,
                                 const fe_arg *coeffs, int ncoeffs);

/* ---------------------------------------------------------------- Global (Sec. 4.3, 4.4)
 * A Global is a tuple of values tied to no set (a 0-linear operator beside the Dat and the Mat,
 * Sec. 4.3).  par_loops reach it either by READ or through a reduction: SUM, MIN or MAX
 * ("Global arguments", Sec. 4.4), for integrated quantities such as an energy.  Every reduction
 * here sums (or takes the minimum or maximum of) per-cell values in a fixed order: one partial
 * per block of cells, then the partials in block order, so its result is the same on every run.
 * fe_global_create: dim FP64 values on the device, library-owned, zeroed on the context's
 * stream.  fe_global_data: their device pointer (read them after fe_sync).
 * Errors: FE_EINVAL (dim < 1, out == NULL), FE_EHANDLE, FE_ENOMEM. */
typedef struct fe_global fe_global;
enum { FE_REDUCE_SUM = 0, FE_REDUCE_MIN = 1, FE_REDUCE_MAX = 2 };
fe_status fe_global_create(fe_ctx *ctx, int dim, fe_global **out);
fe_status fe_global_data(const fe_global *g, double **values);
fe_status fe_global_destroy(fe_global *g);
/* fe_assemble_global: a form of rank 0 into g[0] with SUM access (zero_first != 0 overwrites,
 * else adds).  With a bilinear kernel both arguments become the Function x (READ through map):
 * g = a(x, x) = sum_e x_e^T K_e x_e, the energy of x (the action of Sec. 6.3 applied twice).
 * With FE_FORM_SOURCE the test argument becomes x: g = L(x) = sum_e b_e . x_e, the integral of
 * f x (coeffs[0] = f as for fe_assemble_vec).  Element tensors in FE_PREC_FP64 (every compiled
 * element) or FE_PREC_F32X2 (P1, P2); the sum over cells in FP64.  Scratch (an element stage of
 * ncell * nd values and the partials) is held by g and grows to the largest call.
 * Errors: FE_EINVAL, FE_EARITY, FE_EHANDLE, FE_EUNSUPPORTED, FE_ENOMEM. */
fe_status fe_assemble_global(fe_ctx *ctx, fe_kernel *k, fe_set *cells, fe_global *g, int zero_first,
                             fe_dat *x, fe_map *map, fe_dat *coords, fe_map *coord_map,
                             const fe_arg *coeffs, int ncoeffs);
/* fe_reduce_cell_volume: g[0] (op)= op over the cells of |det J| / dim! (op = FE_REDUCE_SUM: the
 * domain's volume; MIN / MAX: the smallest / largest cell), coordinates READ through coord_map
 * (arity dim + 1, dim 2 or 3).  zero_first != 0 overwrites g[0] with the reduction; with no
 * cells that is 0 (SUM), +inf (MIN) or -inf (MAX).
 * Errors: FE_EINVAL (op, dim), FE_EARITY, FE_EHANDLE, FE_ENOMEM. */
fe_status fe_reduce_cell_volume(fe_ctx *ctx, fe_set *cells, fe_global *g, int op, int zero_first,
                                fe_dat *coords, fe_map *coord_map);

/* ---------------------------------------------------------------- stored element matrices
 * The stored-matrix alternative to fe_action, which recomputes every element matrix at each
 * application.  fe_elem_matrices runs the local kernel of a bilinear form once per cell (the
 * gather of coordinates and coefficients, geometry and element tensor of fe_assemble_mat,
 * Sec. 4.4 and 5.2) and stores the matrices; fe_action_stored applies them,
 * y[map(e)[i]] (INC) += sum_j K_e[i][j] x[map(e)[j]], x READ through map, without the element
 * arithmetic.  The trade: nd(nd+1)/2 FP64 values of device memory per cell (440 bytes for P2
 * tetrahedra) against that arithmetic at every application.
 * Ke: caller-owned device buffer of nd(nd+1)/2 * ncell doubles, entry-major: entry u of the upper
 *     triangle of cell e, u counting the pairs (i, j), i <= j, row by row, is Ke[u * ncell + e].
 *     Ke must not change between the two calls' use of it (stream order).
 * Kernels: bilinear forms in FE_PREC_FP64 (every compiled element) or FE_PREC_F32X2 (P1, P2; the
 *     element tensor and the product in FP32 pairs); stored values and the INC are FP64 in both;
 *     the INC is by FP64 atomics (push; the kernel's strategy field is not used).
 * fe_action_stored: zero_first != 0 clears y first.  With checks on, map values outside the
 *     target set are reported by fe_sync as FE_ERANGE.
 * Errors: FE_EHANDLE, FE_EINVAL (NULL Ke with cells, sets or Dats that do not match, x aliasing
 * y), FE_EARITY, FE_EUNSUPPORTED (linear form, other precisions or elements). */
fe_status fe_elem_matrices(fe_ctx *ctx, fe_kernel *k, fe_set *cells, double *Ke, fe_dat *coords,
                           fe_map *coord_map, const fe_arg *coeffs, int ncoeffs);
fe_status fe_action_stored(fe_ctx *ctx, fe_kernel *k, fe_set *cells, const double *Ke, fe_dat *x,
                           fe_dat *y, fe_map *map, int zero_first);

/* ---------------------------------------------------------------- batches of meshes
 * Many independent problems assembled together (the fixed per-par_loop overhead the paper
 * identifies as the limit of strong scaling, Sec. 6.4.2, paid once for the whole batch).  Each
 * item is one Mat (bilinear kmat, push) with an optional right-hand side (kvec = f v dx with f in
 * the same space, coefficient f): Mass, Laplace or Helmholtz on P1 or P2 triangles, FP64 or
 * double-float.  The batch owns one contiguous buffer of all items' CSR values and one of all
 * right-hand sides (views by fe_batch_values).  fe_batch_assemble zeroes both and assembles every
 * item in one persistent launch: CTAs take (item, cell range) tiles from a device work counter.
 * use_graph != 0 captures the two launches once into a CUDA graph on the context stream and
 * replays it.  fe_batch_tune times tile sizes and grid sizes on the batch (synchronising) and keeps
 * the fastest.  Errors: FE_EUNSUPPORTED (element/form/precision), FE_EINVAL, FE_ENOMEM, FE_ECUDA. */
typedef struct fe_batch fe_batch;
typedef struct {
  fe_kernel *kmat;        /* bilinear form (its strategy is ignored: push)                   */
  fe_kernel *kvec;        /* FE_FORM_SOURCE with coeff_degree = degree, or NULL               */
  fe_set *cells;
  fe_sparsity *sp;        /* built from (map, map) of this item                               */
  fe_dat *coords;         /* dim-2 vertex coordinates                                         */
  fe_map *coord_map;      /* cells -> vertices, arity 3                                       */
  fe_arg f;               /* coefficient of the linear form (ignored if kvec is NULL)         */
} fe_batch_item;
fe_status fe_batch_create(fe_ctx *ctx, int nitems, const fe_batch_item *items, fe_batch **out);
fe_status fe_batch_values(const fe_batch *b, int item, double **values, int64_t *nnz, double **rhs, int64_t *nrows);
fe_status fe_batch_tune(fe_batch *b, int reps, int *tile_cells, int *grid, float *ms_per_step);
fe_status fe_batch_assemble(fe_batch *b, int use_graph);
fe_status fe_batch_destroy(fe_batch *b);

/* ---------------------------------------------------------------- boundary conditions
 * Strong Dirichlet conditions u = g on the rows flagged in is_bc, by symmetric elimination of the
 * assembled system (the Poisson listing of Sec. 3.1 assembles A and b with its boundary condition
 * applied; Sec. 6.2 states u = 0 on the Dirichlet boundary).  For every row i not flagged,
 * b_i -= sum over flagged j of A_ij g_j and A_ij = 0 for flagged j; every flagged row becomes the
 * identity row with b_i = g_i.  A must be square (built from (map, map)); b a scalar Dat on its
 * rows.  is_bc: device uint8[nrows] (non-zero = boundary).  g: device double[nrows], or NULL for
 * g = 0.  One thread per row; deterministic.  Enqueued on the context stream. */
fe_status fe_dirichlet_apply(fe_ctx *ctx, fe_mat *A, fe_dat *b, const uint8_t *is_bc, const double *g);

/* ---------------------------------------------------------------- explicit wave steps
 * nsteps steps of the linear wave scheme of Sec. 6.3 on a P1 space (triangles or tetrahedra), in
 * place on phi and p (scalar Dats on map's target): at t = t0 + k dt, phi -= dt/2 p;
 * p += dt (K phi) / m with K phi the action of k (FE_FORM_LAPLACE, degree 1, FE_PREC_FP64 or
 * FE_PREC_F32X2) and m the lumped mass (device double[nrows], the linear form v dx, e.g. from
 * fe_assemble_vec with f = 1); p = sin(10 pi t) on the nodes flagged in is_bc (device uint8[nrows],
 * or NULL for none); phi -= dt/2 p.  The second half step of one time step and the first of the
 * next are merged, so a time step is two launches: the pull action's element kernel, then one
 * thread per node summing its staged contributions in fixed order and applying all pointwise
 * updates (deterministic).  sp: the sparsity built from (map, map) (its row incidence).
 * Errors: FE_EUNSUPPORTED (element, form, precision), FE_EINVAL, FE_ENOMEM, FE_ECUDA. */
fe_status fe_wave_steps(fe_ctx *ctx, fe_kernel *k, fe_set *cells, fe_dat *phi, fe_dat *p, const double *mass,
                        const uint8_t *is_bc, fe_map *map, fe_dat *coords, fe_map *coord_map, const fe_sparsity *sp,
                        double t0, double dt, int nsteps);

/* ---------------------------------------------------------------- batched Jacobi-CG
 * Conjugate gradients with the Jacobi preconditioner M = diag(A) (the Poisson experiment of
 * Sec. 6.2 solves with CG) for many independent SPD CSR systems at once: every fe_cg_iterate runs
 * `iters` iterations of all added, unfinished systems with two persistent launches per iteration
 * (captured once into a CUDA graph when use_graph != 0, replayed on the context stream).  Dot
 * products are FP64 sums over fixed tiles added in tile order (Globals with SUM access,
 * Sec. 4.4.2).  A tile is 512 rows, or for a system larger than 512 rows per resident block its
 * rows split evenly over those blocks; the tiling depends only on the system and the device, so a
 * system's iterates are bitwise the same alone or beside others.  The
 * products q = A p follow from the SpMV w = A z and q = w + beta q_old (algebraically equal to the
 * textbook order).  Stopping test after every iteration: ||r||_2 <= rtol ||b||_2, or maxit
 * iterations.  fe_cg_add copies A's values into the engine's sliced layout (SELL-32: slices of 32
 * rows stored column by column; later changes to A are not seen), reads b, and updates x
 * (initial guess on entry, iterate after each call) in place; A, b and x must stay alive until
 * fe_cg_remove.  fe_cg_poll
 * synchronises the context stream and reports, for slots 0..nslots-1: status (FE_CG_* below,
 * -1 for a free slot), iterations, ||r|| and ||b||.  fe_cg_remove synchronises, then frees the
 * slot's vectors.  Errors: FE_EINVAL (no free slot, bad sizes), FE_ENOMEM, FE_ECUDA. */
#define FE_CG_RUNNING 0
#define FE_CG_CONVERGED 1
#define FE_CG_MAXIT 2
#define FE_CG_BREAKDOWN 3   /* a diagonal entry or p.Ap not positive: A is not SPD */
typedef struct fe_cg fe_cg;
fe_status fe_cg_create(fe_ctx *ctx, int max_systems, fe_cg **out);
fe_status fe_cg_add(fe_cg *cg, fe_mat *A, fe_dat *b, fe_dat *x, double rtol, int maxit, int *slot);
fe_status fe_cg_iterate(fe_cg *cg, int iters, int use_graph);
fe_status fe_cg_poll(fe_cg *cg, int nslots, int *status, int *iters, double *rnorm, double *bnorm);
fe_status fe_cg_remove(fe_cg *cg, int slot);
fe_status fe_cg_destroy(fe_cg *cg);

/* ---------------------------------------------------------------- serving
 * A request loop for Poisson solves on triangle meshes: -lap u = f, u = 0 on the flagged nodes;
 * a = inner(grad u, grad v) dx and L = f v dx (f given by its P_p nodal values) assembled with the
 * deterministic pull strategy, Dirichlet elimination, then Jacobi-CG.  fe_server_run processes
 * every submitted request: it admits requests in arrival order (arrival_s seconds after the call
 * starts) while fewer than max_active are iterating and the request's worst-case device footprint
 * fits beside what is held within hbm_budget; it advances all admitted systems together
 * (iters_per_tick CG iterations between status polls); a converged system's solution is copied to
 * x_out and all its device memory is freed at once.  Each tick is launched without waiting, and
 * requests that arrived meanwhile are admitted on a second stream while it runs.  Systems too large
 * for one wave of 512-row CG tiles iterate in a second engine on a high-priority stream that uses
 * 15/16 of the resident blocks, so the smaller systems run beside them.  The server creates its
 * own streams; the context's stream orders nothing inside fe_server_run.  A request whose footprint alone exceeds the
 * budget is refused.  max_active = 1 gives the plain one-request-at-a-time path with the same
 * kernels.  Host arrays of a request must stay valid until fe_server_run returns.  Device memory
 * comes from the server's own stream-ordered CUDA memory pool on the context's device (kept up to
 * hbm_budget bytes between requests) and is counted exactly (fe_server_stats). */
#define FE_SOLVE_PENDING 0
#define FE_SOLVE_CONVERGED 1
#define FE_SOLVE_MAXIT 2
#define FE_SOLVE_BREAKDOWN 3
#define FE_SOLVE_REFUSED 4
typedef struct fe_server fe_server;
typedef struct {
  size_t hbm_budget;       /* bytes the server may hold on the device at once (its own tables included) */
  int max_active;          /* systems iterating together; 1 = one request at a time                   */
  int iters_per_tick;      /* CG iterations between status polls                                        */
  double rtol;             /* relative residual tolerance                                               */
  int maxit;
  int precision;           /* element tensors: FE_PREC_FP64 or FE_PREC_F32X2                            */
} fe_server_config;
typedef struct {
  int degree;              /* 1 or 2                                                                    */
  int64_t ncell, nnodes, nvert;
  const int32_t *cell_node;   /* host [ncell][(p+1)(p+2)/2]                                             */
  const int32_t *cell_vertex; /* host [ncell][3]                                                        */
  const double *coords;       /* host [nvert][2]                                                        */
  const double *f;            /* host [nnodes] nodal values of the source                               */
  const uint8_t *is_bc;       /* host [nnodes], non-zero on the Dirichlet boundary                      */
  double *x_out;              /* host [nnodes], the solution on completion                              */
  double arrival_s;           /* seconds after fe_server_run starts                                     */
  uint64_t mesh_key;          /* 0, or a key the caller gives every request on the same mesh (same maps,
                                 coordinates, degree and boundary flags): such requests share one device
                                 copy of the mesh and its sparsity, kept across requests and evicted,
                                 least recently used first, when admission needs the memory          */
} fe_solve_request;
typedef struct {
  int status;              /* FE_SOLVE_*                                                                */
  int iters;
  double rnorm, bnorm;
  double admitted_s, finished_s;   /* seconds after fe_server_run started                               */
  size_t bytes;            /* device bytes held while the request was iterating                         */
  size_t estimate;         /* worst-case footprint charged at admission (bounds the bytes held while built) */
} fe_solve_result;
typedef struct {
  size_t peak_bytes, live_bytes, base_bytes;
  int submitted, converged, refused, estimate_misses;
  double run_s;
  int64_t cg_launches;     /* kernels the CG engine launched (set-up, iterations, polls)                 */
  double admit_s, tick_s, retire_s;  /* host time spent admitting, iterating (launch + poll), retiring  */
  int cache_hits, cache_misses, cache_evictions;  /* requests whose mesh was cached / built and cached;
                                                      cached meshes freed to make room            */
  int sparsity_builds;     /* sparsity builds run (one per mesh built, none on a cache hit)              */
  size_t cache_bytes;      /* device bytes held by cached meshes at the end of the run                  */
} fe_server_stats;
fe_status fe_server_create(fe_ctx *ctx, const fe_server_config *cfg, fe_server **out);
fe_status fe_server_submit(fe_server *srv, const fe_solve_request *req, int64_t *id);
fe_status fe_server_run(fe_server *srv);
fe_status fe_server_result(const fe_server *srv, int64_t id, fe_solve_result *out);
fe_status fe_server_stats_get(const fe_server *srv, fe_server_stats *out);
fe_status fe_server_destroy(fe_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* FE_H */
