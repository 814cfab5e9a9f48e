// Sparsity build that allocates no device memory: the same device kernels as fe_sparsity_build,
// with their scratch taken from one file-scope static device array instead of the allocator.
//
// It serves callers that must not allocate device memory themselves: code whose device memory
// is a budget owned by another runtime (an arena or pool that stray cudaMalloc calls would bypass
// or overrun), and code that cannot afford cudaMalloc's latency and device-wide synchronisation
// where it builds patterns.
//
// The array (kScratchBytes, about 23 MB) is part of the module and stays resident on every device
// that loads the library until the process exits.  Its device address is looked up once per
// device, with that device current, on the first call made on that device; make that first call
// before any stream capture.  The address is kept until the process exits, so a cudaDeviceReset
// (which unloads the module and the array with it) ends this entry point's use on that device.
// All calls share the array and it keeps the last call's contents: everything that must start at
// zero is cleared by each call, and calls that overlap on the GPU (on different streams, or from
// several host threads) race on it.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "fe_internal.h"

namespace fe {
namespace {

constexpr int64_t kMaxRows = int64_t(1) << 18;        // rows of the pattern (target set of rmap)
constexpr int64_t kMaxInc = int64_t(1) << 20;         // cell-node incidences ncell * ndr
constexpr int64_t kMaxCandTotal = int64_t(1) << 22;   // candidates ncell * ndr * ndc

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffErr = 0;                                                        // int[4]
constexpr size_t kOffMax = align256(kOffErr + 4 * sizeof(int));                      // int[1]
constexpr size_t kOffAdjptr = align256(kOffMax + sizeof(int));                       // int64[kMaxRows+1]
constexpr size_t kOffRowcnt = align256(kOffAdjptr + (kMaxRows + 1) * sizeof(int64_t));  // int32[kMaxRows]
constexpr size_t kOffAdj = align256(kOffRowcnt + kMaxRows * sizeof(int32_t));        // int32[kMaxInc]
constexpr size_t kOffCol = align256(kOffAdj + kMaxInc * sizeof(int32_t));            // int32[kMaxCandTotal]
constexpr size_t kOffScan = align256(kOffCol + kMaxCandTotal * sizeof(int32_t));     // int64[scan blocks]
constexpr size_t kScanElems = (kMaxRows + 4095) / 4096 + 1;
constexpr size_t kScratchBytes = align256(kOffScan + kScanElems * sizeof(int64_t));

// The scratch.  Host code must not take its address directly (that is a host-side stand-in):
// the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices] = {};

thread_local char g_msg[512];

cudaError_t scratch_for_current_device(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_ptr[dev]);
  return cudaSuccess;
}

}  // namespace

const char *noalloc_message() { return g_msg; }

size_t noalloc_scratch_bytes() { return kScratchBytes; }

// Host-side flag read (pageable memcpy, synchronises the stream).
static fe_status read_flags(int *d_err, cudaStream_t s, const char *who) {
  int h[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(h, d_err, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "%s: CUDA error %d (%s)", who, (int)e, cudaGetErrorString(e));
    return FE_ECUDA;
  }
  if (h[0] & ERR_RANGE) {
    snprintf(g_msg, sizeof g_msg, "%s: a map value lies outside its target set (index %d)", who, h[1]);
    return FE_ERANGE;
  }
  if (h[0] & (ERR_ROW_TOO_LONG | ERR_CAND_OVERFLOW)) {
    snprintf(g_msg, sizeof g_msg, "%s: a row exceeds %d columns or %d candidates (row %d)", who, kMaxRowLen,
             kMaxCand, h[1]);
    return FE_EUNSUPPORTED;
  }
  if (h[0]) {
    snprintf(g_msg, sizeof g_msg, "%s: device error flags 0x%x", who, h[0]);
    return FE_ECUDA;
  }
  return FE_OK;
}

fe_status sparsity_build_noalloc(const int32_t *rmap, int ndr, const int32_t *cmap, int ndc, int64_t ncell,
                                 int64_t nrows, int64_t ncols, int64_t *rowptr, int32_t *colidx,
                                 int64_t colidx_capacity, uint8_t *lut, int64_t *nnz_out, cudaStream_t s) {
  const char *who = "fe_sparsity_build_noalloc";
  g_msg[0] = 0;
  if (ndr < 1 || ndc < 1 || ndr > 64 || ndc > 64 || ncell < 0 || nrows < 0 || ncols < 0 || !rowptr || !nnz_out ||
      (ncell > 0 && (!rmap || !cmap || !lut)) || colidx_capacity < 0 || (colidx_capacity > 0 && !colidx)) {
    snprintf(g_msg, sizeof g_msg, "%s: bad arguments", who);
    return FE_EINVAL;
  }
  if (nrows > kMaxRows || ncell * ndr > kMaxInc || ncell * ndr * ndc > kMaxCandTotal || ncols > INT32_MAX) {
    snprintf(g_msg, sizeof g_msg,
             "%s: size beyond the static scratch (rows %lld > %lld, incidences %lld > %lld or candidates %lld > %lld); "
             "use fe_sparsity_build", who, (long long)nrows, (long long)kMaxRows, (long long)(ncell * ndr),
             (long long)kMaxInc, (long long)(ncell * ndr * ndc), (long long)kMaxCandTotal);
    return FE_EUNSUPPORTED;
  }
  unsigned char *base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "%s: cudaGetSymbolAddress failed: %s", who, cudaGetErrorString(e));
    return FE_ECUDA;
  }
  int *d_err = reinterpret_cast<int *>(base + kOffErr);
  // stand-in handles over caller buffers and the static scratch, for the shared launch code
  fe_set sfrom{kMagicSet, nullptr, ncell}, srow{kMagicSet, nullptr, nrows}, scol{kMagicSet, nullptr, ncols};
  fe_map mr{kMagicMap, nullptr, &sfrom, &srow, ndr, rmap}, mc{kMagicMap, nullptr, &sfrom, &scol, ndc, cmap};
  fe_sparsity sp;
  memset(&sp, 0, sizeof sp);
  sp.rmap = &mr;
  sp.cmap = &mc;
  sp.nrows = nrows;
  sp.ncols = ncols;
  sp.ncell = ncell;
  sp.ndr = ndr;
  sp.ndc = ndc;
  sp.rowptr = rowptr;
  sp.colidx = colidx;
  sp.lut = lut;
  sp.adjptr = reinterpret_cast<int64_t *>(base + kOffAdjptr);
  sp.adj = reinterpret_cast<int32_t *>(base + kOffAdj);
  sp.rowcnt = reinterpret_cast<int32_t *>(base + kOffRowcnt);
  sp.coltmp = reinterpret_cast<int32_t *>(base + kOffCol);
  sp.scan_tmp = reinterpret_cast<int64_t *>(base + kOffScan);
  sp.scan_tmp_elems = (int64_t)kScanElems;
  sp.d_maxcnt = reinterpret_cast<int *>(base + kOffMax);
  // 1. clear the flags, incidence (validates rmap), longest incidence list, cmap range check
  e = launch_zero_i32(d_err, 4, s);
  if (e == cudaSuccess) e = sparsity_incidence(&sp, s, d_err);
  if (e == cudaSuccess && ncell > 0) e = launch_map_validate(cmap, ncell * ndc, ncols, d_err, s);
  int maxcnt = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&maxcnt, sp.d_maxcnt, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "%s: CUDA error %d (%s)", who, (int)e, cudaGetErrorString(e));
    return FE_ECUDA;
  }
  fe_status st = read_flags(d_err, s, who);
  if (st != FE_OK) return st;
  const int64_t maxcand = (int64_t)maxcnt * ndc;
  if (maxcand > kMaxCand) {
    snprintf(g_msg, sizeof g_msg, "%s: a row has %lld candidate entries (limit %d)", who, (long long)maxcand, kMaxCand);
    return FE_EUNSUPPORTED;
  }
  sp.cap = 32;
  while (sp.cap < maxcand) sp.cap <<= 1;
  sp.acap = 4;
  while (sp.acap < maxcnt) sp.acap += 4;
  // 2. rows: lookup table, unique columns, rowptr
  int64_t nnz = 0;
  e = sparsity_rows(&sp, s, d_err);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz, rowptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "%s: CUDA error %d (%s)", who, (int)e, cudaGetErrorString(e));
    return FE_ECUDA;
  }
  st = read_flags(d_err, s, who);
  if (st != FE_OK) return st;
  *nnz_out = nnz;
  if (!colidx) return FE_OK;  // size query: rowptr and lut are written, colidx is not
  if (nnz > colidx_capacity) {
    snprintf(g_msg, sizeof g_msg, "%s: colidx holds %lld entries, the pattern has %lld", who,
             (long long)colidx_capacity, (long long)nnz);
    return FE_EINVAL;
  }
  // 3. unique columns into colidx
  sp.nnz = nnz;
  e = sparsity_compact(&sp, s, d_err, 0);
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "%s: CUDA error %d (%s)", who, (int)e, cudaGetErrorString(e));
    return FE_ECUDA;
  }
  return read_flags(d_err, s, who);
}

}  // namespace fe
