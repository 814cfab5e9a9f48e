// Sparsity construction on the device (Sec. 4.4.3: a Mat is built from a pair of Maps; its
// pattern is the union over cells e of {(rmap(e)[i], cmap(e)[j])}), plus the per-cell lookup
// table that replaces the column search of MatSetValues, the row -> (cell, local index)
// incidence used by the row-owner kernels, a device-wide scan and small fill kernels.
//
// Everything is row-centric and deterministic: each row's incidence list is sorted, its
// candidate columns are sorted with a warp bitonic network in shared memory, duplicates are
// dropped, and ranks are written to the lookup table.  The CSR result is bitwise identical
// to a sort-unique of the pair set regardless of the atomics' ordering in the incidence fill.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fe_internal.h"

namespace fe {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096 items per block

__device__ __forceinline__ void flag(int *err, int bit, int64_t idx) {
  if (atomicOr(err, bit) == 0) err[1] = (int)idx;
}

// block-wide inclusive scan of one int64 per thread (kScanThreads threads); returns the
// inclusive prefix of this thread and the block total through *total.
__device__ __forceinline__ int64_t block_scan_incl(int64_t v, int64_t *total) {
  __shared__ int64_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_sums[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = w;
  }
  __syncthreads();
  int64_t off = wid > 0 ? warp_sums[wid - 1] : 0;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return v + off;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t *__restrict__ in, int64_t n,
                                                               int64_t *__restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++)
    if (base + k < n) s += in[base + k];
  int64_t tot;
  block_scan_incl(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: exclusive scan of the block sums in place (any count, chunked)
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t *bsum, int64_t nb) {
  int64_t carry = 0;
  for (int64_t c = 0; c < nb; c += kScanThreads) {
    int64_t i = c + threadIdx.x;
    int64_t v = i < nb ? bsum[i] : 0, tot;
    int64_t incl = block_scan_incl(v, &tot);
    if (i < nb) bsum[i] = carry + incl - v;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int32_t *__restrict__ in, int64_t n,
                                                              const int64_t *__restrict__ bsum,
                                                              int64_t *__restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  int64_t tot;
  int64_t run = block_scan_incl(s, &tot) - s + bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  // the thread holding item n-1 writes the total
  if (n > 0 && base <= n - 1 && n - 1 < base + kScanItems) out[n] = run;
}

__global__ void k_map_validate(const int32_t *__restrict__ v, int64_t n, int64_t limit, int *err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = v[i];
    if (x < 0 || x >= limit) flag(err, ERR_RANGE, i);
  }
}

__global__ void k_zero_i32(int32_t *p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0;
}

__global__ void k_zero_i64(int64_t *p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0;
}

__global__ void k_zero_f64(double *__restrict__ p, int64_t n) {
  // 16-byte stores for the aligned body, scalar head/tail
  int64_t head = ((16 - ((uintptr_t)p & 15)) & 15) / 8;
  if (head > n) head = n;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  if (t < head) p[t] = 0.0;
  double2 *q = reinterpret_cast<double2 *>(p + head);
  int64_t nq = (n - head) / 2;
  for (int64_t i = t; i < nq; i += st) q[i] = make_double2(0.0, 0.0);
  int64_t tail = head + 2 * nq;
  if (t == 0 && tail < n) p[tail] = 0.0;
}

// incidence counts: rowcnt[r] = #(e, i) with rmap(e)[i] = r
__global__ void k_inc_count(const int32_t *__restrict__ rmap, int64_t n, int64_t nrows, int32_t *cnt, int *err) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = rmap[k];
    if (r < 0 || r >= nrows) {
      flag(err, ERR_RANGE, k);
      continue;
    }
    atomicAdd(&cnt[r], 1);
  }
}

__global__ void k_max_count(const int32_t *__restrict__ cnt, int64_t n, int *out) {
  int m = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    m = max(m, cnt[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// incidence fill: adj[adjptr[r] + slot] = k (k = e*ndr + i); slot order is arbitrary here and
// made canonical by the row sort.
__global__ void k_inc_fill(const int32_t *__restrict__ rmap, int64_t n, int64_t nrows,
                           const int64_t *__restrict__ adjptr, int32_t *cursor, int32_t *__restrict__ adj) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = rmap[k];
    if (r < 0 || r >= nrows) continue;
    int slot = atomicAdd(&cursor[r], 1);
    adj[adjptr[r] + slot] = (int32_t)k;
  }
}

__device__ __forceinline__ void warp_bitonic_sort(uint64_t *s, int P) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < (P >> 1); t += 32) {
        int lo = 2 * j * (t / j) + (t % j), hi = lo + j;
        bool up = (lo & k) == 0;
        uint64_t a = s[lo], b = s[hi];
        if ((a > b) == up) {
          s[lo] = b;
          s[hi] = a;
        }
      }
      __syncwarp();
    }
  }
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 2;
  while (p < x) p <<= 1;
  return p;
}

// One warp per row.  Shared memory per warp: cap uint64 keys.
//  1. sort the row's incidence list (e*ndr+i ascending) and write it back
//  2. candidates key = (col << 20) | (a*ndc + j), sort
//  3. unique columns -> coltmp[adjptr[r]*ndc + rank]; ranks -> lut[(adj[a])*ndc + j]
//  4. rowcnt[r] = number of unique columns
__global__ void k_rows_sort(int64_t nrows, int ndr, int ndc, const int32_t *__restrict__ cmap,
                            const int64_t *__restrict__ adjptr, int32_t *__restrict__ adj,
                            int32_t *__restrict__ rowlen, int32_t *__restrict__ coltmp,
                            uint8_t *__restrict__ lut, int cap, int *err) {
  extern __shared__ uint64_t smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  uint64_t *s = smem + (size_t)wid * cap;
  for (int64_t r = (int64_t)blockIdx.x * wpb + wid; r < nrows; r += (int64_t)gridDim.x * wpb) {
    const int64_t a0 = adjptr[r];
    const int na = (int)(adjptr[r + 1] - a0);
    const int ncand = na * ndc;
    if (ncand > cap || na > (1 << 20) / (ndc > 0 ? ndc : 1)) {
      if (lane == 0) flag(err, ERR_CAND_OVERFLOW, r);
      if (lane == 0) rowlen[r] = 0;
      continue;
    }
    if (na == 0) {
      if (lane == 0) rowlen[r] = 0;
      continue;
    }
    // 1. canonical incidence order
    int Pa = next_pow2(na);
    for (int t = lane; t < Pa; t += 32) s[t] = t < na ? (uint64_t)(uint32_t)adj[a0 + t] : ~0ull;
    __syncwarp();
    warp_bitonic_sort(s, Pa);
    for (int t = lane; t < na; t += 32) adj[a0 + t] = (int32_t)(uint32_t)s[t];
    __syncwarp();
    // 2. candidates
    int P = next_pow2(ncand);
    for (int t = lane; t < P; t += 32) {
      uint64_t key = ~0ull;
      if (t < ncand) {
        int a = t / ndc, j = t - a * ndc;
        int32_t k = adj[a0 + a];
        int64_t e = k / ndr;
        uint32_t col = (uint32_t)cmap[e * ndc + j];
        key = ((uint64_t)col << 20) | (uint64_t)t;
      }
      s[t] = key;
    }
    __syncwarp();
    warp_bitonic_sort(s, P);
    // 3. ranks
    int carry = 0;
    for (int c0 = 0; c0 < ncand; c0 += 32) {
      int t = c0 + lane;
      uint64_t key = t < ncand ? s[t] : ~0ull;
      uint32_t col = (uint32_t)(key >> 20);
      bool head = false;
      if (t < ncand) head = (t == 0) || ((uint32_t)(s[t - 1] >> 20) != col);
      unsigned hm = __ballot_sync(0xffffffffu, head);
      int rank = carry + __popc(hm & ((2u << lane) - 1u)) - 1;
      if (t < ncand) {
        int orig = (int)(key & 0xFFFFFu);
        int a = orig / ndc, j = orig - a * ndc;
        if (rank < kMaxRowLen) lut[(int64_t)adj[a0 + a] * ndc + j] = (uint8_t)rank;
        if (head) coltmp[a0 * ndc + rank] = (int32_t)col;
      }
      carry += __popc(hm);
    }
    if (lane == 0) {
      rowlen[r] = carry;
      if (carry > kMaxRowLen) flag(err, ERR_ROW_TOO_LONG, r);
    }
    __syncwarp();
  }
}

// warp per row: colidx[rowptr[r] + k] = coltmp[adjptr[r]*ndc + k]; guarded against a pattern that
// grew beyond the allocated nnz (rebuild with different maps).
__global__ void k_rows_compact(int64_t nrows, int ndc, const int64_t *__restrict__ adjptr,
                               const int64_t *__restrict__ rowptr, const int32_t *__restrict__ coltmp,
                               int32_t *__restrict__ colidx, int64_t nnz_cap, int check_nnz, int *err) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  if (check_nnz && blockIdx.x == 0 && threadIdx.x == 0 && rowptr[nrows] != nnz_cap) flag(err, ERR_NNZ_CHANGED, nrows);
  for (int64_t r = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); r < nrows; r += (int64_t)gridDim.x * wpb) {
    int64_t b = rowptr[r], n = rowptr[r + 1] - b, src = adjptr[r] * ndc;
    if (b + n > nnz_cap) continue;
    for (int64_t k = lane; k < n; k += 32) colidx[b + k] = coltmp[src + k];
  }
}

int grid_for(int64_t n, int threads, int max_blocks = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

}  // namespace

int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) {  // n == 0: out[0] = 0
    k_zero_i64<<<1, 32, 0, s>>>(out, 1);
    return cudaGetLastError();
  }
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
  k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp, nb);
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp, out);
  return cudaGetLastError();
}

cudaError_t launch_map_validate(const int32_t *v, int64_t n, int64_t limit, int *err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_map_validate<<<grid_for(n, 256), 256, 0, s>>>(v, n, limit, err);
  return cudaGetLastError();
}

cudaError_t launch_zero_f64(double *p, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_zero_f64<<<grid_for((n + 1) / 2, 256, 152 * 8), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

cudaError_t sparsity_incidence(fe_sparsity *sp, cudaStream_t s, int *err) {
  const int64_t n = sp->ncell * sp->ndr;
  k_zero_i32<<<grid_for(sp->nrows, 256), 256, 0, s>>>(sp->rowcnt, sp->nrows);
  if (n > 0) k_inc_count<<<grid_for(n, 256), 256, 0, s>>>(sp->rmap->values, n, sp->nrows, sp->rowcnt, err);
  k_zero_i32<<<1, 32, 0, s>>>(sp->d_maxcnt, 1);
  if (sp->nrows > 0) k_max_count<<<grid_for(sp->nrows, 256, 152 * 4), 256, 0, s>>>(sp->rowcnt, sp->nrows, sp->d_maxcnt);
  cudaError_t e = exclusive_scan_i32_to_i64(sp->rowcnt, sp->adjptr, sp->nrows, sp->scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_zero_i32<<<grid_for(sp->nrows, 256), 256, 0, s>>>(sp->rowcnt, sp->nrows);
  if (n > 0)
    k_inc_fill<<<grid_for(n, 256), 256, 0, s>>>(sp->rmap->values, n, sp->nrows, sp->adjptr, sp->rowcnt, sp->adj);
  return cudaGetLastError();
}

cudaError_t sparsity_rows(fe_sparsity *sp, cudaStream_t s, int *err) {
  const int warps = 4;
  size_t smem = (size_t)warps * sp->cap * sizeof(uint64_t);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_rows_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (sp->nrows > 0)
    k_rows_sort<<<grid_for(sp->nrows, warps, 152 * 32), warps * 32, smem, s>>>(
        sp->nrows, sp->ndr, sp->ndc, sp->cmap->values, sp->adjptr, sp->adj, sp->rowcnt, sp->coltmp, sp->lut,
        sp->cap, err);
  return exclusive_scan_i32_to_i64(sp->rowcnt, sp->rowptr, sp->nrows, sp->scan_tmp, s);
}

cudaError_t sparsity_compact(fe_sparsity *sp, cudaStream_t s, int *err, int check_nnz) {
  const int warps = 8;
  if (sp->nrows > 0)
    k_rows_compact<<<grid_for(sp->nrows, warps, 152 * 16), warps * 32, 0, s>>>(
        sp->nrows, sp->ndc, sp->adjptr, sp->rowptr, sp->coltmp, sp->colidx, sp->nnz, check_nnz, err);
  return cudaGetLastError();
}

}  // namespace fe
