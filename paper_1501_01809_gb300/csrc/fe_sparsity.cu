// Sparsity construction on the device (Sec. 4.4.3: a Mat is built from a pair of Maps; its
// pattern is the union over cells e of {(rmap(e)[i], cmap(e)[j])}), plus the per-cell lookup
// table that replaces the column search of MatSetValues, the row -> (cell, local index)
// incidence used by the row-owner kernels, a device-wide scan and small fill kernels.
//
// Everything is row-centric and deterministic: each row's candidate columns are deduplicated by a
// warp sort of packed keys (or, for rows of more than 256 candidates, in a shared-memory hash
// table), the unique columns are ranked, and the ranks go to the lookup table.  The CSR result is
// bitwise identical to a sort-unique of the pair set whatever the ordering of the atomics in the
// incidence fill.  The incidence lists themselves stay in fill order until a row-owner kernel
// needs a fixed order (sparsity_canonical).
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
                                                               int64_t *__restrict__ bsum, const int *gate) {
  if (gate && *gate == 0) return;
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
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t *bsum, int64_t nb, const int *gate) {
  if (gate && *gate == 0) return;
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
                                                              int64_t *__restrict__ out, const int *gate) {
  if (gate && *gate == 0) return;
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

__global__ void k_zero_i32(int32_t *p, int64_t n, const int *gate = nullptr) {
  if (gate && *gate == 0) return;
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
__global__ void k_inc_count(const int32_t *__restrict__ rmap, int64_t n, int64_t nrows, int32_t *cnt, int *err,
                            const int *gate = nullptr) {
  if (gate && *gate == 0) return;
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
// made canonical by sparsity_canonical when an order-sensitive kernel needs it.
// Each thread takes four incidences per round and issues their four cursor atomics before it
// needs any result, so that the round trips of the returning atomics overlap.  Launched with one
// round per thread (up to 152 * 256 blocks), so that blocks start as SMs free up.  guarded (a rebuild
// filling against the previous row offsets): a slot past the row's previous length is not written
// (the row pass then sees the changed count), and a map value out of range is flagged.
__global__ void k_inc_fill(const int32_t *__restrict__ rmap, int64_t n, int64_t nrows,
                           const int64_t *__restrict__ adjptr, int32_t *cursor, int32_t *__restrict__ adj,
                           int guarded = 0, int *err = nullptr, const int *gate = nullptr) {
  if (gate && *gate == 0) return;
  constexpr int U = 4;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k0 < n; k0 += U * st) {
    int32_t r[U];
    int slot[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t k = k0 + u * st;
      r[u] = k < n ? rmap[k] : -1;
    }
#pragma unroll
    for (int u = 0; u < U; u++) slot[u] = (r[u] >= 0 && r[u] < nrows) ? atomicAdd(&cursor[r[u]], 1) : 0;
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (r[u] >= 0 && r[u] < nrows) {
        const int64_t b = adjptr[r[u]];
        if (!guarded || b + slot[u] < adjptr[r[u] + 1]) adj[b + slot[u]] = (int32_t)(k0 + u * st);
      } else if (guarded && k0 + u * st < n) {
        flag(err, ERR_RANGE, k0 + u * st);
      }
    }
  }
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

__device__ __forceinline__ uint32_t hash_slot(uint32_t key, int logH) { return (key * 2654435761u) >> (32 - logH); }

// For distinct values v[0..n) in shared memory (v 16-byte aligned), rank[q] = #{s : v[s] < v[q]},
// written for q = lane, lane + 32, ...: one pass of broadcast 16-byte loads per round of 32.
template <class F>
__device__ __forceinline__ void warp_rank_distinct(const uint32_t *v, int n, F &&sink) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < n; base += 32) {
    const int q = base + lane;
    const uint32_t mine = q < n ? v[q] : 0xFFFFFFFFu;
    int cnt = 0, s = 0;
    for (; s + 4 <= n; s += 4) {
      const uint4 w = *reinterpret_cast<const uint4 *>(v + s);
      cnt += (w.x < mine) + (w.y < mine) + (w.z < mine) + (w.w < mine);
    }
    for (; s < n; s++) cnt += v[s] < mine;
    if (q < n) sink(q, cnt);
  }
}


// lower ? min(v, o) : max(v, o) as two predicated instructions (the lanes of one stage split
// between them) instead of a minimum, a maximum and a select.
__device__ __forceinline__ uint32_t keep_min_or_max(uint32_t v, uint32_t o, bool lower) {
  asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p min.u32 %0, %0, %1;\n\t@!p max.u32 %0, %0, %1;\n\t}"
      : "+r"(v)
      : "r"(o), "r"((uint32_t)lower));
  return v;
}

// Bitonic sort of 32 E packed 32-bit values across a warp, ascending: lane l holds elements
// E l .. E l + E - 1 in v[0..E).  Each merge of size k starts with a mirror stage (element i against
// i ^ (k - 1)), after which every half-cleaner stage sorts ascending, so compare-exchanges inside a
// lane need no direction select.  Stages between lanes exchange with lane l ^ (stride / E); the lane
// holding the lower index keeps the minimum.
// NL = 16 (or 8) sorts NL E values in each group of NL lanes independently (every exchange mask
// is below NL).
template <int E, int NL = 32>
__device__ __forceinline__ void warp_bitonic_packed(uint32_t (&v)[E]) {
  const int lane = threadIdx.x & 31;
  constexpr int LG = E == 1 ? 0 : E == 2 ? 1 : E == 4 ? 2 : E == 8 ? 3 : E == 16 ? 4 : -1;
  static_assert(LG >= 0, "E must be a power of two up to 16");
  static_assert(NL == 32 || NL == 16 || NL == 8, "a warp, a half-warp or a quarter-warp");
#pragma unroll
  for (int k = 2; k <= NL * E; k <<= 1) {
    if (k <= E) {  // mirror stage inside the lane
#pragma unroll
      for (int h = 0; h < E; h++) {
        const int ph = h ^ (k - 1);
        if (h < ph) {
          const uint32_t a = v[h], b = v[ph];
          v[h] = umin(a, b);
          v[ph] = umax(a, b);
        }
      }
    } else {  // mirror stage between lanes: element h meets the partner lane's element E - 1 - h
      const int m = (k >> LG) - 1;
      const bool lower = (lane & (k >> (LG + 1))) == 0;
      uint32_t o[E];
#pragma unroll
      for (int h = 0; h < E; h++) o[h] = __shfl_xor_sync(0xffffffffu, v[E - 1 - h], m);
#pragma unroll
      for (int h = 0; h < E; h++) v[h] = keep_min_or_max(v[h], o[h], lower);
    }
#pragma unroll
    for (int j = k >> 2; j > 0; j >>= 1) {
      if (j < E) {
#pragma unroll
        for (int h = 0; h < E; h++) {
          if ((h & j) == 0) {
            const uint32_t a = v[h], b = v[h | j];
            v[h] = umin(a, b);
            v[h | j] = umax(a, b);
          }
        }
      } else {
        const int m = j >> LG;
        const bool lower = (lane & m) == 0;
#pragma unroll
        for (int h = 0; h < E; h++) {
          const uint32_t o = __shfl_xor_sync(0xffffffffu, v[h], m);
          v[h] = keep_min_or_max(v[h], o, lower);
        }
      }
    }
  }
}

struct RowsParams {
  int64_t nrows;
  int ndr, ndc;
  const int32_t *cmap;
  const int64_t *adjptr;
  int32_t *adj;
  int32_t *rowlen;
  int32_t *coltmp;
  uint8_t *lut;
  int cap, acap;      // candidate capacity per row (power of two), incidence capacity (multiple of 4)
  uint64_t mdiv_ndr;  // floor(2^64 / ndr) + 1: exact k / ndr = __umul64hi(k, mdiv_ndr) for k < 2^32
  uint32_t mdiv_ndc;  // floor(2^32 / ndc) + 1: exact t / ndc = __umulhi(t, mdiv_ndc) for t < 2^26
  int packed_ok;      // ncols < 2^24 - 1: (column << 8 | candidate) fits 32 bits below the padding value
  int sort_only;      // every row takes the sort path: shared memory holds only the incidence lists
  int pairs;          // ndc even and cmap 8-byte aligned: the sort paths load candidates two at a time
  int lut_pairs;      // ndc even and lut 2-byte aligned: the sort paths write the table two bytes at a time
  int *err;
  // in-place rebuild pass (colidx != NULL): a row whose length equals rowptr[r+1] - rowptr[r]
  // writes its columns to colidx + rowptr[r]; any other row sets *changed
  int32_t *colidx;
  const int64_t *rowptr;
  int64_t nnz;
  int *changed;
  const int *gate;  // NULL, or a device flag: 0 = return without work
  int canon;        // also put every row's incidence list in ascending order (else it stays in fill order)
  int check_counts; // rowlen holds a guarded fill's incidence counts: a row whose count differs from its
                    // previous range sets *changed (read before the row's length overwrites it)
  int *cols_changed; // in-place pass: a column written in place that differs from the one already
                     // there sets *cols_changed (equal columns are not written again)
};

// Where row r's nu unique columns go: colidx in place when the in-place pass applies and the
// row's length is unchanged (and inside the nnz entries), else coltmp at the incidence offset.
__device__ __forceinline__ int32_t *row_out(const RowsParams &p, int64_t r, int64_t a0, int nu,
                                            bool leader = (threadIdx.x & 31) == 0) {
  if (p.colidx) {
    const int64_t b = p.rowptr[r];
    if (p.rowptr[r + 1] - b == nu && b >= 0 && b + nu <= p.nnz) return p.colidx + b;
    if (leader) *p.changed = 1;
  }
  return p.coltmp + a0 * p.ndc;
}

// Column k of a row whose columns go to outc.  With TRACK, in place (the row kept its length in an
// in-place pass) the column is compared with the one already there and written only when it
// differs, which also records that the pattern changed; otherwise it is written.
template <bool TRACK>
__device__ __forceinline__ void put_col(const RowsParams &p, int32_t *outc, int k, int32_t col, bool in_place) {
  if (!TRACK || !in_place) {
    outc[k] = col;
  } else if (outc[k] != col) {
    outc[k] = col;
    *p.cols_changed = 1;
  }
}

__device__ __forceinline__ uint32_t div_ndr(uint32_t k, const RowsParams &p) {
  return p.ndr == 1 ? k : (uint32_t)__umul64hi((uint64_t)k, p.mdiv_ndr);
}
__device__ __forceinline__ uint32_t div_ndc(uint32_t t, const RowsParams &p) {
  return p.ndc == 1 ? t : __umulhi(t, p.mdiv_ndc);
}


// The packed keys (column << SH | candidate t) of one row's ncand candidates, E per lane of a group
// of W lanes (lane l of the group: candidates W h + l, or with p.pairs 2 (W h' + l) and the next,
// both of one incidence, from one 8-byte load); slots past ncand hold the padding value.  Candidate
// t = (a, j) is column j of incidence a, whose cell is adje[a].
template <int E, int SH, int W>
__device__ __forceinline__ void load_keys(const RowsParams &p, int l, int ncand, const uint32_t *adje,
                                          uint32_t (&key)[E]) {
  const int ndc = p.ndc;
  if (p.pairs) {
#pragma unroll
    for (int hp = 0; hp < E / 2; hp++) {
      const uint32_t t = 2u * (uint32_t)(W * hp + l);  // ncand is even: t < ncand covers t + 1
      key[2 * hp] = key[2 * hp + 1] = 0xFFFFFFFFu;
      if ((int)t < ncand) {
        const uint32_t a = div_ndc(t, p), j = t - a * (uint32_t)ndc;
        const int2 c = *reinterpret_cast<const int2 *>(p.cmap + (int64_t)adje[a] * ndc + j);
        key[2 * hp] = ((uint32_t)c.x << SH) | t;
        key[2 * hp + 1] = ((uint32_t)c.y << SH) | (t + 1);
      }
    }
  } else {
#pragma unroll
    for (int h = 0; h < E; h++) {
      const uint32_t t = (uint32_t)(W * h + l);
      key[h] = 0xFFFFFFFFu;
      if ((int)t < ncand) {
        const uint32_t a = div_ndc(t, p), j = t - a * (uint32_t)ndc;
        key[h] = ((uint32_t)p.cmap[(int64_t)adje[a] * ndc + j] << SH) | t;
      }
    }
  }
}

// lut[(adjs[a]) ndc + j] = lbuf[t] for the row's candidates t = (a, j), lane l of a group of W
// taking t = l, l + W, ... (with p.lut_pairs: the pairs 2 q, 2 q + 1 of one incidence, q = l, l + W,
// ..., as one 2-byte store).
template <int W>
__device__ __forceinline__ void store_lut(const RowsParams &p, int l, int ncand, const uint32_t *adjs,
                                          const uint8_t *lbuf) {
  const int ndc = p.ndc;
  if (p.lut_pairs) {
    for (int q = l; 2 * q < ncand; q += W) {
      const uint32_t t = 2u * (uint32_t)q, a = div_ndc(t, p), j = t - a * (uint32_t)ndc;
      *reinterpret_cast<uint16_t *>(p.lut + (int64_t)adjs[a] * ndc + j) = *reinterpret_cast<const uint16_t *>(lbuf + t);
    }
  } else {
    for (int t = l; t < ncand; t += W) {
      const uint32_t a = div_ndc((uint32_t)t, p), j = (uint32_t)t - a * (uint32_t)ndc;
      p.lut[(int64_t)adjs[a] * ndc + j] = lbuf[t];
    }
  }
}

// One row by sorting packed (column << SH | candidate) values, E per lane (32 E >= ncand, na <= 32):
// the incidence list (ranked into ascending order when p.canon), candidates, sort, first element
// of each run of equal columns, ranks
// by a warp prefix count, unique columns (ascending) to coltmp and every candidate's rank to the
// lookup table.  Returns the number of unique columns (valid in every lane).
// adje (na words) and lbuf (256 bytes) are per-warp shared scratch: the cell of each incidence, and
// each candidate's rank, which the warp then writes to the lookup table incidence by incidence.
template <int E, int SH, bool TRACK>
__device__ __forceinline__ int row_by_sort(const RowsParams &p, int64_t r, int64_t a0, int na, int ncand,
                                           uint32_t *adjs, uint32_t *adje, uint8_t *lbuf) {
  const int lane = threadIdx.x & 31;
  const int ndc = p.ndc;
  const uint32_t tmask = (1u << SH) - 1u;
  // 1. the row's incidences (in ascending order by rank when canonicalising)
  const uint32_t v = lane < na ? (uint32_t)p.adj[a0 + lane] : 0xFFFFFFFFu;
  int rk = lane;
  if (p.canon) {
    rk = 0;
    for (int q = 0; q < na; q++) rk += __shfl_sync(0xffffffffu, v, q) < v;
  }
  if (lane < na) {
    adjs[rk] = v;
    adje[rk] = div_ndr(v, p);  // the incidence's cell, once per incidence
    if (p.canon) p.adj[a0 + rk] = (int32_t)v;
  }
  __syncwarp();
  // 2. candidates t = 32 h + lane (consecutive lanes read consecutive map entries), packed
  //    (column << SH | t); padding sorts last.  The sort does not depend on the starting slots.
  uint32_t key[E];
  load_keys<E, SH, 32>(p, lane, ncand, adje, key);
  warp_bitonic_packed<E>(key);
  // 3. first element of each run of equal columns, ranks by a warp prefix count
  const uint32_t prev = __shfl_up_sync(0xffffffffu, key[E - 1], 1);
  int f[E], c = 0;
#pragma unroll
  for (int h = 0; h < E; h++) {
    const uint32_t before = h == 0 ? prev : key[h - 1];
    f[h] = key[h] != 0xFFFFFFFFu && ((h == 0 && lane == 0) || (key[h] >> SH) != (before >> SH));
    c += f[h];
  }
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  const int nu = __shfl_sync(0xffffffffu, incl, 31);
  int32_t *outc = row_out(p, r, a0, nu);
  const bool in_place = TRACK && outc != p.coltmp + a0 * ndc;
  int rank = incl - c - 1;  // rank of the run before this lane's first element
#pragma unroll
  for (int h = 0; h < E; h++) {
    rank += f[h];
    if (key[h] == 0xFFFFFFFFu) continue;
    if (f[h]) put_col<TRACK>(p, outc, rank, (int32_t)(key[h] >> SH), in_place);
    lbuf[key[h] & tmask] = (uint8_t)rank;  // ranks past the row limit are flagged by the caller
  }
  __syncwarp();
  // the lookup table in incidence order: candidate t = (a, j) goes to row a's ndc bytes, so the
  // lanes of one store write a few contiguous segments instead of one byte per segment each
  store_lut<32>(p, lane, ncand, adjs, lbuf);
  __syncwarp();
  return nu;
}

// Up to 32 / NL rows at once, one per group of NL lanes: the steps of row_by_sort inside each
// group (E keys per lane, at most NL E candidates and NL incidences per row).  Every shuffle has
// width NL, so the groups never exchange values; adjs, adje (NL words) and lbuf (NL E bytes) are
// this group's scratch.  A group without a row (r < 0, na = ncand = 0) takes part in the warp-wide
// steps with padding keys only and writes nothing.  Returns this group's number of unique columns.
template <int E, int SH, int NL, bool TRACK>
__device__ __forceinline__ int row_by_sort_group(const RowsParams &p, int64_t r, int64_t a0, int na, int ncand,
                                                 uint32_t *adjs, uint32_t *adje, uint8_t *lbuf) {
  const int gl = threadIdx.x & (NL - 1);
  const unsigned full = 0xffffffffu;
  const int ndc = p.ndc;
  const uint32_t tmask = (1u << SH) - 1u;
  const uint32_t v = gl < na ? (uint32_t)p.adj[a0 + gl] : 0xFFFFFFFFu;
  int rk = gl;
  if (p.canon) {
    rk = 0;
    for (int q = 0; q < NL; q++) {
      const uint32_t w = __shfl_sync(full, v, q, NL);
      rk += (q < na) && (w < v);
    }
  }
  if (gl < na) {
    adjs[rk] = v;
    adje[rk] = div_ndr(v, p);
    if (p.canon) p.adj[a0 + rk] = (int32_t)v;
  }
  __syncwarp();
  uint32_t key[E];
  load_keys<E, SH, NL>(p, gl, ncand, adje, key);
  warp_bitonic_packed<E, NL>(key);
  const uint32_t prev = __shfl_up_sync(full, key[E - 1], 1, NL);
  int f[E], c = 0;
#pragma unroll
  for (int h = 0; h < E; h++) {
    const uint32_t before = h == 0 ? prev : key[h - 1];
    f[h] = key[h] != 0xFFFFFFFFu && ((h == 0 && gl == 0) || (key[h] >> SH) != (before >> SH));
    c += f[h];
  }
  int incl = c;
#pragma unroll
  for (int o = 1; o < NL; o <<= 1) {
    const int n = __shfl_up_sync(full, incl, o, NL);
    if (gl >= o) incl += n;
  }
  const int nu = __shfl_sync(full, incl, NL - 1, NL);
  if (r >= 0) {
    int32_t *outc = row_out(p, r, a0, nu, gl == 0);
    const bool in_place = TRACK && outc != p.coltmp + a0 * ndc;
    int rank = incl - c - 1;
#pragma unroll
    for (int h = 0; h < E; h++) {
      rank += f[h];
      if (key[h] == 0xFFFFFFFFu) continue;
      if (f[h]) put_col<TRACK>(p, outc, rank, (int32_t)(key[h] >> SH), in_place);
      lbuf[key[h] & tmask] = (uint8_t)rank;
    }
  }
  __syncwarp();
  store_lut<NL>(p, gl, ncand, adjs, lbuf);
  __syncwarp();
  return nu;
}

// The rows of the pattern (rows = target set of the row map), eight consecutive rows per warp at
// a time.  Rows of at most 8 incidences and 64 candidates go four at a time through
// row_by_sort_group (one per quarter-warp); other rows take the whole warp, one at a time: rows of
// at most 256 candidates and 32 incidences through row_by_sort, the others:
//  1. load the row's incidence list {e*ndr + i : rmap(e)[i] = r} (all distinct) into shared
//     memory (ranked into ascending order and written back when p.canon is set);
//  2. insert every candidate column cmap(e)[j] of every incident cell into a shared-memory hash
//     table sized to the row (deduplication), remembering each candidate's slot;
//  3. compact the unique columns (remembering their slots) and rank them by counting;
//     write them to coltmp at the row's incidence-based offset in ascending order and their
//     ranks into the table;
//  4. lut[(e*ndr + i)*ndc + j] = rank of the candidate's slot; rowlen[r] = number of unique columns.
// Shared memory per warp (32-bit words): hkey[cap], hrank[cap], ucol[cap], uslot[cap], cslot[cap],
// adju[acap], adjs[acap], then the sort paths' scratch: rank bytes (64) and the quarter-warp rows'
// incidences, cells and rank bytes (128).
// TRACK (in-place pass only): compare the columns written in place; without it the in-place pass
// sets *p.cols_changed at once (a column may have changed).
template <bool TRACK>
__global__ void __launch_bounds__(256, 5) k_rows_build(const RowsParams p) {
  extern __shared__ __align__(16) int32_t smem_i[];
  if (p.gate && *p.gate == 0) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int cap = p.cap;
  if (p.colidx && blockIdx.x == 0 && threadIdx.x == 0) {
    if (p.rowptr[p.nrows] != p.nnz) *p.changed = 1;
    if (!TRACK) *p.cols_changed = 1;
  }
  // per warp: hash tables (5 cap words) unless every row is sorted, then the incidence lists, then
  // 64 words of rank bytes for the sort path, then 128 words for the quarter-warp rows (incidences,
  // cells and rank bytes of each quarter)
  int32_t *hkey = smem_i + (size_t)wid * ((p.sort_only ? 0 : 5 * cap) + 2 * p.acap + 64 + 128);
  int32_t *hrank = hkey + cap;
  uint32_t *ucol = reinterpret_cast<uint32_t *>(hrank + cap);
  int32_t *uslot = reinterpret_cast<int32_t *>(ucol + cap);
  int32_t *cslot = uslot + cap;
  uint32_t *adju = p.sort_only ? reinterpret_cast<uint32_t *>(hkey) : reinterpret_cast<uint32_t *>(cslot + cap);
  uint32_t *adjs = adju + p.acap;
  uint8_t *lbuf = reinterpret_cast<uint8_t *>(adjs + p.acap);
  const int grp = lane >> 3;
  uint32_t *gadjs = reinterpret_cast<uint32_t *>(lbuf + 256) + 8 * grp;
  uint32_t *gadje = reinterpret_cast<uint32_t *>(lbuf + 256) + 32 + 8 * grp;
  uint8_t *glbuf = lbuf + 256 + 256 + 64 * grp;
  const int ndc = p.ndc;
  const unsigned full = 0xffffffffu;
  // Rows go to warps in chunks of 8.  The rows of at most 8 incidences and 64 candidates (every
  // edge row of a P2 tetrahedral mesh, every row of P1-P3 triangles) are sorted four at a time,
  // one per quarter-warp, eight keys per lane (four when no row of the four has more than 32
  // candidates); every other row takes the whole warp.
  for (int64_t ch = (int64_t)blockIdx.x * wpb + wid; 8 * ch < p.nrows; ch += (int64_t)gridDim.x * wpb) {
    const int64_t rb = 8 * ch;
    const int64_t rl = rb + (lane & 7);  // lanes k and k + 8, k + 16, k + 24 look at row rb + k
    int64_t al = 0;
    int nl = 0;
    if (rl < p.nrows) {
      al = p.adjptr[rl];
      nl = (int)(p.adjptr[rl + 1] - al);
    }
    if (p.check_counts) {  // the guarded fill's count against the range it was filled into
      if (lane < 8 && rl < p.nrows && p.rowlen[rl] != nl) *p.changed = 1;
      __syncwarp();
    }
    const bool small = p.packed_ok && rl < p.nrows && nl > 0 && nl <= 8 && nl * ndc <= 64;
    unsigned qmask = __ballot_sync(full, small) & 0xFFu;                     // bit k: row rb + k
    unsigned wmask = (__ballot_sync(full, rl < p.nrows) & 0xFFu) & ~qmask;  // the rows left
    while (qmask) {
      unsigned m = qmask;  // quarter g takes the (g + 1)-th remaining small row, if there is one
      for (int g = 0; g < grp; g++) m &= m - 1;
      const bool have = m != 0;
      const int k = have ? __ffs(m) - 1 : 0;
      const int na = __shfl_sync(full, nl, k);
      const int64_t a0 = __shfl_sync(full, al, k);
      const int nag = have ? na : 0;
      const int64_t r = have ? rb + k : -1;
      const bool wide = __any_sync(full, nag * ndc > 32);
      const int nu = wide ? row_by_sort_group<8, 6, 8, TRACK>(p, r, a0, nag, nag * ndc, gadjs, gadje, glbuf)
                          : row_by_sort_group<4, 6, 8, TRACK>(p, r, a0, nag, nag * ndc, gadjs, gadje, glbuf);
      if (have && (lane & 7) == 0) p.rowlen[r] = nu;  // at most 64 columns: within the row limit
      __syncwarp();
      for (int g = 0; g < 4; g++) qmask &= qmask - 1;  // the (up to) four rows just done
    }
    while (wmask) {
      const int64_t r = rb + (__ffs(wmask) - 1);
      wmask &= wmask - 1;
      const int64_t a0 = p.adjptr[r];
      const int na = (int)(p.adjptr[r + 1] - a0);
      const int ncand = na * ndc;
      if (na > p.acap || ncand > cap) {
        if (lane == 0) {
          flag(p.err, ERR_CAND_OVERFLOW, r);
          p.rowlen[r] = 0;
        }
        continue;
      }
      if (na == 0) {
        if (lane == 0) p.rowlen[r] = 0;
        continue;
      }
      if (p.packed_ok && na <= 32 && ncand <= 256) {
        // rows of up to 256 candidates (every row of P1 and P2 meshes and of P3 triangles): sort packed values
        const int nu = ncand <= 64    ? row_by_sort<2, 6, TRACK>(p, r, a0, na, ncand, adjs, adju, lbuf)
                       : ncand <= 128 ? row_by_sort<4, 7, TRACK>(p, r, a0, na, ncand, adjs, adju, lbuf)
                                      : row_by_sort<8, 8, TRACK>(p, r, a0, na, ncand, adjs, adju, lbuf);
        if (lane == 0) {
          p.rowlen[r] = nu;
          if (nu > kMaxRowLen) flag(p.err, ERR_ROW_TOO_LONG, r);
        }
        __syncwarp();
        continue;
      }
      const int H = next_pow2(ncand);  // <= cap
      int logH = 5;
      while ((1 << logH) < H) logH++;
      // 1. the row's incidences (in ascending order when canonicalising)
      for (int t = lane; t < na; t += 32) adju[t] = (uint32_t)p.adj[a0 + t];
      for (int t = lane; t < H; t += 32) hkey[t] = -1;
      __syncwarp();
      if (p.canon) {
        warp_rank_distinct(adju, na, [&](int q, int rk) { adjs[rk] = adju[q]; });
        __syncwarp();
        for (int t = lane; t < na; t += 32) p.adj[a0 + t] = (int32_t)adjs[t];
      } else {
        for (int t = lane; t < na; t += 32) adjs[t] = adju[t];
      }
      // 2. insert candidates, remember their slots
      for (int t = lane; t < ncand; t += 32) {
        const uint32_t a = div_ndc((uint32_t)t, p);
        const uint32_t j = (uint32_t)t - a * (uint32_t)ndc;
        const uint32_t e = div_ndr(adjs[a], p);
        const int32_t col = p.cmap[(int64_t)e * ndc + j];
        uint32_t h = hash_slot((uint32_t)col, logH);
        for (int q = 0; q < H; q++) {
          const int32_t prev = atomicCAS(&hkey[h], -1, col);
          if (prev == -1 || prev == col) break;
          h = (h + 1) & (H - 1);
        }
        cslot[t] = (int32_t)h;
      }
      __syncwarp();
      // 3. compact the unique columns, rank them, write them in ascending order
      int nu = 0;
      for (int b = 0; b < H; b += 32) {
        const int32_t key = hkey[b + lane];
        const unsigned m = __ballot_sync(0xffffffffu, key >= 0);
        if (key >= 0) {
          const int pos = nu + __popc(m & ((1u << lane) - 1u));
          ucol[pos] = (uint32_t)key;
          uslot[pos] = b + lane;
        }
        nu += __popc(m);
      }
      __syncwarp();
      int32_t *outc = row_out(p, r, a0, nu);
      const bool in_place = TRACK && outc != p.coltmp + a0 * ndc;
      warp_rank_distinct(ucol, nu, [&](int q, int rk) {
        hrank[uslot[q]] = rk;
        put_col<TRACK>(p, outc, rk, (int32_t)ucol[q], in_place);
      });
      __syncwarp();
      // 4. rank of every candidate -> lookup table (candidate t = (a, j) of incident k = adjs[a])
      for (int t = lane; t < ncand; t += 32) {
        const uint32_t a = div_ndc((uint32_t)t, p);
        const uint32_t j = (uint32_t)t - a * (uint32_t)ndc;
        const int rank = hrank[cslot[t]];
        if (rank < kMaxRowLen) p.lut[(int64_t)adjs[a] * ndc + j] = (uint8_t)rank;
      }
      if (lane == 0) {
        p.rowlen[r] = nu;
        if (nu > kMaxRowLen) flag(p.err, ERR_ROW_TOO_LONG, r);
      }
      __syncwarp();
    }
  }
}

// One warp per 32 consecutive rows: colidx[rowptr[r] + k] = coltmp[adjptr[r]*ndc + k].  Guarded
// against a pattern that grew beyond the allocated nnz (rebuild with different maps).
__global__ void k_rows_compact(int64_t nrows, int ndc, const int64_t *__restrict__ adjptr,
                               const int64_t *__restrict__ rowptr, const int32_t *__restrict__ coltmp,
                               int32_t *__restrict__ colidx, int64_t nnz_cap, int check_nnz, int *err,
                               const int *gate) {
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  if (check_nnz && blockIdx.x == 0 && threadIdx.x == 0 && rowptr[nrows] != nnz_cap) flag(err, ERR_NNZ_CHANGED, nrows);
  for (int64_t r0 = ((int64_t)blockIdx.x * wpb + (threadIdx.x >> 5)) * 32; r0 < nrows;
       r0 += (int64_t)gridDim.x * wpb * 32) {
    const int64_t r = r0 + lane;
    long long b = 0, n = 0, src = 0;
    if (r < nrows) {
      b = rowptr[r];
      n = rowptr[r + 1] - b;
      src = adjptr[r] * ndc;
    }
    const int nq = (int)(nrows - r0 < 32 ? nrows - r0 : 32);
    for (int q = 0; q < nq; q++) {
      long long bq = __shfl_sync(0xffffffffu, b, q), cq = __shfl_sync(0xffffffffu, n, q);
      long long sq = __shfl_sync(0xffffffffu, src, q);
      if (bq + cq > nnz_cap) continue;
      for (long long k = lane; k < cq; k += 32) colidx[bq + k] = coltmp[sq + k];
    }
  }
}

// One warp per row: the row's incidence list (distinct values e*ndr+i) in ascending order, in place.
// Rows of at most 32 incidences rank in registers, longer ones through shared memory (acap words
// twice per warp; no row is longer than acap, which the row kernel has checked).
__global__ void k_adj_canon(int64_t nrows, const int64_t *__restrict__ adjptr, int32_t *__restrict__ adj, int acap) {
  extern __shared__ __align__(16) uint32_t sm_canon[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  uint32_t *u = sm_canon + (size_t)wid * 2 * acap, *o = u + acap;
  for (int64_t r = (int64_t)blockIdx.x * wpb + wid; r < nrows; r += (int64_t)gridDim.x * wpb) {
    const int64_t a0 = adjptr[r];
    const int na = (int)(adjptr[r + 1] - a0);
    if (na <= 32) {
      const uint32_t v = lane < na ? (uint32_t)adj[a0 + lane] : 0xFFFFFFFFu;
      int rk = 0;
      for (int q = 0; q < na; q++) rk += __shfl_sync(0xffffffffu, v, q) < v;
      __syncwarp();
      if (lane < na) adj[a0 + rk] = (int32_t)v;
    } else if (na <= acap) {
      for (int t = lane; t < na; t += 32) u[t] = (uint32_t)adj[a0 + t];
      __syncwarp();
      warp_rank_distinct(u, na, [&](int q, int rk) { o[rk] = u[q]; });
      __syncwarp();
      for (int t = lane; t < na; t += 32) adj[a0 + t] = (int32_t)o[t];
    }
    __syncwarp();
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

cudaError_t exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s,
                                      const int *gate) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) {  // n == 0: out[0] = 0 (already so when gated: an empty scan never changes)
    if (!gate) k_zero_i64<<<1, 32, 0, s>>>(out, 1);
    return cudaGetLastError();
  }
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp, gate);
  k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp, nb, gate);
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp, out, gate);
  return cudaGetLastError();
}

cudaError_t launch_map_validate(const int32_t *v, int64_t n, int64_t limit, int *err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_map_validate<<<grid_for(n, 256), 256, 0, s>>>(v, n, limit, err);
  return cudaGetLastError();
}

cudaError_t launch_zero_i32(int32_t *p, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_zero_i32<<<grid_for(n, 256), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_max_i32(const int32_t *v, int64_t n, int *out, cudaStream_t s) {
  k_zero_i32<<<1, 32, 0, s>>>(out, 1);
  if (n > 0) k_max_count<<<grid_for(n, 256, 152 * 4), 256, 0, s>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t launch_zero_f64(double *p, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_zero_f64<<<grid_for((n + 1) / 2, 256, 152 * 8), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

// Rebuild: the incidence filled against the previous row offsets (no count, no scan); the
// in-place row pass checks every row's count, and sparsity_incidence_gated redoes the incidence
// from scratch when some count changed.
cudaError_t sparsity_incidence_reuse(fe_sparsity *sp, cudaStream_t s, int *err) {
  const int64_t n = sp->ncell * sp->ndr;
  k_zero_i32<<<grid_for(sp->nrows, 256), 256, 0, s>>>(sp->rowcnt, sp->nrows);
  if (n > 0)
    k_inc_fill<<<grid_for((n + 3) / 4, 256, 152 * 256), 256, 0, s>>>(sp->rmap->values, n, sp->nrows, sp->adjptr, sp->rowcnt, sp->adj, 1,
                                                 err);
  return cudaGetLastError();
}

cudaError_t sparsity_incidence_gated(fe_sparsity *sp, cudaStream_t s, int *err, const int *gate) {
  const int64_t n = sp->ncell * sp->ndr;
  k_zero_i32<<<grid_for(sp->nrows, 256), 256, 0, s>>>(sp->rowcnt, sp->nrows, gate);
  if (n > 0) k_inc_count<<<grid_for(n, 256), 256, 0, s>>>(sp->rmap->values, n, sp->nrows, sp->rowcnt, err, gate);
  cudaError_t e = exclusive_scan_i32_to_i64(sp->rowcnt, sp->adjptr, sp->nrows, sp->scan_tmp, s, gate);
  if (e != cudaSuccess) return e;
  k_zero_i32<<<grid_for(sp->nrows, 256), 256, 0, s>>>(sp->rowcnt, sp->nrows, gate);
  if (n > 0)
    k_inc_fill<<<grid_for((n + 3) / 4, 256, 152 * 256), 256, 0, s>>>(sp->rmap->values, n, sp->nrows, sp->adjptr, sp->rowcnt, sp->adj, 0,
                                                 nullptr, gate);
  return cudaGetLastError();
}

cudaError_t sparsity_incidence(fe_sparsity *sp, cudaStream_t s, int *err, int with_max) {
  const int64_t n = sp->ncell * sp->ndr;
  k_zero_i32<<<grid_for(sp->nrows, 256), 256, 0, s>>>(sp->rowcnt, sp->nrows);
  if (n > 0) k_inc_count<<<grid_for(n, 256), 256, 0, s>>>(sp->rmap->values, n, sp->nrows, sp->rowcnt, err);
  if (with_max) {
    k_zero_i32<<<1, 32, 0, s>>>(sp->d_maxcnt, 1);
    if (sp->nrows > 0)
      k_max_count<<<grid_for(sp->nrows, 256, 152 * 4), 256, 0, s>>>(sp->rowcnt, sp->nrows, sp->d_maxcnt);
  }
  cudaError_t e = exclusive_scan_i32_to_i64(sp->rowcnt, sp->adjptr, sp->nrows, sp->scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_zero_i32<<<grid_for(sp->nrows, 256), 256, 0, s>>>(sp->rowcnt, sp->nrows);
  if (n > 0)
    k_inc_fill<<<grid_for((n + 3) / 4, 256, 152 * 256), 256, 0, s>>>(sp->rmap->values, n, sp->nrows, sp->adjptr, sp->rowcnt, sp->adj);
  return cudaGetLastError();
}

namespace {
cudaError_t launch_rows(fe_sparsity *sp, cudaStream_t s, int *err, int *changed, const int *gate) {
  sp->adj_canonical = 0;  // the row kernel leaves each incidence list in fill order
  RowsParams p;
  p.nrows = sp->nrows;
  p.ndr = sp->ndr;
  p.ndc = sp->ndc;
  p.cmap = sp->cmap->values;
  p.adjptr = sp->adjptr;
  p.adj = sp->adj;
  p.rowlen = sp->rowcnt;
  p.coltmp = sp->coltmp;
  p.lut = sp->lut;
  p.cap = sp->cap;
  p.acap = sp->acap;
  p.mdiv_ndr = sp->ndr > 1 ? (~0ull / (uint64_t)sp->ndr) + 1 : 0;
  p.mdiv_ndc = sp->ndc > 1 ? (uint32_t)((0xFFFFFFFFull / (uint64_t)sp->ndc) + 1) : 0;
  p.packed_ok = sp->ncols < (int64_t)(1 << 24) - 1;
  p.err = err;
  // rows of at most 256 candidates and 32 incidences are sorted (no hash tables needed)
  p.sort_only = p.packed_ok && sp->cap <= 256 && sp->acap <= 32;
  p.pairs = sp->ndc % 2 == 0 && (reinterpret_cast<uintptr_t>(p.cmap) & 7) == 0;
  p.lut_pairs = sp->ndc % 2 == 0 && (reinterpret_cast<uintptr_t>(p.lut) & 1) == 0;
  p.colidx = changed ? sp->colidx : nullptr;
  p.rowptr = sp->rowptr;
  p.nnz = sp->nnz;
  p.changed = changed;
  p.gate = gate;
  p.canon = 0;
  p.check_counts = changed != nullptr;  // the in-place pass of a rebuild follows a guarded fill
  p.cols_changed = changed ? changed + 1 : nullptr;  // the second flag word: a column changed in place
  const size_t per_warp = (size_t)((p.sort_only ? 0 : 5 * sp->cap) + 2 * sp->acap + 64 + 128) * sizeof(int32_t);
  int warps = 8;
  while (warps > 1 && warps * per_warp > 96 * 1024) warps >>= 1;
  const size_t smem = warps * per_warp;
  auto kern = p.cols_changed && sp->track_cols ? k_rows_build<true> : k_rows_build<false>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // One chunk of eight rows per warp (up to 152 * 256 blocks, then the warps loop): the blocks are
  // scheduled as SMs free up, which balances the chunks' uneven cost (a chunk with vertex rows costs
  // several times one of edge rows); a grid of one resident wave looping over fixed chunks
  // measured 1.22 against 1.02 ms at P2 64^3, the former cap of 152 * 32 blocks 1.07 ms.
  const int64_t chunks = (sp->nrows + 7) / 8, blocks = (chunks + warps - 1) / warps;
  const int grid = (int)(blocks < 152 * 256 ? blocks : 152 * 256);
  if (sp->nrows > 0) kern<<<grid, warps * 32, smem, s>>>(p);
  return cudaGetLastError();
}
}  // namespace

cudaError_t sparsity_rows(fe_sparsity *sp, cudaStream_t s, int *err, const int *gate) {
  cudaError_t e = launch_rows(sp, s, err, nullptr, gate);
  if (e != cudaSuccess) return e;
  return exclusive_scan_i32_to_i64(sp->rowcnt, sp->rowptr, sp->nrows, sp->scan_tmp, s, gate);
}

cudaError_t sparsity_rows_inplace(fe_sparsity *sp, cudaStream_t s, int *err, int *changed) {
  return launch_rows(sp, s, err, changed, nullptr);
}

cudaError_t sparsity_canonical(fe_sparsity *sp, cudaStream_t s) {
  if (sp->adj_canonical) return cudaSuccess;
  const int warps = 8;
  const size_t smem = (size_t)warps * 2 * sp->acap * sizeof(uint32_t);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_adj_canon, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (sp->nrows > 0)
    k_adj_canon<<<grid_for(sp->nrows, warps, 152 * 16), warps * 32, smem, s>>>(sp->nrows, sp->adjptr, sp->adj, sp->acap);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) sp->adj_canonical = 1;
  return e;
}

cudaError_t sparsity_compact(fe_sparsity *sp, cudaStream_t s, int *err, int check_nnz, const int *gate) {
  const int warps = 8;
  if (sp->nrows > 0)
    k_rows_compact<<<grid_for((sp->nrows + 31) / 32, warps, 152 * 16), warps * 32, 0, s>>>(
        sp->nrows, sp->ndc, sp->adjptr, sp->rowptr, sp->coltmp, sp->colidx, sp->nnz, check_nnz, err, gate);
  return cudaGetLastError();
}

}  // namespace fe
