// P4 kappa-diffusion element tensors on the tensor cores (tcgen05, kind::tf32, TMEM accumulator),
// FP64 global accumulation: the high-order precision study (the kernels COFFEE optimises most,
// Sec. 4.5).
//
// With kappa in P1 the element tensor of a triangle is a dense contraction: K_upper[n] =
// sum_k KL[k] C[n][k], KL = kappa_a * Lam_mn (3 x 6 = 18 per cell, k = a * 6 + mn) and C the
// reference tensor (120 x 18, generated from exact rationals, stored in FP32).  A block takes 128
// cells: each of its first 128 threads writes its cell's 18 coefficients as a row of A (K padded
// to 24), the other 128 write C as B (N = 120 padded to 128), and one thread issues the M = 128,
// N = 128 products into TMEM.  Each operand is split into TF32 hi + lo parts and the product is
// hi*hi + hi*lo + lo*hi (three TF32 products, FP32 accumulation): about FP32 accuracy.  Then the
// rows (one per cell) are read back from TMEM into shared memory and added into the CSR values
// with FP64 atomics through the lookup table, row by row of the element matrix (both triangles),
// so that consecutive atomics of a thread hit the same CSR row.
//
// TMEM: 128 columns per block; shared memory (62 KB) allows at most 3 blocks per SM, so at most
// 384 of the 512 columns are ever requested and allocation never waits.  The mbarrier wait is bounded: on
// a time-out the block flags the error, skips its scatter and still frees its columns.
#define FE_GEN_KAPPA_TC_TABLES  // the generated contraction tables of KappaTC<2, 4> (device arrays)
#include "fe_kernels.cuh"
#include "fe_tc.cuh"

namespace fe {
namespace {
using namespace kern;

using KT = fe_gen::KappaTC<2, 4>;
constexpr int kTcM = 128, kTcN = 128, kTcK = 24, kTcKC = kTcK / 4, kTcCols = 128, kTcThreads = 256;
constexpr int kTcSplit = 64;  // columns [0, 64) read from TMEM by warps 0-3, [64, 120) by warps 4-7
constexpr size_t kTcTileBytes = (size_t)kTcM * kTcK * 4;  // one operand part (12 KB)
constexpr int kTcStride = KT::N + 1;                       // staged results: 121 floats per cell (no bank conflicts)
constexpr size_t kTcStageBytes = (size_t)kTcM * kTcStride * 4;
constexpr size_t kTcData = kTcStageBytes > 4 * kTcTileBytes ? kTcStageBytes : 4 * kTcTileBytes;
constexpr size_t kTcSmem = kTcData + 64;  // operands (A hi, A lo, B hi, B lo), later the staged results; mbarrier, TMEM slot
constexpr unsigned kTcPolls = 1u << 22;
static_assert(KT::N <= kTcN && KT::K <= kTcK, "tile too small for the contraction");

// 256 threads: threads 0..127 build the A rows (cells), threads 128..255 the B rows; after the
// products, warps w and w + 4 read the same TMEM lanes (cells 32 (w % 4) ..) and split the 120
// columns between them into shared memory; then each warp scatters whole cells.
__global__ void __launch_bounds__(kTcThreads) k_mat_push_tc_kappa_p4(const AsmArgs a) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  float *Ahi = reinterpret_cast<float *>(dsm);
  float *Alo = reinterpret_cast<float *>(dsm + kTcTileBytes);
  float *Bhi = reinterpret_cast<float *>(dsm + 2 * kTcTileBytes);
  float *Blo = reinterpret_cast<float *>(dsm + 3 * kTcTileBytes);
  float *S = reinterpret_cast<float *>(dsm);  // after the products: S[cell][n], n < 120
  uint64_t *bar = reinterpret_cast<uint64_t *>(dsm + kTcData);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(dsm + kTcData + 16);
  constexpr int ND = KT::ND;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;

  if (t < 32) tc::tmem_alloc(tslot, kTcCols);
  if (t == 0) tc::mbar_init(bar, 1);

  if (t >= kTcM) {
    // B: row n = upper-triangle pair n of the element matrix, column k = coefficient k
    const int n = t - kTcM;
#pragma unroll 4
    for (int k = 0; k < kTcK; k++) {
      const float v = (n < KT::N && k < KT::K) ? fe_gen::kKappaTC24_C[n][k] : 0.0f;
      const float hi = tc::to_tf32(v);
      const int o = tc::kmajor_off(n, k, kTcKC) / 4;
      Bhi[o] = hi;
      Blo[o] = tc::to_tf32(v - hi);
    }
  } else {
    // A: row m = cell e's coefficients KL = kappa_a * Lam_mn (zero rows past the last cell)
    const int64_t e = blockIdx.x * (int64_t)kTcM + t;
    float KL[kTcK];
#pragma unroll
    for (int k = 0; k < kTcK; k++) KL[k] = 0.0f;
    if (e < a.ncell) {
      double x[3][2], kap[3];
      int32_t v[3], rows[ND];
      bool ok = gather_coords<2>(a, e, x, v);
      ok &= gather_rows<ND>(a, e, rows);
      ok &= gather_kappa<2>(a, e, kap);
      if (!ok) {
        flag(a.err, ERR_RANGE, e);
      } else {
        float Lam[Geo<2>::NLAM], vol;
        Geo<2>::template compute<OpsF32>(x, Lam, vol);
#pragma unroll
        for (int m = 0; m < 3; m++)
#pragma unroll
          for (int q = 0; q < Geo<2>::NLAM; q++) KL[m * Geo<2>::NLAM + q] = OpsF32::from_f64(kap[m]) * Lam[q];
      }
    }
#pragma unroll
    for (int k = 0; k < kTcK; k++) {
      const float hi = tc::to_tf32(KL[k]);
      const int o = tc::kmajor_off(t, k, kTcKC) / 4;
      Ahi[o] = hi;
      Alo[o] = tc::to_tf32(KL[k] - hi);
    }
  }
  tc::fence_proxy_async_smem();  // the generic-proxy writes above are read by the tensor cores
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (t == 0) {
    constexpr uint32_t idesc = tc::idesc_tf32(kTcM, kTcN);
    constexpr unsigned lbo = 128, sbo = kTcKC * 128;
#pragma unroll
    for (int s = 0; s < kTcK / 8; s++) {  // K = 8 per product: two core matrices along K
      const uint64_t ah = tc::smem_desc(reinterpret_cast<unsigned char *>(Ahi) + s * 256, lbo, sbo);
      const uint64_t al = tc::smem_desc(reinterpret_cast<unsigned char *>(Alo) + s * 256, lbo, sbo);
      const uint64_t bh = tc::smem_desc(reinterpret_cast<unsigned char *>(Bhi) + s * 256, lbo, sbo);
      const uint64_t bl = tc::smem_desc(reinterpret_cast<unsigned char *>(Blo) + s * 256, lbo, sbo);
      tc::mma_tf32(tmem, ah, bh, idesc, s > 0);
      tc::mma_tf32(tmem, ah, bl, idesc, 1);
      tc::mma_tf32(tmem, al, bh, idesc, 1);
    }
    tc::mma_commit(bar);
  }
  const bool done = tc::mbar_wait_bounded(bar, 0, kTcPolls);
  tc::fence_after_sync();
  const int timeout = __syncthreads_or(!done);  // uniform across the block from here on
  if (timeout) {
    if (t == 0) flag(a.err, ERR_TC_TIMEOUT, blockIdx.x);
  } else {
    // 1. TMEM -> shared memory (the operands are no longer read: the products have completed)
    const int quad = w & 3, half = w >> 2;
    const uint32_t tbase = tmem + ((uint32_t)(32 * quad) << 16);
    float *Srow = S + (size_t)(32 * quad + lane) * kTcStride;
#pragma unroll 1
    for (int c0 = half ? kTcSplit : 0; c0 < (half ? KT::N : kTcSplit); c0 += 8) {
      float vv[8];
      tc::tmem_ld8(tbase + (uint32_t)c0, vv);
#pragma unroll
      for (int j = 0; j < 8; j++)
        if (c0 + j < KT::N) Srow[c0 + j] = vv[j];
    }
  }
  __syncthreads();
  if (!timeout) {
    // 2. scatter, one warp per cell: lane l takes entries q = l, l + 32, ... of the element matrix
    //    in row-major order, so a warp's lookup-table loads are 32 consecutive bytes and its
    //    atomics of one instruction fall in two or three CSR rows of the cell
    for (int m = w; m < kTcM; m += kTcThreads / 32) {
      const int64_t e = blockIdx.x * (int64_t)kTcM + m;
      if (e >= a.ncell) break;  // warp-uniform
      int64_t rp = 0, rl = 0;
      bool ok = true;
      if (lane < ND) {
        const int32_t r = a.map[e * ND + lane];
        ok = !a.checks || (r >= 0 && r < a.nrows);  // a bad value was flagged when the cell was built
        if (ok) rp = a.rowptr[r];
        if (ok && a.checks) rl = a.rowptr[r + 1] - rp;
      }
      if (!__all_sync(0xffffffffu, ok)) continue;
      const uint8_t *L = a.lut + e * (ND * ND);
      const float *Sm = S + (size_t)m * kTcStride;
      if (a.checks) {  // check mode (a separate loop, so that the normal scatter stays as it is)
#pragma unroll
        for (int k = 0; k < (ND * ND + 31) / 32; k++) {
          const int q = 32 * k + lane;
          const int i = q / ND, j = q - (q / ND) * ND;
          const int64_t base = __shfl_sync(0xffffffffu, rp, i < ND ? i : 0);
          const int64_t len = __shfl_sync(0xffffffffu, rl, i < ND ? i : 0);
          if (q < ND * ND) {
            const int lo = i < j ? i : j, hi = i < j ? j : i;
            const int n = lo * ND - lo * (lo - 1) / 2 + (hi - lo);  // upper-triangle index of (lo, hi)
            if (L[q] >= len)  // a lookup-table entry beyond its row is skipped
              flag(a.err, ERR_LUT, e);
            else
              red_add_f64(a.vals + base + L[q], f32_to_f64_exact(Sm[n]));
          }
        }
        continue;
      }
#pragma unroll
      for (int k = 0; k < (ND * ND + 31) / 32; k++) {
        const int q = 32 * k + lane;
        const int i = q / ND, j = q - (q / ND) * ND;
        const int64_t base = __shfl_sync(0xffffffffu, rp, i < ND ? i : 0);
        if (q < ND * ND) {
          const int lo = i < j ? i : j, hi = i < j ? j : i;
          const int n = lo * ND - lo * (lo - 1) / 2 + (hi - lo);  // upper-triangle index of (lo, hi)
          red_add_f64(a.vals + base + L[q], f32_to_f64_exact(Sm[n]));
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (t < 32) tc::tmem_dealloc(tmem, kTcCols);
}

cudaError_t mat_push_tc_kappa_p4(const AsmArgs &a, cudaStream_t s) {
  if (a.ncell <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_mat_push_tc_kappa_p4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (a.ncell + kTcM - 1) / kTcM;
  k_mat_push_tc_kappa_p4<<<(unsigned)blocks, kTcThreads, kTcSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

LaunchFn pick_mat_push_tc(const fe_form_desc &d) {
  if (d.form == FE_FORM_KAPPA_DIFFUSION && d.dim == 2 && d.degree == 4) return &mat_push_tc_kappa_p4;
  return nullptr;
}

}  // namespace fe
