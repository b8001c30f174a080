// Split-BF16 GEMM on the 5th-generation tensor cores (tcgen05, TMEM accumulators, TMA loads).
//
//   D[M x N] (FP32, row-major) = sum over segments s of  sign_s * A_s[M x K] * B_s[N x K]^T  (+ D)
//
// Every operand is given as two BF16 planes (hi = bf16(x), lo = bf16(x - hi)), both K-major
// (row-major with K contiguous).  Each K step issues the three products hi*hi, hi*lo, lo*hi into
// one FP32 accumulator in tensor memory ("BF16x3"; the lo*lo term is below the accuracy of the
// other three).  Used for the multi-RHS complex products with the resident operator blocks and
// for the dense products of the factor refinement.
//
// Kernel layout: one persistent CTA per SM, 192 threads, 128 x BN output tiles.  Thread 0 issues
// the TMA loads of a stage ring (each stage: A hi, A lo, B hi, B lo tiles of 128 x 64 BF16 with
// the 128-byte swizzle) across tile boundaries, thread 32 issues the MMAs (tcgen05.mma kind::f16,
// M = 128, N = BN, K = 16 per instruction) into one of two tensor-memory accumulators and commits
// them to the stage's "empty" barrier, and warps 2-5 drain the other accumulator (tcgen05.ld
// 32x32b) through a shared-memory transpose into D with row-contiguous stores.  Every wait is
// bounded by a clock limit; on timeout the kernel records an error code, waits (bounded) for its
// own MMAs and copies, releases its tensor memory, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "rfcmp_internal.h"
#include "tc_common.cuh"

namespace rfcmp {

namespace {

using namespace tc;
constexpr int TILE_A = BM * BK * 2;  // 16 KiB per BF16 plane

// N tile (output columns per CTA) and ring depth: narrow tiles for narrow right-hand-side blocks
template <int BN>
struct TileCfg {
  static constexpr int STAGES = BN >= 128 ? 3 : (BN >= 64 ? 4 : 5);
  static constexpr int TILE_B = BN * BK * 2;
  static constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;
  static constexpr int EPI_BYTES = 4 * 32 * 33 * 4;  // a 32 x 33 FP32 transpose buffer per epilogue warp
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr uint32_t TMEM_COLS = 2 * (BN < 32 ? 32 : BN);  // two accumulators
};

struct GemmMaps {
  CUtensorMap a[2][2];  // [segment][hi, lo]
  CUtensorMap b[2][2];
};

constexpr int GEMM_THREADS = 192;  // warp 0 loads, warp 1 issues MMAs, warps 2-5 drain accumulators

// Output tile of linear index lin: groups of GROUP_M row tiles, the row tile fastest within a
// group.  The CTAs working at one time then cover a block of about GROUP_M x (SMs / GROUP_M)
// tiles and share its A and B panels in L2; in plain N-fastest order a wide result (N of many
// tiles, as in the Newton-Schulz products) has every CTA stream its own B panel from HBM.
constexpr int GROUP_M = 8;
__device__ __forceinline__ void tile_of(int lin, int tm, int tn, int& tile_m, int& tile_n) {
  const int grp = lin / (GROUP_M * tn), first = grp * GROUP_M, gs = min(tm - first, GROUP_M);
  const int local = lin - grp * GROUP_M * tn;
  tile_m = first + local % gs;
  tile_n = local / gs;
}

// The same order restricted to the tiles on or above the diagonal of a t x t tile grid, numbered
// without gaps (so that a stride over them gives every CTA the same number of tiles): group g
// holds rows first .. first + gs - 1; its columns first .. first + gs - 1 hold 1, 2, .., gs tiles
// (rows up to the column), the columns after them gs tiles each.
__device__ __forceinline__ void upper_tile_of(int c, int t, int& tile_m, int& tile_n) {
  int first = 0;
  for (;;) {
    const int gs = min(t - first, GROUP_M);
    const int tri = gs * (gs + 1) / 2;
    const int cnt = tri + gs * (t - first - gs);
    if (c < cnt || first + gs >= t) {
      if (c < tri) {  // column first + j holds rows first .. first + j
        int j = 0;
        while ((j + 1) * (j + 2) / 2 <= c) ++j;
        tile_n = first + j;
        tile_m = first + (c - j * (j + 1) / 2);
      } else {
        c -= tri;
        tile_n = first + gs + c / gs;
        tile_m = first + c % gs;
      }
      return;
    }
    c -= cnt;
    first += gs;
  }
}

// tile i of the kernel's sequence: all tiles, or (upper) those on or above the diagonal
__device__ __forceinline__ void seq_tile(int i, int tm, int tn, int upper, int& tile_m, int& tile_n) {
  if (upper) upper_tile_of(i, tn, tile_m, tile_n);
  else tile_of(i, tm, tn, tile_m, tile_n);
}

// Persistent kernel: CTA b takes the tiles b, b + G, b + 2G, ... (G CTAs, one per SM).  The
// producer keeps the stage ring full across tile boundaries; the MMA warp accumulates tile t into
// tensor-memory buffer t % 2 while the epilogue warps drain buffer (t - 1) % 2, so a tile's
// epilogue overlaps the next tile's main loop.  The epilogue goes through a shared-memory
// transpose so that each warp store writes 128 contiguous bytes of one row of D.
template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
gemm_bf16x3_kernel(const __grid_constant__ GemmMaps maps, int nseg, int neg_mask, int M, int N, int K,
                   float* __restrict__ D, long long ldd, int accumulate, int* __restrict__ err, int upper) {
  RF_COUNT_LAUNCH();
  using C = TileCfg<BN>;
  constexpr int STAGES = C::STAGES, STAGE_BYTES = C::STAGE_BYTES, TILE_B = C::TILE_B;
  constexpr uint32_t ACC_COLS = BN < 32 ? 32 : BN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* epi = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + C::EPI_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;  // [2]: the MMAs of a tile have completed
  uint64_t* acc_empty = acc_full + 2;   // [2]: the epilogue has read the buffer
  uint64_t* drained = acc_empty + 2;    // every MMA this CTA issued has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tn = (N + BN - 1) / BN, tm = (M + BM - 1) / BM;
  // upper (BN == BM, tm >= tn): the tn (tn + 1) / 2 tiles on or above the diagonal
  const int tiles = upper ? tn * (tn + 1) / 2 : tm * tn;
  const int kblocks = (K + BK - 1) / BK;
  const int total = nseg * kblocks;  // ring iterations per tile

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(drained, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: TMA loads into the stage ring, tile after tile
      long long it = 0;
      bool ok = true;
      for (int lin = blockIdx.x; lin < tiles && ok; lin += gridDim.x) {
        int tile_m, tile_n;
        seq_tile(lin, tm, tn, upper, tile_m, tile_n);
        const int m0 = tile_m * BM, n0 = tile_n * BN;
        for (int q = 0; q < total; ++q, ++it) {
          const int s = (int)(it % STAGES);
          const long long round = it / STAGES;
          if (round > 0 && !mbar_wait(&empty[s], (uint32_t)((round - 1) & 1))) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          const int seg = q / kblocks, kx = (q % kblocks) * BK;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          tma_load_2d(st, &maps.a[seg][0], &full[s], kx, m0);
          tma_load_2d(st + TILE_A, &maps.a[seg][1], &full[s], kx, m0);
          tma_load_2d(st + 2 * TILE_A, &maps.b[seg][0], &full[s], kx, n0);
          tma_load_2d(st + 2 * TILE_A + TILE_B, &maps.b[seg][1], &full[s], kx, n0);
        }
      }
      // the copies of the last rounds have landed before the CTA may exit (bounded)
      for (long long j = it - 1; j >= 0 && j >= it - STAGES; --j)
        if (!mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1))) atomicExch(err, 4);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      const uint32_t id_pos = idesc_bf16(BM, BN, false), id_neg = idesc_bf16(BM, BN, true);
      long long it = 0;
      int t = 0;  // tiles of this CTA so far
      bool ok = true;
      for (int lin = blockIdx.x; lin < tiles && ok; lin += gridDim.x) {
        int tile_m, tile_n;
        seq_tile(lin, tm, tn, upper, tile_m, tile_n);
        const int b = t & 1, use = t >> 1;
        if (use > 0 && !mbar_wait(&acc_empty[b], (uint32_t)((use - 1) & 1))) {
          atomicExch(err, 5);
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)b * ACC_COLS;
        for (int q = 0; q < total; ++q, ++it) {
          const int s = (int)(it % STAGES);
          const long long round = it / STAGES;
          if (!mbar_wait(&full[s], (uint32_t)(round & 1))) {
            atomicExch(err, 2);
            ok = false;
            break;
          }
          tc_fence_after();
          const int seg = q / kblocks;
          const uint32_t idesc = (neg_mask >> seg) & 1 ? id_neg : id_pos;
          const uint32_t a_hi = smem_u32(smem + s * STAGE_BYTES), a_lo = a_hi + TILE_A;
          const uint32_t b_hi = a_hi + 2 * TILE_A, b_lo = b_hi + TILE_B;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint32_t off = kk * 32;  // 16 BF16 along K inside the 128-byte swizzled row
            const uint64_t ah = sw128_desc(a_hi + off), al = sw128_desc(a_lo + off);
            const uint64_t bh = sw128_desc(b_hi + off), bl = sw128_desc(b_lo + off);
            mma_bf16(acc, ah, bh, idesc, (q > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(acc, ah, bl, idesc, 1u);
            mma_bf16(acc, al, bh, idesc, 1u);
          }
          mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(&acc_full[b]);  // arrives when the tile's MMAs have completed
        ++t;
      }
      // every MMA issued above has completed before tensor memory is released (bounded)
      mma_commit(drained);
      if (!mbar_wait(drained, 0)) atomicExch(err, 6);
    }
  } else {
    // epilogue: warp w drains accumulator lanes (rows) 32 (w % 4) .. + 31
    const int quarter = warp & 3;
    float* tb = epi + (warp - 2) * 32 * 33;
    int t = 0;
    for (int lin = blockIdx.x; lin < tiles; lin += gridDim.x) {
      int tile_m, tile_n;
      seq_tile(lin, tm, tn, upper, tile_m, tile_n);
      const int b = t & 1, use = t >> 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (uint32_t)(use & 1)));
      if (!ok) {
        if (lane == 0) atomicExch(err, 3);
        break;
      }
      tc_fence_after();
      const int r0 = tile_m * BM + 32 * quarter, n0 = tile_n * BN;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)b * ACC_COLS + (uint32_t)c0, r);
        // lane = row of the block; transpose so that lane = column for the stores
#pragma unroll
        for (int j = 0; j < 32; ++j) tb[lane * 33 + j] = __uint_as_float(r[j]);
        __syncwarp();
        const int col = n0 + c0 + lane;
        if (col < N) {
#pragma unroll 4
          for (int i = 0; i < 32; ++i) {
            const int row = r0 + i;
            if (row >= M) break;
            float* dst = D + (size_t)row * ldd + col;
            float v = tb[i * 33 + lane];
            if (accumulate) v += *dst;
            *dst = v;
          }
        }
        __syncwarp();
      }
      // the buffer's loads have completed (tmem_ld32 waits): hand it back to the MMA warp
      tc_fence_before();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
      ++t;
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
}

// FP32 (or FP64) -> BF16 hi/lo planes; CTAs take whole rows (no per-element index division)
template <class T>
__global__ void split_bf16_kernel(const T* __restrict__ src, long long ld_src, int rows, int cols,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long long ld_dst) {
  RF_COUNT_LAUNCH();
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const T* sr = src + (size_t)r * ld_src;
    __nv_bfloat16* hr = hi + (size_t)r * ld_dst;
    __nv_bfloat16* lr = lo + (size_t)r * ld_dst;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) {
      const float v = (float)sr[c];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      hr[c] = h;
      lr[c] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

template <int BN>
cudaError_t gemm_launch(const SplitOperand* A, const SplitOperand* B, const int* negate, int nseg, int M, int N, int K,
                        float* D, long long ldd, bool accumulate, int* err_dev, cudaStream_t s, bool upper) {
  if (upper && BN != BM) return cudaErrorInvalidValue;
  using C = TileCfg<BN>;
  GemmMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  int neg_mask = 0;
  for (int g = 0; g < nseg; ++g) {
    if (A[g].rows < M || B[g].rows < N) return cudaErrorInvalidValue;
    if (!make_map(&maps.a[g][0], A[g].hi, M, K, A[g].ld, BM) || !make_map(&maps.a[g][1], A[g].lo, M, K, A[g].ld, BM) ||
        !make_map(&maps.b[g][0], B[g].hi, N, K, B[g].ld, BN) || !make_map(&maps.b[g][1], B[g].lo, N, K, B[g].ld, BN))
      return cudaErrorInvalidValue;
    if (negate && negate[g]) neg_mask |= 1 << g;
  }
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err =
        cudaFuncSetAttribute(gemm_bf16x3_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const long long tnl = (N + BN - 1) / BN, tml = (M + BM - 1) / BM;
  if (upper && tml < tnl) return cudaErrorInvalidValue;
  const long long tiles = upper ? tnl * (tnl + 1) / 2 : tnl * tml;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  // the SM count, read once (launches may come from several host threads)
  static std::once_flag sms_once;
  static int sms = 0;
  static cudaError_t sms_err = cudaSuccess;
  std::call_once(sms_once, [] {
    int dev = 0;
    sms_err = cudaGetDevice(&dev);
    if (sms_err == cudaSuccess) sms_err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  if (sms_err != cudaSuccess || sms <= 0) return sms_err != cudaSuccess ? sms_err : cudaErrorInvalidValue;
  const int grid = (int)std::max(1LL, std::min<long long>(tiles, sms));
  double frac = 1.0;  // share of the output tiles computed
  if (upper) {
    const double tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
    frac = std::min(1.0, tn * (tn + 1) / 2.0 / (tm * tn));  // tiles with n-tile >= m-tile (tm >= tn)
  }
  ProfScope prof("gemm_bf16x3", 0.0, 6.0 * (double)M * N * K * nseg * frac, s);
  gemm_bf16x3_kernel<BN><<<grid, GEMM_THREADS, C::SMEM_BYTES, s>>>(maps, nseg, neg_mask, M, N, K, D, ldd,
                                                                   accumulate ? 1 : 0, err_dev, upper ? 1 : 0);
  return cudaGetLastError();
}

// complex64 matrix (row stride ld) -> BF16 planes Re hi/lo, Im hi/lo (row stride ldp); CTAs take
// whole rows
__global__ void split_c64_kernel(const float2* __restrict__ M, int n, long long ld, __nv_bfloat16* __restrict__ rh,
                                 __nv_bfloat16* __restrict__ rl, __nv_bfloat16* __restrict__ ih,
                                 __nv_bfloat16* __restrict__ il, long long ldp) {
  RF_COUNT_LAUNCH();
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const float2* mr = M + (size_t)r * ld;
    const size_t o0 = (size_t)r * ldp;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const float2 v = mr[c];
      const __nv_bfloat16 a = __float2bfloat16_rn(v.x), b = __float2bfloat16_rn(v.y);
      const size_t o = o0 + c;
      rh[o] = a;
      rl[o] = __float2bfloat16_rn(v.x - __bfloat162float(a));
      ih[o] = b;
      il[o] = __float2bfloat16_rn(v.y - __bfloat162float(b));
    }
  }
}

// X (complex128, column-major n x nr) -> BF16 planes of Re X^T and Im X^T (nr x ldp each, hi and lo);
// with stacked, Re and Im share one operand of 2 nr rows (rows nr.. hold Im).
__global__ void split_x_kernel(const double2* __restrict__ X, int n, int nr, long long ldp, bool stacked,
                               __nv_bfloat16* __restrict__ rh, __nv_bfloat16* __restrict__ rl,
                               __nv_bfloat16* __restrict__ ih, __nv_bfloat16* __restrict__ il) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.y;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < ldp; k += (long long)gridDim.x * blockDim.x) {
    const double2 v = k < n ? X[(size_t)r * n + k] : make_double2(0.0, 0.0);
    const float re = (float)v.x, im = (float)v.y;
    const __nv_bfloat16 a = __float2bfloat16_rn(re), b = __float2bfloat16_rn(im);
    const size_t orow = (size_t)r * ldp + k;
    const size_t irow = stacked ? (size_t)(nr + r) * ldp + k : orow;
    rh[orow] = a;
    rl[orow] = __float2bfloat16_rn(re - __bfloat162float(a));
    ih[irow] = b;
    il[irow] = __float2bfloat16_rn(im - __bfloat162float(b));
  }
}

// Y[:, r] = scale * op(T) X[:, r] (+ Y) from D = [Tr; Ti] [Xr Xi] (2n x 2nr, row stride ldd):
// T X = (Tr Xr - Ti Xi) + i (Tr Xi + Ti Xr); conj(T) flips the sign of the Ti terms.  With real,
// D = P [Xr Xi] (n x 2nr) of a real P and Y = scale * (D[:, r] + i D[:, nr + r]) (+ Y).
// 32 x 32 tiles of (row i, column r) go through shared memory so that both the reads of D
// (along r) and the writes of Y (along i) are coalesced.
constexpr int CT = 32;
__global__ void combine_cplx_kernel(const float* __restrict__ D, long long ldd, int n, int nr, int conj, int real,
                                    double2 scale, int accumulate, double2* __restrict__ Y) {
  RF_COUNT_LAUNCH();
  __shared__ double2 t[CT][CT + 1];
  const int i0 = blockIdx.x * CT, r0 = blockIdx.y * CT;
  const double sg = conj ? -1.0 : 1.0;
  for (int ii = threadIdx.y; ii < CT; ii += blockDim.y) {
    const int i = i0 + ii, r = r0 + threadIdx.x;
    double2 v = make_double2(0.0, 0.0);
    if (i < n && r < nr) {
      const float* top = D + (size_t)i * ldd;
      if (real) {
        v.x = (double)top[r];
        v.y = (double)top[nr + r];
      } else {
        const float* bot = D + (size_t)(n + i) * ldd;
        v.x = (double)top[r] - sg * (double)bot[nr + r];
        v.y = (double)top[nr + r] + sg * (double)bot[r];
      }
    }
    t[ii][threadIdx.x] = v;
  }
  __syncthreads();
  for (int rr = threadIdx.y; rr < CT; rr += blockDim.y) {
    const int r = r0 + rr, i = i0 + threadIdx.x;
    if (i >= n || r >= nr) continue;
    const double2 v = t[threadIdx.x][rr];
    double2 o = make_double2(scale.x * v.x - scale.y * v.y, scale.x * v.y + scale.y * v.x);
    if (accumulate) {
      const double2 p = Y[(size_t)r * n + i];
      o.x += p.x;
      o.y += p.y;
    }
    Y[(size_t)r * n + i] = o;
  }
}

}  // namespace

cudaError_t split_c64_planes(const float2* M, int n, long long ld, const CplxPlanes& P, cudaStream_t s) {
  const int blocks = std::max(1, std::min(n, 8 * 152));
  split_c64_kernel<<<blocks, 256, 0, s>>>(M, n, ld, P.rh, P.rl, P.ih, P.il, P.ldp);
  return cudaGetLastError();
}

cudaError_t cplx_gemm(const CplxPlanes& T, const double2* X, double2* Y, int nr, bool conj, double2 scale,
                      bool accumulate, MrhsScratch& w, cudaStream_t s) {
  const int n = T.n;
  const long long ldp = T.ldp;
  if (nr > w.cap_cols || ldp > w.cap_ld || n > w.cap_n) return cudaErrorInvalidValue;
  if (T.ih != T.rh + (size_t)n * ldp || T.il != T.rl + (size_t)n * ldp) return cudaErrorInvalidValue;
  __nv_bfloat16* xb = w.xb;
  const size_t pl = (size_t)2 * nr * ldp;  // stacked Re / Im rows of X^T
  __nv_bfloat16 *bh = xb, *bl = xb + pl;
  dim3 g1((unsigned)std::min<long long>((ldp + 255) / 256, 64), nr);
  split_x_kernel<<<g1, 256, 0, s>>>(X, n, nr, ldp, true, bh, bl, bh, bl);
  // one pass over the matrix: D = [Tr; Ti] [Xr Xi]  (2n x 2nr)
  SplitOperand A, B;
  A.hi = T.rh; A.lo = T.rl; A.rows = 2 * n; A.ld = ldp;
  B.hi = bh; B.lo = bl; B.rows = 2 * nr; B.ld = ldp;
  cudaError_t e;
  if ((e = gemm_bf16x3(&A, &B, nullptr, 1, 2 * n, 2 * nr, n, w.D, 2 * nr, false, w.err, s, w.bn)) != cudaSuccess)
    return e;
  dim3 g2((n + CT - 1) / CT, (nr + CT - 1) / CT), b2(CT, 8);
  combine_cplx_kernel<<<g2, b2, 0, s>>>(w.D, 2 * nr, n, nr, conj ? 1 : 0, 0, scale, accumulate ? 1 : 0, Y);
  return cudaGetLastError();
}

cudaError_t real_gemm(const RealPlanes& P, const double2* X, double2* Y, int nr, double scale, bool accumulate,
                      MrhsScratch& w, cudaStream_t s) {
  const int n = P.n;
  const long long ldp = P.ldp;
  if (2 * nr > 2 * w.cap_cols || ldp > w.cap_ld || n > w.cap_n) return cudaErrorInvalidValue;
  __nv_bfloat16* xb = w.xb;
  const size_t pl = (size_t)2 * nr * ldp;  // stacked Re / Im rows
  __nv_bfloat16 *bh = xb, *bl = xb + pl;
  dim3 g1((unsigned)std::min<long long>((ldp + 255) / 256, 64), nr);
  split_x_kernel<<<g1, 256, 0, s>>>(X, n, nr, ldp, true, bh, bl, bh, bl);
  SplitOperand A, B;
  A.hi = P.h; A.lo = P.l; A.rows = n; A.ld = ldp;
  B.hi = bh; B.lo = bl; B.rows = 2 * nr; B.ld = ldp;
  cudaError_t e;
  if ((e = gemm_bf16x3(&A, &B, nullptr, 1, n, 2 * nr, n, w.D, 2 * nr, false, w.err, s, w.bn)) != cudaSuccess) return e;
  dim3 g2((n + CT - 1) / CT, (nr + CT - 1) / CT), b2(CT, 8);
  combine_cplx_kernel<<<g2, b2, 0, s>>>(w.D, 2 * nr, n, nr, 0, 1, make_double2(scale, 0.0), accumulate ? 1 : 0, Y);
  return cudaGetLastError();
}

cudaError_t split_bf16_f32(const float* src, long long ld_src, int rows, int cols, __nv_bfloat16* hi,
                           __nv_bfloat16* lo, long long ld_dst, cudaStream_t s) {
  const int blocks = std::max(1, std::min(rows, 8 * 152));
  split_bf16_kernel<float><<<blocks, 256, 0, s>>>(src, ld_src, rows, cols, hi, lo, ld_dst);
  return cudaGetLastError();
}

cudaError_t split_bf16_f64(const double* src, long long ld_src, int rows, int cols, __nv_bfloat16* hi,
                           __nv_bfloat16* lo, long long ld_dst, cudaStream_t s) {
  const int blocks = std::max(1, std::min(rows, 8 * 152));
  split_bf16_kernel<double><<<blocks, 256, 0, s>>>(src, ld_src, rows, cols, hi, lo, ld_dst);
  return cudaGetLastError();
}

cudaError_t gemm_bf16x3(const SplitOperand* A, const SplitOperand* B, const int* negate, int nseg, int M, int N,
                        int K, float* D, long long ldd, bool accumulate, int* err_dev, cudaStream_t s, int bn,
                        bool upper) {
  if (nseg < 1 || nseg > 2 || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  if (upper) bn = 128;
  if (bn == 0) bn = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  switch (bn) {
    case 32:
      return gemm_launch<32>(A, B, negate, nseg, M, N, K, D, ldd, accumulate, err_dev, s, upper);
    case 64:
      return gemm_launch<64>(A, B, negate, nseg, M, N, K, D, ldd, accumulate, err_dev, s, upper);
    case 128:
      return gemm_launch<128>(A, B, negate, nseg, M, N, K, D, ldd, accumulate, err_dev, s, upper);
    default:
      return cudaErrorInvalidValue;
  }
}

RF_LAUNCH_READER(launches_gemm)

}  // namespace rfcmp
