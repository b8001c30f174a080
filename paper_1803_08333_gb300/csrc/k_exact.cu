// Exact-digit GEMM: float-float accurate multi-column products on the tensor cores.
//
// The refinement residual r = b - A i and the right-hand side b need products about 40 bits
// accurate, where the split-BF16 GEMM gives 16 and a float-float GEMV costs some 40 FP32
// instructions per complex multiply-add.  Here every row of an operand (a row of the matrix, or
// a column of the right-hand-side block) is scaled by a power of two 2^e that puts its entries
// in [-1/2, 1/2] and written as S = 6 signed 8-bit digits
//
//     v = 2^e sum_{s<S} d_s 256^-(s+1),   d_s integer, |d_s| <= 128,
//
// every digit exact in BF16.  A product of two digits is an integer of magnitude at most 2^14,
// so the level sums P_L = sum_{s+t=L} D_s E_t^T over a K-block of KB = 128 columns stay below
// 6 * 128 * 2^14 < 2^24 and the FP32 tensor-memory accumulators hold them exactly, whatever
// the order of the additions.  After every K-block the epilogue warps fold the level sums into
// two 64-bit integer accumulators per output, H += P_0 2^16 + P_1 2^8 + P_2 and
// G += P_3 2^16 + P_4 2^8 + P_5, and at the end
//     D = 2^(eA_i + eB_j) 2^-56 (2^24 H + G)
// is rounded once to FP64.  Digit pairs of level S and beyond are dropped together with the
// digits past S: per term a truncation of about 2^-48 of the row scale times the column scale,
// the only error of the product.
//
// Kernel layout: one CTA per 128 x 32 output tile, 320 threads.  Warp 0 lane 0 issues the TMA
// loads of a 3-stage ring (each stage: the S digit planes of A, 128 x 32, and the S of B, 32 x 32,
// BF16 with the 64-byte swizzle; the B planes lie back to back, so B_0..B_t read as one operand
// of 32 (t + 1) rows).  Warp 1 lane 0 issues, per 16-wide K step, one MMA per A plane s against
// B_0..B_{S-1-s}: its N = 32 (S - s) output columns land on the accumulators of levels s..S-1,
// which sit side by side in tensor memory (level L at column 32 L), so S MMAs cover all S(S+1)/2
// digit pairs and every A plane is read from shared memory once per K step.  Two sets of level
// accumulators alternate between K-blocks; warps 2..9 fold a finished K-block (two warps per
// 32-lane quadrant of tensor memory, 16 columns each) while the next one accumulates, and write D.  Every wait
// is bounded; on timeout the kernel records an error code, frees its tensor memory and returns.
#include <cuda.h>
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

constexpr int XS = EXACT_DIGITS;  // digits per value
static_assert(XS == 6, "the integer fold below is written for 6 digits");
constexpr int XBN = 32;           // output columns per CTA
constexpr int XBK = 32;           // K per ring step (64-byte rows)
constexpr int XKB = 128;          // K-block between integer folds
constexpr int XSTAGES = 3;
constexpr int XSPK = XKB / XBK;   // ring steps per K-block
constexpr int XTILE_A = BM * XBK * 2;
constexpr int XTILE_B = XBN * XBK * 2;
constexpr int XSTAGE = XS * (XTILE_A + XTILE_B);
constexpr int XSMEM = XSTAGES * XSTAGE + 1024 + 256;
constexpr int XBUF = XS * XBN;  // tensor-memory columns of one set of level accumulators
constexpr uint32_t XTMEM_COLS = 2 * XBUF <= 128 ? 128 : (2 * XBUF <= 256 ? 256 : 512);
static_assert(2 * XBUF <= 512, "level accumulators exceed tensor memory");
static_assert(XS * XBN <= 256, "one MMA spans the accumulators of all levels");
static_assert((long long)XS * (128LL * 128LL) * XKB < (1LL << 24), "K-block level sums must stay exact in FP32");
static_assert(XSMEM <= 227 * 1024, "shared memory");
static_assert(XKB % XBK == 0 && XTILE_B % 512 == 0 && XTILE_A % 1024 == 0, "tile geometry");

struct ExactMaps {
  CUtensorMap a[XS];
  CUtensorMap b[XS];
};

constexpr int XTHREADS = 320;  // producer warp, MMA warp, 8 epilogue warps
static_assert(XBN == 32, "two epilogue warps of 16 columns per tensor-memory quadrant");

__global__ void __launch_bounds__(XTHREADS, 1)
exact_gemm_kernel(const __grid_constant__ ExactMaps maps, int M, int N, int K, const int* __restrict__ ea,
                  const int* __restrict__ eb, double* __restrict__ D, long long ldd, int* __restrict__ err) {
  RF_COUNT_LAUNCH();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + XSTAGES * XSTAGE);
  uint64_t* empty = full + XSTAGES;
  uint64_t* acc_full = empty + XSTAGES;  // [2]
  uint64_t* acc_empty = acc_full + 2;    // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * XBN, m0 = blockIdx.y * BM;  // N tiles fastest: CTAs sharing A run together
  const int ksteps = (K + XBK - 1) / XBK;
  const int nkb = (ksteps + XSPK - 1) / XSPK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < XSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 8);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(XTMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      for (int it = 0; it < ksteps; ++it) {
        const int s = it % XSTAGES, round = it / XSTAGES;
        if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1)) {
          atomicExch(err, 11);
          break;
        }
        uint8_t* st = smem + s * XSTAGE;
        const int kx = it * XBK;
        mbar_expect_tx(&full[s], XSTAGE);
#pragma unroll
        for (int p = 0; p < XS; ++p) tma_load_2d(st + p * XTILE_A, &maps.a[p], &full[s], kx, m0);
#pragma unroll
        for (int p = 0; p < XS; ++p) tma_load_2d(st + XS * XTILE_A + p * XTILE_B, &maps.b[p], &full[s], kx, n0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int it = 0; it < ksteps; ++it) {
        const int s = it % XSTAGES, round = it / XSTAGES;
        const int kb = it / XSPK, buf = kb & 1;
        const bool first = (it % XSPK) == 0;
        // this buffer's level sums of K-block kb - 2 must have been folded
        if (first && kb >= 2 && !mbar_wait(&acc_empty[buf], ((kb >> 1) - 1) & 1)) {
          atomicExch(err, 12);
          break;
        }
        if (!mbar_wait(&full[s], round & 1)) {
          atomicExch(err, 13);
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(smem + s * XSTAGE), b0 = a0 + XS * XTILE_A;
        const uint32_t t0 = tmem + (uint32_t)(buf * XBUF);
#pragma unroll
        for (int kk = 0; kk < XBK / 16; ++kk) {
          const uint32_t off = kk * 32;  // 16 BF16 along K inside the 64-byte swizzled row
          const uint64_t bd = sw64_desc(b0 + off);
#pragma unroll
          for (int sa = 0; sa < XS; ++sa)
            mma_bf16(t0 + (uint32_t)(sa * XBN), sw64_desc(a0 + sa * XTILE_A + off), bd,
                     idesc_bf16(BM, (XS - sa) * XBN, false), (first && kk == 0 && sa == 0) ? 0u : 1u);
        }
        mma_commit(&empty[s]);
        if ((it % XSPK) == XSPK - 1 || it == ksteps - 1) mma_commit(&acc_full[buf]);
      }
    }
  } else {
    // epilogue warps 2..9: warp w reads tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31 and
    // folds output columns 16 h .. 16 h + 15, h = (w - 2) / 4
    const int q = warp & 3, h = ((warp - 2) >> 2) * 16;
    const int row = m0 + 32 * q + lane;
    long long H[16], G[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) H[j] = G[j] = 0;
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      const int buf = kb & 1;
      ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (kb >> 1) & 1));
      if (!ok) {
        if (lane == 0) atomicExch(err, 14);
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * XBUF + h);
      uint32_t r[XS][16];
#pragma unroll
      for (int L = 0; L < XS; ++L) tmem_ld16_async(base + (uint32_t)(L * XBN), r[L]);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);  // the buffer may take the next K-block
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        long long p[XS];
#pragma unroll
        for (int L = 0; L < XS; ++L) p[L] = (long long)__float2int_rn(__uint_as_float(r[L][j]));
        H[j] += p[0] * 65536LL + p[1] * 256LL + p[2];
        G[j] += p[3] * 65536LL + p[4] * 256LL + p[5];
      }
    }
    if (ok && row < M) {
      const int er = ea[row];
      double* dst = D + (size_t)row * ldd;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = n0 + h + j;
        if (col < N) {
          const int e = er + eb[col];
          dst[col] = ldexp((double)H[j], e - 32) + ldexp((double)G[j], e - 56);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(XTMEM_COLS) : "memory");
}

// ---- digit planes ----
struct SrcC64Stacked {  // rows 0..n-1: Re of the complex64 matrix rows, rows n..2n-1: Im
  const float2* M;
  long long ld;
  int n;
  __device__ double operator()(int r, int k) const {
    return r < n ? (double)M[(size_t)r * ld + k].x : (double)M[(size_t)(r - n) * ld + k].y;
  }
};
struct SrcF32Pair {  // hi + lo FP32 planes of an FP64-accurate real matrix
  const float* hi;
  const float* lo;
  long long ld;
  __device__ double operator()(int r, int k) const {
    const size_t o = (size_t)r * ld + k;
    return (double)hi[o] + (double)lo[o];
  }
};
struct SrcXStacked {  // rows 0..nr-1: Re of the columns of X (n x nr, column-major), rows nr..: Im
  const double2* X;
  int n, nr;
  __device__ double operator()(int r, int k) const {
    return r < nr ? X[(size_t)r * n + k].x : X[(size_t)(r - nr) * n + k].y;
  }
};

constexpr int DT = 256;

// One CTA per row: the row's power-of-two scale 2^e (|v| 2^-e <= 1/2) and its XS base-256
// digits, by repeated rounding of the scaled value, written to XS planes (zeros in the padding).
template <class Src>
__global__ void __launch_bounds__(DT) digits_kernel(Src src, int K, long long ldp, __nv_bfloat16* __restrict__ planes,
                                                    long long plane_stride, int* __restrict__ e_out) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.x;
  double m = 0.0;
  for (int k = threadIdx.x; k < K; k += DT) m = fmax(m, fabs(src(r, k)));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  __shared__ double red[DT / 32];
  __shared__ int e_sh;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < DT / 32; ++w) t = fmax(t, red[w]);
    const int e = t > 0.0 ? ilogb(t) + 2 : 0;  // t < 2^(ilogb(t) + 1) = 2^(e - 1)
    e_sh = e;
    e_out[r] = e;
  }
  __syncthreads();
  const int e = e_sh;
  for (long long k = threadIdx.x; k < ldp; k += DT) {
    double u = k < K ? ldexp(src(r, (int)k), -e) : 0.0;
#pragma unroll
    for (int s = 0; s < XS; ++s) {
      const double t = u * 256.0;
      const double d = rint(t);
      u = t - d;
      planes[s * plane_stride + (size_t)r * ldp + k] = __double2bfloat16(d);
    }
  }
}

// Y[:, r] = scale * op(T) X[:, r] (+ Y) from D = [Tr; Ti] [Xr Xi] (FP64, 2n x 2nr) or, with real,
// D = P [Xr Xi] (n x 2nr); the same tiled combination as the split-BF16 path.
constexpr int CT = 32;
__global__ void combine_f64_kernel(const double* __restrict__ D, long long ldd, int n, int nr, int conj, int real,
                                   double2 scale, int accumulate, double2* __restrict__ Y) {
  RF_COUNT_LAUNCH();
  __shared__ double2 t[CT][CT + 1];
  const int i0 = blockIdx.x * CT, r0 = blockIdx.y * CT;
  const double sg = conj ? -1.0 : 1.0;
  for (int ii = threadIdx.y; ii < CT; ii += blockDim.y) {
    const int i = i0 + ii, r = r0 + threadIdx.x;
    double2 v = make_double2(0.0, 0.0);
    if (i < n && r < nr) {
      const double* top = D + (size_t)i * ldd;
      if (real) {
        v.x = top[r];
        v.y = top[nr + r];
      } else {
        const double* bot = D + (size_t)(n + i) * ldd;
        v.x = top[r] - sg * bot[nr + r];
        v.y = top[nr + r] + sg * bot[r];
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

cudaError_t exact_gemm(const ExactOperand& A, const ExactOperand& B, int M, int N, int K, double* D, long long ldd,
                       int* err, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0 || A.rows < M || B.rows < N) return cudaErrorInvalidValue;
  ExactMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int p = 0; p < XS; ++p)
    if (!make_map(&maps.a[p], A.d + p * A.plane_stride, M, K, A.ldp, BM, XBK) ||
        !make_map(&maps.b[p], B.d + p * B.plane_stride, N, K, B.ldp, XBN, XBK))
      return cudaErrorInvalidValue;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(exact_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, XSMEM);
  });
  if (attr != cudaSuccess) return attr;
  const dim3 grid((N + XBN - 1) / XBN, (M + BM - 1) / BM);
  ProfScope prof("gemm_exact", 0.0, 2.0 * (XS * (XS + 1) / 2) * (double)M * N * K, s);
  exact_gemm_kernel<<<grid, XTHREADS, XSMEM, s>>>(maps, M, N, K, A.e, B.e, D, ldd, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t exact_digits_c64(const float2* M, int n, long long ld, const ExactOperand& out, cudaStream_t s) {
  if (out.rows < 2 * n || out.ldp < ld) return cudaErrorInvalidValue;
  SrcC64Stacked src{M, ld, n};
  digits_kernel<<<2 * n, DT, 0, s>>>(src, n, out.ldp, out.d, out.plane_stride, out.e);
  return cudaGetLastError();
}

cudaError_t exact_digits_f32pair(const float* hi, const float* lo, int n, long long ld, const ExactOperand& out,
                                 cudaStream_t s) {
  if (out.rows < n || out.ldp < ld) return cudaErrorInvalidValue;
  SrcF32Pair src{hi, lo, ld};
  digits_kernel<<<n, DT, 0, s>>>(src, n, out.ldp, out.d, out.plane_stride, out.e);
  return cudaGetLastError();
}

cudaError_t exact_cplx_gemm(const ExactOperand& T, int n, const double2* X, double2* Y, int nr, bool conj,
                            double2 scale, bool accumulate, MrhsScratch& w, cudaStream_t s) {
  if (nr > w.cap_cols || n > w.cap_n || T.ldp > w.cap_ld || !w.xd || T.rows < 2 * n) return cudaErrorInvalidValue;
  ExactOperand B;
  B.d = w.xd;
  B.e = w.xe;
  B.rows = 2 * nr;
  B.ldp = T.ldp;
  B.plane_stride = (long long)2 * nr * T.ldp;
  SrcXStacked src{X, n, nr};
  digits_kernel<<<2 * nr, DT, 0, s>>>(src, n, B.ldp, B.d, B.plane_stride, B.e);
  cudaError_t e;
  if ((e = exact_gemm(T, B, 2 * n, 2 * nr, n, w.D64, 2 * nr, w.err, s)) != cudaSuccess) return e;
  const dim3 g((n + CT - 1) / CT, (nr + CT - 1) / CT), b(CT, 8);
  combine_f64_kernel<<<g, b, 0, s>>>(w.D64, 2 * nr, n, nr, conj ? 1 : 0, 0, scale, accumulate ? 1 : 0, Y);
  return cudaGetLastError();
}

cudaError_t exact_real_gemm(const ExactOperand& P, int n, const double2* X, double2* Y, int nr, double scale,
                            bool accumulate, MrhsScratch& w, cudaStream_t s) {
  if (nr > w.cap_cols || n > w.cap_n || P.ldp > w.cap_ld || !w.xd || P.rows < n) return cudaErrorInvalidValue;
  ExactOperand B;
  B.d = w.xd;
  B.e = w.xe;
  B.rows = 2 * nr;
  B.ldp = P.ldp;
  B.plane_stride = (long long)2 * nr * P.ldp;
  SrcXStacked src{X, n, nr};
  digits_kernel<<<2 * nr, DT, 0, s>>>(src, n, B.ldp, B.d, B.plane_stride, B.e);
  cudaError_t e;
  if ((e = exact_gemm(P, B, n, 2 * nr, n, w.D64, 2 * nr, w.err, s)) != cudaSuccess) return e;
  const dim3 g((n + CT - 1) / CT, (nr + CT - 1) / CT), b(CT, 8);
  combine_f64_kernel<<<g, b, 0, s>>>(w.D64, 2 * nr, n, nr, 0, 1, make_double2(scale, 0.0), accumulate ? 1 : 0, Y);
  return cudaGetLastError();
}

RF_LAUNCH_READER(launches_exact)

}  // namespace rfcmp
