// Dense and sparse linear algebra of the RF-CMP application (Sec. 3, Sec. 4):
//  * GEMV over the resident complex64 blocks T_A, V (and conj for T^H = conj(T conj x),
//    Sec. 3.4) and over the real dense factors (Sigma^T Sigma)^+ and G_ll^{-1},
//    in two arithmetic modes:
//      GEMV_F32  x rounded to FP32, FP32 FMAs, partial sums flushed to FP64 per chunk
//      GEMV_FF   x split in FP32 hi + lo, exact products (fmaf residual), float-float
//                accumulation: about 1e-14 of sum |terms|, an FP64-equivalent residual
//  * sparse Sigma^T, Lambda^T, Sigma^T Sigma and the fused edge-space combinations,
//  * per-column CG scalars kept on the device,
//  * block CG building the dense inverses of the sparse SPD factors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <set>
#include <vector>

#include "rfcmp_internal.h"

namespace rfcmp {

namespace {

constexpr int GEMV_ROWS_PER_WARP = 4;
constexpr int GEMV_WARPS = 8;
constexpr int GEMV_ROWS = GEMV_ROWS_PER_WARP * GEMV_WARPS;  // 32 rows per work unit
constexpr int GEMV_CHUNK = 1024;                            // columns per work unit

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// float-float accumulation of a product a*b (a, b FP32; b = bh + bl)
__device__ __forceinline__ void ff_mac(float& hi, float& lo, float a, float bh, float bl) {
  const float p = a * bh;
  const float e = fmaf(a, bh, -p);
  const float c = fmaf(a, bl, e);
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += err + c;
}

// streaming load of the matrix: read once, kept out of L1
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// x (complex128, n x nr) -> FP32 hi (and lo) copies padded to ld, and zero the accumulator
__global__ void gemv_prep_kernel(const double2* __restrict__ x, int n, int ld, int nr, float2* __restrict__ xh,
                                 float2* __restrict__ xl, double2* __restrict__ y) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ld; i += gridDim.x * blockDim.x) {
    const double2 v = i < n ? x[(size_t)r * n + i] : make_double2(0.0, 0.0);
    const float2 h = make_float2((float)v.x, (float)v.y);
    xh[(size_t)r * ld + i] = h;
    if (xl) xl[(size_t)r * ld + i] = make_float2((float)(v.x - (double)h.x), (float)(v.y - (double)h.y));
    // the product adds into y: a fresh product starts from zero (x is read above, first)
    if (y && i < n) y[(size_t)r * n + i] = make_double2(0.0, 0.0);
  }
}

// Adds scale times the per-lane FP64 row sums of one row block into the output.
template <int NR>
__device__ __forceinline__ void flush_rows(double (&acc)[GEMV_ROWS_PER_WARP][NR][2], int row0, int n, int lane,
                                           double2* __restrict__ out, double scale) {
#pragma unroll
  for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const double re = warp_sum(acc[a][r][0]);
      const double im = warp_sum(acc[a][r][1]);
      acc[a][r][0] = acc[a][r][1] = 0.0;
      if (lane == 0 && row0 + a < n) {
        double* o = reinterpret_cast<double*>(out + (size_t)r * n + row0 + a);
        atomicAdd(o, scale * re);
        atomicAdd(o + 1, scale * im);
      }
    }
}

// ---------------------------------------------------------------- complex64 GEMV (persistent)
// Work unit u = (row block rb, column chunk cc); CTA g owns units [u0, u1) of the
// row-major unit order, so every CTA streams the same number of matrix bytes.
template <int NR, bool FF, bool CONJ>
__global__ void __launch_bounds__(GEMV_WARPS * 32)
gemv_c64_kernel(const float2* __restrict__ M, int ld, int n, const float2* __restrict__ xh,
                const float2* __restrict__ xl, double2* __restrict__ out, double scale, long long units, int upr, int chunk) {
  RF_COUNT_LAUNCH();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  double acc[GEMV_ROWS_PER_WARP][NR][2];
#pragma unroll
  for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[a][r][0] = acc[a][r][1] = 0.0;
  long long cur_rb = -1;
  for (long long u = u0; u < u1; ++u) {
    const int rb = (int)(u / upr), cc = (int)(u % upr);
    const int row0 = rb * GEMV_ROWS + warp * GEMV_ROWS_PER_WARP;
    if (rb != cur_rb) {
      if (cur_rb >= 0) flush_rows<NR>(acc, (int)cur_rb * GEMV_ROWS + warp * GEMV_ROWS_PER_WARP, n, lane, out, scale);
      cur_rb = rb;
    }
    const int cb = cc * chunk;
    const int npair = min(chunk, ld - cb) / 2;
    float fh[GEMV_ROWS_PER_WARP][NR][2], fl[GEMV_ROWS_PER_WARP][NR][2];
#pragma unroll
    for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
      for (int r = 0; r < NR; ++r) fh[a][r][0] = fh[a][r][1] = fl[a][r][0] = fl[a][r][1] = 0.f;
    const float4* rowp[GEMV_ROWS_PER_WARP];
#pragma unroll
    for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
      rowp[a] = reinterpret_cast<const float4*>(M + (size_t)min(row0 + a, n - 1) * ld + cb);
#pragma unroll 4
    for (int p = lane; p < npair; p += 32) {
      float4 m[GEMV_ROWS_PER_WARP];
#pragma unroll
      for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
        m[a] = row0 + a < n ? ld_stream(rowp[a] + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (CONJ) {
          m[a].y = -m[a].y;
          m[a].w = -m[a].w;
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const float4 x4 = __ldg(reinterpret_cast<const float4*>(xh + (size_t)r * ld + cb) + p);
        if (!FF) {
#pragma unroll
          for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
            float re = fh[a][r][0], im = fh[a][r][1];
            re = fmaf(m[a].x, x4.x, re);
            re = fmaf(-m[a].y, x4.y, re);
            re = fmaf(m[a].z, x4.z, re);
            re = fmaf(-m[a].w, x4.w, re);
            im = fmaf(m[a].x, x4.y, im);
            im = fmaf(m[a].y, x4.x, im);
            im = fmaf(m[a].z, x4.w, im);
            im = fmaf(m[a].w, x4.z, im);
            fh[a][r][0] = re;
            fh[a][r][1] = im;
          }
        } else {
          const float4 l4 = __ldg(reinterpret_cast<const float4*>(xl + (size_t)r * ld + cb) + p);
#pragma unroll
          for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
            ff_mac(fh[a][r][0], fl[a][r][0], m[a].x, x4.x, l4.x);
            ff_mac(fh[a][r][0], fl[a][r][0], -m[a].y, x4.y, l4.y);
            ff_mac(fh[a][r][0], fl[a][r][0], m[a].z, x4.z, l4.z);
            ff_mac(fh[a][r][0], fl[a][r][0], -m[a].w, x4.w, l4.w);
            ff_mac(fh[a][r][1], fl[a][r][1], m[a].x, x4.y, l4.y);
            ff_mac(fh[a][r][1], fl[a][r][1], m[a].y, x4.x, l4.x);
            ff_mac(fh[a][r][1], fl[a][r][1], m[a].z, x4.w, l4.w);
            ff_mac(fh[a][r][1], fl[a][r][1], m[a].w, x4.z, l4.z);
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        acc[a][r][0] += (double)fh[a][r][0] + (double)fl[a][r][0];
        acc[a][r][1] += (double)fh[a][r][1] + (double)fl[a][r][1];
      }
  }
  if (cur_rb >= 0) flush_rows<NR>(acc, (int)cur_rb * GEMV_ROWS + warp * GEMV_ROWS_PER_WARP, n, lane, out, scale);
}

// ---------------------------------------------------------------- real (hi + lo) GEMV (persistent)
template <int NR, bool FF>
__global__ void __launch_bounds__(GEMV_WARPS * 32)
gemv_r32_kernel(const float* __restrict__ Mhi, const float* __restrict__ Mlo, int ld, int n,
                const float2* __restrict__ xh, const float2* __restrict__ xl, double2* __restrict__ out, double scale,
                long long units, int upr, int chunk) {
  RF_COUNT_LAUNCH();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  double acc[GEMV_ROWS_PER_WARP][NR][2];
#pragma unroll
  for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[a][r][0] = acc[a][r][1] = 0.0;
  long long cur_rb = -1;
  for (long long u = u0; u < u1; ++u) {
    const int rb = (int)(u / upr), cc = (int)(u % upr);
    const int row0 = rb * GEMV_ROWS + warp * GEMV_ROWS_PER_WARP;
    if (rb != cur_rb) {
      if (cur_rb >= 0) flush_rows<NR>(acc, (int)cur_rb * GEMV_ROWS + warp * GEMV_ROWS_PER_WARP, n, lane, out, scale);
      cur_rb = rb;
    }
    const int cb = cc * chunk;
    const int nquad = min(chunk, ld - cb) / 4;
    float fh[GEMV_ROWS_PER_WARP][NR][2], fl[GEMV_ROWS_PER_WARP][NR][2];
#pragma unroll
    for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
      for (int r = 0; r < NR; ++r) fh[a][r][0] = fh[a][r][1] = fl[a][r][0] = fl[a][r][1] = 0.f;
    const float4* rh[GEMV_ROWS_PER_WARP];
    const float4* rl[GEMV_ROWS_PER_WARP];
#pragma unroll
    for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
      const size_t off = (size_t)min(row0 + a, n - 1) * ld + cb;
      rh[a] = reinterpret_cast<const float4*>(Mhi + off);
      rl[a] = reinterpret_cast<const float4*>(Mlo + off);
    }
#pragma unroll 2
    for (int q = lane; q < nquad; q += 32) {
      float4 mh[GEMV_ROWS_PER_WARP], ml[GEMV_ROWS_PER_WARP];
#pragma unroll
      for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
        const bool ok = row0 + a < n;
        mh[a] = ok ? ld_stream(rh[a] + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (FF) ml[a] = ok ? ld_stream(rl[a] + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const float4* xr = reinterpret_cast<const float4*>(xh + (size_t)r * ld + cb);
        const float4 x0 = __ldg(xr + 2 * q), x1 = __ldg(xr + 2 * q + 1);
        if (!FF) {
#pragma unroll
          for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
            float re = fh[a][r][0], im = fh[a][r][1];
            re = fmaf(mh[a].x, x0.x, re);
            im = fmaf(mh[a].x, x0.y, im);
            re = fmaf(mh[a].y, x0.z, re);
            im = fmaf(mh[a].y, x0.w, im);
            re = fmaf(mh[a].z, x1.x, re);
            im = fmaf(mh[a].z, x1.y, im);
            re = fmaf(mh[a].w, x1.z, re);
            im = fmaf(mh[a].w, x1.w, im);
            fh[a][r][0] = re;
            fh[a][r][1] = im;
          }
        } else {
          const float4* lr = reinterpret_cast<const float4*>(xl + (size_t)r * ld + cb);
          const float4 l0 = __ldg(lr + 2 * q), l1 = __ldg(lr + 2 * q + 1);
#pragma unroll
          for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
            // (mh + ml)(xh + xl): mh*xh exact in float-float, mh*xl + ml*xh folded into the low word
            ff_mac(fh[a][r][0], fl[a][r][0], mh[a].x, x0.x, l0.x);
            ff_mac(fh[a][r][1], fl[a][r][1], mh[a].x, x0.y, l0.y);
            ff_mac(fh[a][r][0], fl[a][r][0], mh[a].y, x0.z, l0.z);
            ff_mac(fh[a][r][1], fl[a][r][1], mh[a].y, x0.w, l0.w);
            ff_mac(fh[a][r][0], fl[a][r][0], mh[a].z, x1.x, l1.x);
            ff_mac(fh[a][r][1], fl[a][r][1], mh[a].z, x1.y, l1.y);
            ff_mac(fh[a][r][0], fl[a][r][0], mh[a].w, x1.z, l1.z);
            ff_mac(fh[a][r][1], fl[a][r][1], mh[a].w, x1.w, l1.w);
            fl[a][r][0] = fmaf(ml[a].x, x0.x, fl[a][r][0]);
            fl[a][r][1] = fmaf(ml[a].x, x0.y, fl[a][r][1]);
            fl[a][r][0] = fmaf(ml[a].y, x0.z, fl[a][r][0]);
            fl[a][r][1] = fmaf(ml[a].y, x0.w, fl[a][r][1]);
            fl[a][r][0] = fmaf(ml[a].z, x1.x, fl[a][r][0]);
            fl[a][r][1] = fmaf(ml[a].z, x1.y, fl[a][r][1]);
            fl[a][r][0] = fmaf(ml[a].w, x1.z, fl[a][r][0]);
            fl[a][r][1] = fmaf(ml[a].w, x1.w, fl[a][r][1]);
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        acc[a][r][0] += (double)fh[a][r][0] + (double)fl[a][r][0];
        acc[a][r][1] += (double)fh[a][r][1] + (double)fl[a][r][1];
      }
  }
  if (cur_rb >= 0) flush_rows<NR>(acc, (int)cur_rb * GEMV_ROWS + warp * GEMV_ROWS_PER_WARP, n, lane, out, scale);
}

// persistent grid: SMs x resident CTAs of this kernel (cached per kernel and device)
template <class K>
int persistent_grid(K kernel) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_pair(reinterpret_cast<const void*>(kernel), dev);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, GEMV_WARPS * 32, 0);
  const int g = std::max(1, sms * std::max(1, per));
  cache[key] = g;
  return g;
}

// grid of a persistent GEMV launch: the work units, capped at SMs x CTAs per SM (the plan's
// count, else the occupancy maximum)
template <class K>
long long gemv_grid(K kernel, long long units, const GemvScratch& w) {
  long long cap = persistent_grid(kernel);
  if (w.ctas_per_sm > 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cap = (long long)std::max(1, sms) * w.ctas_per_sm;
  }
  return std::max(1LL, std::min(units, cap));
}

int gemv_chunk(const GemvScratch& w) { return w.chunk > 0 ? w.chunk : GEMV_CHUNK; }

// x -> FP32 hi (and lo) in w.xh / w.xl; y zeroed unless the product accumulates into it; the
// product that follows adds scale times its partial sums into y
cudaError_t gemv_prep(const double2* x, double2* y, int n, int ld, int nr, bool ff, bool accumulate, double scale,
                      GemvScratch& w, cudaStream_t s) {
  w.out = y;
  w.scale = scale;
  dim3 grid(std::min((ld + 255) / 256, 4 * 152), nr);
  gemv_prep_kernel<<<grid, 256, 0, s>>>(x, n, ld, nr, w.xh, ff ? w.xl : nullptr, accumulate ? nullptr : y);
  return cudaGetLastError();
}

template <int NR>
cudaError_t gemv_c64_dispatch(const float2* M, int ld, int n, bool conj, GemvMode mode, GemvScratch& w,
                              cudaStream_t s) {
  const int rowblocks = (n + GEMV_ROWS - 1) / GEMV_ROWS;
  const int chunk = gemv_chunk(w);
  const int upr = (ld + chunk - 1) / chunk;
  const long long units = (long long)rowblocks * upr;
  const bool stream = mode == GEMV_F32 && NR <= 2 && w.chunk == 0 && w.ctas_per_sm == 0 && w.err && w.symmetric;
  // algorithmic bytes: the matrix (its upper triangle where the symmetric kernel reads only that)
  // plus the vectors
  const double mbytes = stream ? 4.0 * n * (n + 1.0) : 8.0 * n * n;
  ProfScope prof(mode == GEMV_FF ? "gemv_c64_ff" : "gemv_c64_f32", mbytes + 32.0 * n * NR, 8.0 * n * n * NR, s);
  if (stream) return gemv_stream_c64<NR <= 1 ? 1 : 2>(M, ld, n, conj, w, s);
  if (NR == 1 && mode == GEMV_FF && w.chunk == 0 && w.ctas_per_sm == 0 && w.err) return gemv_stream_c64_ff(M, ld, n, conj, w, s);
#define RF_LAUNCH_C(FFV, CJ)                                                                      \
  {                                                                                               \
    auto k = gemv_c64_kernel<NR, FFV, CJ>;                                                        \
    const int grid = (int)gemv_grid(k, units, w);                                                 \
    k<<<grid, GEMV_WARPS * 32, 0, s>>>(M, ld, n, w.xh, w.xl, w.out, w.scale, units, upr, chunk);           \
  }
  if (mode == GEMV_FF) {
    if (conj) RF_LAUNCH_C(true, true) else RF_LAUNCH_C(true, false)
  } else {
    if (conj) RF_LAUNCH_C(false, true) else RF_LAUNCH_C(false, false)
  }
#undef RF_LAUNCH_C
  return cudaGetLastError();
}

template <int NR>
cudaError_t gemv_r32_dispatch(const float* Mhi, const float* Mlo, int ld, int n, GemvMode mode, GemvScratch& w,
                              cudaStream_t s) {
  const int rowblocks = (n + GEMV_ROWS - 1) / GEMV_ROWS;
  const int chunk = gemv_chunk(w);
  const int upr = (ld + chunk - 1) / chunk;
  const long long units = (long long)rowblocks * upr;
  const bool stream = mode == GEMV_F32 && NR <= 2 && w.chunk == 0 && w.ctas_per_sm == 0 && w.err && w.symmetric;
  const double mbytes = mode == GEMV_FF ? 8.0 * n * n : (stream ? 2.0 * n * (n + 1.0) : 4.0 * n * n);
  ProfScope prof(mode == GEMV_FF ? "gemv_r32_ff" : "gemv_r32_f32", mbytes + 32.0 * n * NR, 4.0 * n * n * NR, s);
  if (stream) return gemv_stream_r32<NR <= 1 ? 1 : 2>(Mhi, ld, n, w, s);
  if (mode == GEMV_FF) {
    auto k = gemv_r32_kernel<NR, true>;
    const int grid = (int)gemv_grid(k, units, w);
    k<<<grid, GEMV_WARPS * 32, 0, s>>>(Mhi, Mlo, ld, n, w.xh, w.xl, w.out, w.scale, units, upr, chunk);
  } else {
    auto k = gemv_r32_kernel<NR, false>;
    const int grid = (int)gemv_grid(k, units, w);
    k<<<grid, GEMV_WARPS * 32, 0, s>>>(Mhi, Mlo, ld, n, w.xh, w.xl, w.out, w.scale, units, upr, chunk);
  }
  return cudaGetLastError();
}

}  // namespace

int padded_ld(int n) { return (n + 63) / 64 * 64; }

namespace {
std::mutex g_pool_mu;
std::set<int> g_pool_ready;  // devices whose default pool keeps freed memory
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_ready.count(dev)) {
      cudaMemPool_t pool;
      if ((e = cudaDeviceGetDefaultMemPool(&pool, dev)) != cudaSuccess) return e;
      uint64_t keep = UINT64_MAX;
      if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
      g_pool_ready.insert(dev);
    }
  }
  // On the legacy default stream: the allocation is ordered after all earlier work of the blocking
  // streams and before all their later work, so no host synchronisation is needed (non-blocking
  // caller streams are ordered explicitly by the C ABI's entry points).
  return cudaMallocAsync(p, std::max<size_t>(bytes, 1), 0);
}

cudaError_t dev_free(void* p) {
  if (!p) return cudaSuccess;
  // Freed in the order of the legacy default stream: after every kernel already queued on the
  // blocking streams (those that may still read p); the entry points make the legacy stream wait
  // for the non-blocking streams an operator was used on before they free its memory.
  return cudaFreeAsync(p, 0);
}

void dev_pool_trim() {
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    cudaDeviceSynchronize();
    cudaMemPoolTrimTo(pool, 0);
  }
}

// y = scale * op(M) x (+ y) for a real scale: prep (x -> FP32 hi/lo, y zeroed unless it
// accumulates), then the GEMV, whose CTAs add scale times their FP64 partial sums into y.
cudaError_t gemv_c64(const float2* M, int n, const double2* x, double2* y, int nrhs, bool conjugate, double2 scale,
                     bool accumulate, GemvMode mode, GemvScratch& w, cudaStream_t s, bool fed) {
  const int ld = padded_ld(n);
  if (scale.y != 0.0) return cudaErrorInvalidValue;
  if (fed) {  // split and zeroed y written by the producer of x
    if ((nrhs != 1 && nrhs != 2 && nrhs != 4) || n > w.cap_n || ld > w.cap_ld || nrhs > w.cap_cols ||
        (mode == GEMV_FF && !w.xl))
      return cudaErrorInvalidValue;
    w.out = y;
    w.scale = scale.x;
    if (nrhs == 4) return gemv_c64_dispatch<4>(M, ld, n, conjugate, mode, w, s);
    if (nrhs == 2) return gemv_c64_dispatch<2>(M, ld, n, conjugate, mode, w, s);
    return gemv_c64_dispatch<1>(M, ld, n, conjugate, mode, w, s);
  }
  cudaError_t err = cudaSuccess;
  for (int r = 0; r < nrhs && err == cudaSuccess;) {
    const int nr = std::min(4, nrhs - r) >= 4 ? 4 : (nrhs - r >= 2 ? 2 : 1);
    if (n > w.cap_n || ld > w.cap_ld || nr > w.cap_cols) return cudaErrorInvalidValue;
    const double2* xr = x + (size_t)r * n;
    double2* yr = y + (size_t)r * n;
    if ((err = gemv_prep(xr, yr, n, ld, nr, mode == GEMV_FF, accumulate, scale.x, w, s)) != cudaSuccess) break;
    if (nr == 4) err = gemv_c64_dispatch<4>(M, ld, n, conjugate, mode, w, s);
    else if (nr == 2) err = gemv_c64_dispatch<2>(M, ld, n, conjugate, mode, w, s);
    else err = gemv_c64_dispatch<1>(M, ld, n, conjugate, mode, w, s);
    r += nr;
  }
  return err;
}

// The same complex GEMV without profiling events and without the cached grid map: it
// performs no allocation of any kind (device, driver or host heap).
cudaError_t gemv_c64_plain(const float2* M, int n, const double2* x, double2* y, int nrhs, bool conjugate,
                           GemvMode mode, GemvScratch& w, cudaStream_t s) {
  const int ld = padded_ld(n);
  int dev = 0, sms = 0, per = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int r = 0; r < nrhs && err == cudaSuccess;) {
    const int nr = nrhs - r >= 4 ? 4 : (nrhs - r >= 2 ? 2 : 1);
    if (n > w.cap_n || ld > w.cap_ld || nr > w.cap_cols) return cudaErrorInvalidValue;
    const double2* xr = x + (size_t)r * n;
    double2* yr = y + (size_t)r * n;
    if ((err = gemv_prep(xr, yr, n, ld, nr, mode == GEMV_FF, false, 1.0, w, s)) != cudaSuccess) break;
    const int rowblocks = (n + GEMV_ROWS - 1) / GEMV_ROWS;
    const int upr = (ld + GEMV_CHUNK - 1) / GEMV_CHUNK;
    const long long units = (long long)rowblocks * upr;
#define RF_PLAIN(NRV, FFV, CJ)                                                                   \
  {                                                                                              \
    auto k = gemv_c64_kernel<NRV, FFV, CJ>;                                                      \
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, GEMV_WARPS * 32, 0)) !=     \
        cudaSuccess)                                                                             \
      break;                                                                                     \
    const int grid = (int)std::min<long long>(units, (long long)sms * std::max(1, per));         \
    k<<<grid, GEMV_WARPS * 32, 0, s>>>(M, ld, n, w.xh, w.xl, w.out, w.scale, units, upr, GEMV_CHUNK);     \
  }
#define RF_PLAIN_NR(NRV)                                           \
  if (mode == GEMV_FF) {                                           \
    if (conjugate) RF_PLAIN(NRV, true, true) else RF_PLAIN(NRV, true, false)   \
  } else {                                                         \
    if (conjugate) RF_PLAIN(NRV, false, true) else RF_PLAIN(NRV, false, false) \
  }
    if (nr == 4) {
      RF_PLAIN_NR(4)
    } else if (nr == 2) {
      RF_PLAIN_NR(2)
    } else {
      RF_PLAIN_NR(1)
    }
#undef RF_PLAIN_NR
#undef RF_PLAIN
    if ((err = cudaGetLastError()) != cudaSuccess) break;
    r += nr;
  }
  return err;
}

cudaError_t gemv_r32(const float* Mhi, const float* Mlo, int n, const double2* x, double2* y, int nrhs, double scale,
                     bool accumulate, GemvMode mode, GemvScratch& w, cudaStream_t s, bool fed) {
  const int ld = padded_ld(n);
  if (fed) {  // split and zeroed y written by the producer of x
    if ((nrhs != 1 && nrhs != 2 && nrhs != 4) || n > w.cap_n || ld > w.cap_ld || nrhs > w.cap_cols ||
        (mode == GEMV_FF && !w.xl))
      return cudaErrorInvalidValue;
    w.out = y;
    w.scale = scale;
    if (nrhs == 4) return gemv_r32_dispatch<4>(Mhi, Mlo, ld, n, mode, w, s);
    if (nrhs == 2) return gemv_r32_dispatch<2>(Mhi, Mlo, ld, n, mode, w, s);
    return gemv_r32_dispatch<1>(Mhi, Mlo, ld, n, mode, w, s);
  }
  cudaError_t err = cudaSuccess;
  for (int r = 0; r < nrhs && err == cudaSuccess;) {
    const int nr = nrhs - r >= 4 ? 4 : (nrhs - r >= 2 ? 2 : 1);
    if (n > w.cap_n || ld > w.cap_ld || nr > w.cap_cols) return cudaErrorInvalidValue;
    const double2* xr = x + (size_t)r * n;
    double2* yr = y + (size_t)r * n;
    if ((err = gemv_prep(xr, yr, n, ld, nr, mode == GEMV_FF, accumulate, scale, w, s)) != cudaSuccess) break;
    if (nr == 4) err = gemv_r32_dispatch<4>(Mhi, Mlo, ld, n, mode, w, s);
    else if (nr == 2) err = gemv_r32_dispatch<2>(Mhi, Mlo, ld, n, mode, w, s);
    else err = gemv_r32_dispatch<1>(Mhi, Mlo, ld, n, mode, w, s);
    r += nr;
  }
  return err;
}

// ---------------------------------------------------------------- sparse transforms
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// element i of column r (length n) of a vector a GEMV reads next: its split (as gemv_prep_kernel
// forms it) and the GEMV's zeroed output
__device__ __forceinline__ void feed_out(const GemvFeed& f, int r, int i, int n, double2 v) {
  if (f.xh) {
    const float2 h = make_float2((float)v.x, (float)v.y);
    f.xh[(size_t)r * f.ld + i] = h;
    if (f.xl) f.xl[(size_t)r * f.ld + i] = make_float2((float)(v.x - (double)h.x), (float)(v.y - (double)h.y));
  }
  if (f.y) f.y[(size_t)r * n + i] = make_double2(0.0, 0.0);
  if (f.y2) f.y2[(size_t)r * n + i] = make_double2(0.0, 0.0);
}
// the split's padding n <= i < ld (the grids cover ld: 256-thread blocks over n, ld = n rounded to 64)
__device__ __forceinline__ void feed_pad(const GemvFeed& f, int r, int i) {
  if (f.xh && i < f.ld) {
    f.xh[(size_t)r * f.ld + i] = make_float2(0.f, 0.f);
    if (f.xl) f.xl[(size_t)r * f.ld + i] = make_float2(0.f, 0.f);
  }
}

__global__ void sigma_t_kernel(const int32_t* __restrict__ cell_edges, const int8_t* __restrict__ cell_sign, int nc,
                               int ne, const double2* __restrict__ x, double2* __restrict__ out, GemvFeed f) {
  RF_COUNT_LAUNCH();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= nc) {
    feed_pad(f, r, c);
    return;
  }
  const double2* xr = x + (size_t)r * ne;
  double2 acc = make_double2(0.0, 0.0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int e = cell_edges[3 * c + i];
    if (e < 0) continue;  // a boundary edge of an open surface: no RWG function
    const double sg = (double)cell_sign[3 * c + i];
    const double2 v = xr[e];
    acc.x += sg * v.x;
    acc.y += sg * v.y;
  }
  out[(size_t)r * nc + c] = acc;
  feed_out(f, r, c, nc, acc);
}

__global__ void lambda_t_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ edge,
                                const int8_t* __restrict__ sign, int nv, int ne, const double2* __restrict__ x,
                                double2* __restrict__ out, GemvFeed f) {
  RF_COUNT_LAUNCH();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (v >= nv) {
    feed_pad(f, r, v);
    return;
  }
  const double2* xr = x + (size_t)r * ne;
  double2 acc = make_double2(0.0, 0.0);
  for (int q = ptr[v]; q < ptr[v + 1]; ++q) {
    const double sg = (double)sign[q];
    const double2 val = xr[edge[q]];
    acc.x += sg * val.x;
    acc.y += sg * val.y;
  }
  out[(size_t)r * nv + v] = acc;
  feed_out(f, r, v, nv, acc);
}

__global__ void lap_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const double* __restrict__ val, int nc, const double2* __restrict__ z,
                           double2* __restrict__ out, GemvFeed f) {
  RF_COUNT_LAUNCH();
  // Sigma^T Sigma z (CSR: the cell's RWG edge count on the diagonal, -1 per shared edge)
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= nc) {
    feed_pad(f, r, c);
    return;
  }
  const double2* zr = z + (size_t)r * nc;
  double2 acc = make_double2(0.0, 0.0);
  for (int q = ptr[c]; q < ptr[c + 1]; ++q) {
    const int d = col[q];
    const double w = val[q];
    acc.x += w * zr[d].x;
    acc.y += w * zr[d].y;
  }
  out[(size_t)r * nc + c] = acc;
  feed_out(f, r, c, nc, acc);
}

__global__ void edge_combo_kernel(const int32_t* __restrict__ edge_cells, const int32_t* __restrict__ edge_loops,
                                  int ne, int nc, int nv, EdgeCombo cb, double2* __restrict__ out, GemvFeed f) {
  RF_COUNT_LAUNCH();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (n >= ne) {
    feed_pad(f, r, n);
    return;
  }
  double2 acc = make_double2(0.0, 0.0);
  const size_t oe = (size_t)r * ne;
  if (cb.x) {
    const double2 t = cmul(cb.a, cb.x[oe + n]);
    acc.x += t.x;
    acc.y += t.y;
  }
  const int cp = edge_cells[2 * n], cm = edge_cells[2 * n + 1];
  if (cb.zs) {
    const double2 p = cb.zs[(size_t)r * nc + cp], m = cb.zs[(size_t)r * nc + cm];
    const double2 t = cmul(cb.b, make_double2(p.x - m.x, p.y - m.y));
    acc.x += t.x;
    acc.y += t.y;
  }
  if (cb.zs2) {
    const double2 p = cb.zs2[(size_t)r * nc + cp], m = cb.zs2[(size_t)r * nc + cm];
    const double2 t = cmul(cb.d, make_double2(p.x - m.x, p.y - m.y));
    acc.x += t.x;
    acc.y += t.y;
  }
  if (cb.zl) {
    // loop indices of the edge ends; an end on the boundary of an open surface has none
    const int v1 = edge_loops[2 * n], v2 = edge_loops[2 * n + 1];
    const double2 zero = make_double2(0.0, 0.0);
    const double2 p = v1 >= 0 ? cb.zl[(size_t)r * nv + v1] : zero, m = v2 >= 0 ? cb.zl[(size_t)r * nv + v2] : zero;
    const double2 t = cmul(cb.c, make_double2(p.x - m.x, p.y - m.y));
    acc.x += t.x;
    acc.y += t.y;
  }
  if (cb.w) {
    const double2 t = cmul(cb.e, cb.w[oe + n]);
    acc.x += t.x;
    acc.y += t.y;
  }
  out[oe + n] = acc;
  feed_out(f, r, n, ne, acc);
}

__global__ void column_sum_kernel(const double2* __restrict__ w, int n, double* __restrict__ sums) {
  RF_COUNT_LAUNCH();
  // sums[2r], sums[2r+1] += column r of w (block per (chunk, column))
  const int r = blockIdx.y;
  double sx = 0.0, sy = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    sx += w[(size_t)r * n + i].x;
    sy += w[(size_t)r * n + i].y;
  }
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[2 * r], sx);
    atomicAdd(&sums[2 * r + 1], sy);
  }
}

__global__ void star_middle_kernel(const double* __restrict__ area, int nc, const double2* __restrict__ z,
                                   const double2* __restrict__ w, const double* __restrict__ sums, double scale,
                                   double2* __restrict__ q, GemvFeed f) {
  RF_COUNT_LAUNCH();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= nc) {
    feed_pad(f, r, c);
    return;
  }
  const size_t o = (size_t)r * nc + c;
  double2 v = z[o];
  if (w) {
    const double mx = sums[2 * r] / nc, my = sums[2 * r + 1] / nc;
    v.x += w[o].x - mx;
    v.y += w[o].y - my;
  }
  const double fa = scale * area[c];
  q[o] = make_double2(fa * v.x, fa * v.y);
  feed_out(f, r, c, nc, q[o]);
}

__global__ void cell_combo_kernel(int nc, const double2* __restrict__ z, double2 a, const double2* __restrict__ w,
                                  double2 b, const double* __restrict__ sums, double2* __restrict__ q) {
  RF_COUNT_LAUNCH();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= nc) return;
  const size_t o = (size_t)r * nc + c;
  double2 v = make_double2(0.0, 0.0);
  if (z) v = cmul(a, z[o]);
  if (w) {
    const double2 d = make_double2(w[o].x - sums[2 * r] / nc, w[o].y - sums[2 * r + 1] / nc);
    const double2 t = cmul(b, d);
    v.x += t.x;
    v.y += t.y;
  }
  q[o] = v;
}

}  // namespace

cudaError_t cell_combo(const DeviceGeometry& g, const double2* z, double2 a, const double2* w, double2 b, double2* q,
                       int nrhs, double* scratch_mean, cudaStream_t s) {
  if (w) {
    cudaError_t e = cudaMemsetAsync(scratch_mean, 0, sizeof(double) * 2 * nrhs, s);
    if (e != cudaSuccess) return e;
    dim3 grid(std::min(64, (g.nc + 255) / 256), nrhs);
    column_sum_kernel<<<grid, 256, 0, s>>>(w, g.nc, scratch_mean);
  }
  dim3 grid((g.nc + 255) / 256, nrhs);
  cell_combo_kernel<<<grid, 256, 0, s>>>(g.nc, z, a, w, b, scratch_mean, q);
  return cudaGetLastError();
}

cudaError_t sigma_t(const DeviceGeometry& g, const double2* x, double2* out, int nrhs, cudaStream_t s,
                    const GemvFeed& feed) {
  dim3 grid((g.nc + 255) / 256, nrhs);
  sigma_t_kernel<<<grid, 256, 0, s>>>(g.cell_edges, g.cell_sign, g.nc, g.ne, x, out, feed);
  return cudaGetLastError();
}

cudaError_t lambda_t(const DeviceGeometry& g, const double2* x, double2* out, int nrhs, cudaStream_t s,
                     const GemvFeed& feed) {
  dim3 grid((g.nv + 255) / 256, nrhs);
  lambda_t_kernel<<<grid, 256, 0, s>>>(g.vtx_ptr, g.vtx_edge, g.vtx_sign, g.nv, g.ne, x, out, feed);
  return cudaGetLastError();
}

cudaError_t lap_apply(const DeviceGeometry& g, const double2* z, double2* out, int nrhs, cudaStream_t s,
                      const GemvFeed& feed) {
  dim3 grid((g.nc + 255) / 256, nrhs);
  lap_kernel<<<grid, 256, 0, s>>>(g.lap_ptr, g.lap_col, g.lap_val, g.nc, z, out, feed);
  return cudaGetLastError();
}

cudaError_t edge_combo(const DeviceGeometry& g, const EdgeCombo& c, double2* out, int nrhs, cudaStream_t s,
                       const GemvFeed& feed) {
  dim3 grid((g.ne + 255) / 256, nrhs);
  edge_combo_kernel<<<grid, 256, 0, s>>>(g.edge_cells, g.edge_loops, g.ne, g.nc, g.nv, c, out, feed);
  return cudaGetLastError();
}

cudaError_t star_middle(const DeviceGeometry& g, const double2* z, const double2* w, double scale, double2* q,
                        int nrhs, double* scratch_mean, cudaStream_t s, const GemvFeed& feed) {
  if (w) {
    cudaError_t e = cudaMemsetAsync(scratch_mean, 0, sizeof(double) * 2 * nrhs, s);
    if (e != cudaSuccess) return e;
    dim3 grid(std::min(64, (g.nc + 255) / 256), nrhs);
    column_sum_kernel<<<grid, 256, 0, s>>>(w, g.nc, scratch_mean);
  }
  dim3 grid((g.nc + 255) / 256, nrhs);
  star_middle_kernel<<<grid, 256, 0, s>>>(g.area64, g.nc, z, w, scratch_mean, scale, q, feed);
  return cudaGetLastError();
}

namespace {
__global__ void area_center_kernel(const double* __restrict__ area, int nc, const double2* __restrict__ w,
                                   const double* __restrict__ sums, double2* __restrict__ out) {
  RF_COUNT_LAUNCH();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= nc) return;
  const size_t o = (size_t)r * nc + c;
  const double mx = sums[2 * r] / nc, my = sums[2 * r + 1] / nc;
  out[o] = make_double2(area[c] * (w[o].x - mx), area[c] * (w[o].y - my));
}
__global__ void center_kernel(int nc, const double* __restrict__ sums, double2* __restrict__ out) {
  RF_COUNT_LAUNCH();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= nc) return;
  const size_t o = (size_t)r * nc + c;
  out[o].x -= sums[2 * r] / nc;
  out[o].y -= sums[2 * r + 1] / nc;
}
}  // namespace

cudaError_t pgp_apply(const DeviceGeometry& g, const double2* w, double2* out, int nrhs, double* scratch,
                      cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(double) * 4 * nrhs, s);
  if (e != cudaSuccess) return e;
  dim3 rgrid(std::min(64, (g.nc + 255) / 256), nrhs);
  dim3 grid((g.nc + 255) / 256, nrhs);
  column_sum_kernel<<<rgrid, 256, 0, s>>>(w, g.nc, scratch);
  area_center_kernel<<<grid, 256, 0, s>>>(g.area64, g.nc, w, scratch, out);
  column_sum_kernel<<<rgrid, 256, 0, s>>>(out, g.nc, scratch + 2 * nrhs);
  center_kernel<<<grid, 256, 0, s>>>(g.nc, scratch + 2 * nrhs, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- vector kernels
namespace {

constexpr int DOT_THREADS = 256;

__global__ void dot_kernel(const double2* __restrict__ a, const double2* __restrict__ b, int64_t n,
                           double2* __restrict__ out) {
  RF_COUNT_LAUNCH();
  // out[r] += a_r^H b_r (block per (chunk, column); out zeroed by the caller)
  const int r = blockIdx.y;
  double sx = 0.0, sy = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = a[(size_t)r * n + i], v = b[(size_t)r * n + i];
    sx += u.x * v.x + u.y * v.y;
    sy += u.x * v.y - u.y * v.x;
  }
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  __shared__ double red[DOT_THREADS / 32][2];
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = sx;
    red[threadIdx.x >> 5][1] = sy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tx = 0.0, ty = 0.0;
    for (int w = 0; w < DOT_THREADS / 32; ++w) {
      tx += red[w][0];
      ty += red[w][1];
    }
    atomicAdd(&out[r].x, tx);
    atomicAdd(&out[r].y, ty);
  }
}

__global__ void axpy_cols_kernel(const double* __restrict__ coef, double sgn, const double2* __restrict__ x,
                                 double2* __restrict__ y, int64_t n, const int* __restrict__ active) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const double a = sgn * coef[r];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = x[(size_t)r * n + i];
    double2 v = y[(size_t)r * n + i];
    v.x += a * u.x;
    v.y += a * u.y;
    y[(size_t)r * n + i] = v;
  }
}

__global__ void xpby_cols_kernel(const double2* __restrict__ x, const double* __restrict__ coef,
                                 double2* __restrict__ y, int64_t n, const int* __restrict__ active) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const double b = coef[r];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = x[(size_t)r * n + i];
    double2 v = y[(size_t)r * n + i];
    v.x = u.x + b * v.x;
    v.y = u.y + b * v.y;
    y[(size_t)r * n + i] = v;
  }
}

__global__ void copy_kernel(const double2* __restrict__ x, double2* __restrict__ y, int64_t n) {
  RF_COUNT_LAUNCH();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i];
}

__global__ void copy_scale_cols_kernel(const double2* __restrict__ x, const double* __restrict__ coef,
                                       double2* __restrict__ y, int64_t n) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.y;
  const double a = coef[r];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = x[(size_t)r * n + i];
    y[(size_t)r * n + i] = make_double2(a * u.x, a * u.y);
  }
}

__global__ void scale_kernel(double2* __restrict__ y, double2 a, int64_t n) {
  RF_COUNT_LAUNCH();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = y[i];
    y[i] = make_double2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x);
  }
}

__global__ void cg_alpha_kernel(const double* __restrict__ rr, const double2* __restrict__ pAp,
                                double* __restrict__ alpha, const int* __restrict__ active, int nrhs) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const double d = pAp[r].x;
  alpha[r] = (active && !active[r]) || d == 0.0 ? 0.0 : rr[r] / d;
}

__global__ void cg_beta_kernel(const double2* __restrict__ rr_new2, double* __restrict__ rr, double* __restrict__ beta,
                               const int* __restrict__ active, int nrhs) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  if (active && !active[r]) {
    beta[r] = 0.0;
    return;
  }
  const double nw = rr_new2[r].x;
  beta[r] = rr[r] == 0.0 ? 0.0 : nw / rr[r];
  rr[r] = nw;
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::min<int64_t>(b, 4 * 152);
}

}  // namespace

cudaError_t vec_dot(const double2* a, const double2* b, int64_t n, int nrhs, double2* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double2) * nrhs, s);
  if (e != cudaSuccess) return e;
  dim3 grid(std::min(grid_for(n), 152), nrhs);
  dot_kernel<<<grid, DOT_THREADS, 0, s>>>(a, b, n, out);
  return cudaGetLastError();
}

cudaError_t vec_axpy_cols(const double* coef, bool negate, const double2* x, double2* y, int64_t n, int nrhs,
                          const int* active, cudaStream_t s) {
  dim3 grid(grid_for(n), nrhs);
  axpy_cols_kernel<<<grid, 256, 0, s>>>(coef, negate ? -1.0 : 1.0, x, y, n, active);
  return cudaGetLastError();
}

cudaError_t vec_xpby_cols(const double2* x, const double* coef, double2* y, int64_t n, int nrhs, const int* active,
                          cudaStream_t s) {
  dim3 grid(grid_for(n), nrhs);
  xpby_cols_kernel<<<grid, 256, 0, s>>>(x, coef, y, n, active);
  return cudaGetLastError();
}

cudaError_t vec_copy(const double2* x, double2* y, int64_t n, cudaStream_t s) {
  copy_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t vec_copy_scale_cols(const double2* x, const double* coef, double2* y, int64_t n, int nrhs,
                               cudaStream_t s) {
  dim3 grid(grid_for(n), nrhs);
  copy_scale_cols_kernel<<<grid, 256, 0, s>>>(x, coef, y, n);
  return cudaGetLastError();
}

cudaError_t vec_scale(double2* y, double2 a, int64_t n, cudaStream_t s) {
  scale_kernel<<<grid_for(n), 256, 0, s>>>(y, a, n);
  return cudaGetLastError();
}

cudaError_t cg_scalars_alpha(const double* rr, const double2* pAp, double* alpha, const int* active, int nrhs,
                             cudaStream_t s) {
  cg_alpha_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(rr, pAp, alpha, active, nrhs);
  return cudaGetLastError();
}

cudaError_t cg_scalars_beta(const double2* rr_new2, double* rr, double* beta, const int* active, int nrhs,
                            cudaStream_t s) {
  cg_beta_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(rr_new2, rr, beta, active, nrhs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- dense inverse by block (P)CG
// X = A^{-1} B for the sparse SPD A (or, with project, the graph Laplacian restricted to
// 1^perp: B = I - 1 1^T / n, X = A^+ by the identity of Sec. 3.2), W columns at a time;
// every column runs its own (P)CG with its own scalars.  Arrays are row-major n x W so that
// consecutive threads read consecutive columns.  A column whose residual reached the
// tolerance is frozen: continuing CG on it after p^T A p has fallen to rounding level (or
// below zero on the singular Laplacian) makes the step explode.
namespace {

constexpr int BCG_COLS = 128;  // columns per thread block (64 threads x 2 adjacent columns)
constexpr int BCG_ROWS = 256;  // rows per thread block
constexpr int BCG_THREADS = 256;
constexpr int BCG_RLANES = BCG_THREADS / (BCG_COLS / 2);  // 4 interleaved row lanes

// Thread (column pair, row lane) of a block-CG kernel: columns c, c + 1 (c even), rows
// r0, r0 + 4, ... < r1.  Arrays are row-major n x W with W a multiple of 128.
struct RowIter {
  int c, r0, r1;
  __device__ RowIter(int n) {
    c = 2 * (blockIdx.x * (BCG_COLS / 2) + (threadIdx.x % (BCG_COLS / 2)));
    r0 = blockIdx.y * BCG_ROWS + threadIdx.x / (BCG_COLS / 2);
    r1 = min(n, (int)(blockIdx.y * BCG_ROWS + BCG_ROWS));
  }
  __device__ bool first() const { return blockIdx.y == 0 && threadIdx.x < BCG_COLS / 2; }
};

__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }

// columns c0 + c >= n (padding of the last block) get b = 0: they are frozen from the start
__global__ void bcg_init_kernel(int n, int W, int c0, bool project, double* __restrict__ X, double* __restrict__ R,
                                double* __restrict__ rr0) {
  RF_COUNT_LAUNCH();
  RowIter it(n);
  const double off = project ? 1.0 / n : 0.0;
  const bool v0 = c0 + it.c < n, v1 = c0 + it.c + 1 < n;
  double d0 = 0.0, d1 = 0.0;
  for (int i = it.r0; i < it.r1; i += BCG_RLANES) {
    const double b0 = v0 ? (i == c0 + it.c ? 1.0 : 0.0) - off : 0.0;
    const double b1 = v1 ? (i == c0 + it.c + 1 ? 1.0 : 0.0) - off : 0.0;
    const size_t o = (size_t)i * W + it.c;
    st2(X + o, make_double2(0.0, 0.0));
    st2(R + o, make_double2(b0, b1));
    d0 += b0 * b0;
    d1 += b1 * b1;
  }
  atomicAdd(&rr0[it.c], d0);
  atomicAdd(&rr0[it.c + 1], d1);
}

// out = A in (CSR); with acc, out += A in; with dot, dotp += in . out (per column)
__global__ void __launch_bounds__(BCG_THREADS)
bcg_spmm_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, const double* __restrict__ val,
                int n, int W, const double* __restrict__ in, double* __restrict__ out, int accumulate,
                double* __restrict__ dotp) {
  RF_COUNT_LAUNCH();
  RowIter it(n);
  double d0 = 0.0, d1 = 0.0;
#pragma unroll 4
  for (int i = it.r0; i < it.r1; i += BCG_RLANES) {
    double2 a = make_double2(0.0, 0.0);
    for (int q = ptr[i]; q < ptr[i + 1]; ++q) {
      const double v = val[q];
      const double2 x = ld2(in + (size_t)col[q] * W + it.c);
      a.x += v * x.x;
      a.y += v * x.y;
    }
    const size_t o = (size_t)i * W + it.c;
    if (accumulate) {
      const double2 p = ld2(out + o);
      a.x += p.x;
      a.y += p.y;
    }
    st2(out + o, a);
    if (dotp) {
      const double2 x = ld2(in + o);
      d0 += x.x * a.x;
      d1 += x.y * a.y;
    }
  }
  if (dotp) {
    atomicAdd(&dotp[it.c], d0);
    atomicAdd(&dotp[it.c + 1], d1);
  }
}

// X = w D^{-1} B
__global__ void __launch_bounds__(BCG_THREADS)
mg_smooth0_kernel(int n, int W, double w, const double* __restrict__ diag, const double* __restrict__ B,
                  double* __restrict__ X) {
  RF_COUNT_LAUNCH();
  RowIter it(n);
#pragma unroll 4
  for (int i = it.r0; i < it.r1; i += BCG_RLANES) {
    const size_t o = (size_t)i * W + it.c;
    const double f = w / diag[i];
    const double2 b = ld2(B + o);
    st2(X + o, make_double2(f * b.x, f * b.y));
  }
}

// T = B - A X   (mode 0)   or   T = X + w D^{-1} (B - A X)   (mode 1)
__global__ void __launch_bounds__(BCG_THREADS)
mg_resid_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, const double* __restrict__ val,
                const double* __restrict__ diag, int n, int W, double w, int mode, const double* __restrict__ B,
                const double* __restrict__ X, double* __restrict__ T) {
  RF_COUNT_LAUNCH();
  RowIter it(n);
#pragma unroll 4
  for (int i = it.r0; i < it.r1; i += BCG_RLANES) {
    double2 a = make_double2(0.0, 0.0);
    for (int q = ptr[i]; q < ptr[i + 1]; ++q) {
      const double v = val[q];
      const double2 x = ld2(X + (size_t)col[q] * W + it.c);
      a.x += v * x.x;
      a.y += v * x.y;
    }
    const size_t o = (size_t)i * W + it.c;
    const double2 b = ld2(B + o);
    double2 r = make_double2(b.x - a.x, b.y - a.y);
    if (mode != 0) {
      const double2 x = ld2(X + o);
      const double f = w / diag[i];
      r = make_double2(x.x + f * r.x, x.y + f * r.y);
    }
    st2(T + o, r);
  }
}

// Xc = Cinv Bc (dense m x m times m x W)
__global__ void mg_coarse_kernel(int m, int W, const double* __restrict__ Cinv, const double* __restrict__ Bc,
                                 double* __restrict__ Xc) {
  RF_COUNT_LAUNCH();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (c >= W || i >= m) return;
  double a = 0.0;
  for (int k = 0; k < m; ++k) a += Cinv[(size_t)i * m + k] * Bc[(size_t)k * W + c];
  Xc[(size_t)i * W + c] = a;
}

__device__ __forceinline__ bool frozen(const double* rr, const double* bb, double tol2, int c) {
  return rr[c] <= tol2 * bb[c];
}

// X += a P, R -= a AP, rr_new += R.R with a = rz / pAp (frozen columns untouched)
__global__ void __launch_bounds__(BCG_THREADS)
bcg_update_kernel(int n, int W, const double* __restrict__ rz, const double* __restrict__ rr,
                  const double* __restrict__ pAp, const double* __restrict__ bb, double tol2, double* __restrict__ X,
                  double* __restrict__ R, const double* __restrict__ P, const double* __restrict__ AP,
                  double* __restrict__ rr_new) {
  RF_COUNT_LAUNCH();
  RowIter it(n);
  const bool f0 = frozen(rr, bb, tol2, it.c), f1 = frozen(rr, bb, tol2, it.c + 1);
  if (it.first()) {
    if (f0) rr_new[it.c] = rr[it.c];
    if (f1) rr_new[it.c + 1] = rr[it.c + 1];
  }
  if (f0 && f1) return;
  const double a0 = f0 || !(pAp[it.c] > 0.0) ? 0.0 : rz[it.c] / pAp[it.c];
  const double a1 = f1 || !(pAp[it.c + 1] > 0.0) ? 0.0 : rz[it.c + 1] / pAp[it.c + 1];
  double d0 = 0.0, d1 = 0.0;
#pragma unroll 4
  for (int i = it.r0; i < it.r1; i += BCG_RLANES) {
    const size_t o = (size_t)i * W + it.c;
    double2 x = ld2(X + o), r = ld2(R + o);
    const double2 p = ld2(P + o), ap = ld2(AP + o);
    x.x += a0 * p.x;
    x.y += a1 * p.y;
    r.x -= a0 * ap.x;
    r.y -= a1 * ap.y;
    st2(X + o, x);
    st2(R + o, r);
    d0 += r.x * r.x;
    d1 += r.y * r.y;
  }
  if (!f0) atomicAdd(&rr_new[it.c], d0);
  if (!f1) atomicAdd(&rr_new[it.c + 1], d1);
}

// out += R.Z (per column)
__global__ void __launch_bounds__(BCG_THREADS)
bcg_dot_kernel(int n, int W, const double* __restrict__ R, const double* __restrict__ Z, double* __restrict__ out) {
  RF_COUNT_LAUNCH();
  RowIter it(n);
  double d0 = 0.0, d1 = 0.0;
#pragma unroll 4
  for (int i = it.r0; i < it.r1; i += BCG_RLANES) {
    const size_t o = (size_t)i * W + it.c;
    const double2 r = ld2(R + o), z = ld2(Z + o);
    d0 += r.x * z.x;
    d1 += r.y * z.y;
  }
  atomicAdd(&out[it.c], d0);
  atomicAdd(&out[it.c + 1], d1);
}

// P = Z + (rz_new / rz) P (frozen columns keep P); zero the accumulators of the next iteration
__global__ void __launch_bounds__(BCG_THREADS)
bcg_direction_kernel(int n, int W, const double* __restrict__ rz, const double* __restrict__ rz_new,
                     const double* __restrict__ rr_new, const double* __restrict__ bb, double tol2,
                     const double* __restrict__ Z, double* __restrict__ P, double* __restrict__ pAp,
                     double* __restrict__ zero_a, double* __restrict__ zero_b) {
  RF_COUNT_LAUNCH();
  RowIter it(n);
  if (it.first()) {
    for (int k = 0; k < 2; ++k) {
      pAp[it.c + k] = 0.0;
      zero_a[it.c + k] = 0.0;
      zero_b[it.c + k] = 0.0;
    }
  }
  const bool f0 = frozen(rr_new, bb, tol2, it.c), f1 = frozen(rr_new, bb, tol2, it.c + 1);
  if (f0 && f1) return;
  const double b0 = rz[it.c] > 0.0 ? rz_new[it.c] / rz[it.c] : 0.0;
  const double b1 = rz[it.c + 1] > 0.0 ? rz_new[it.c + 1] / rz[it.c + 1] : 0.0;
#pragma unroll 4
  for (int i = it.r0; i < it.r1; i += BCG_RLANES) {
    const size_t o = (size_t)i * W + it.c;
    const double2 z = ld2(Z + o);
    double2 p = ld2(P + o);
    if (!f0) p.x = z.x + b0 * p.x;
    if (!f1) p.y = z.y + b1 * p.y;
    st2(P + o, p);
  }
}

__global__ void bcg_colsum_kernel(int n, int W, const double* __restrict__ X, double* __restrict__ sums) {
  RF_COUNT_LAUNCH();
  RowIter it(n);
  double s0 = 0.0, s1 = 0.0;
  for (int i = it.r0; i < it.r1; i += BCG_RLANES) {
    const double2 x = ld2(X + (size_t)i * W + it.c);
    s0 += x.x;
    s1 += x.y;
  }
  atomicAdd(&sums[it.c], s0);
  atomicAdd(&sums[it.c + 1], s1);
}

// Xhi/Xlo[i, c0 + c] = X[i, c] - mean_c (projected case), split into FP32 hi + lo
__global__ void bcg_store_kernel(int n, int W, int c0, int ld, const double* __restrict__ X,
                                 const double* __restrict__ sums, bool project, float* __restrict__ Xhi,
                                 float* __restrict__ Xlo) {
  RF_COUNT_LAUNCH();
  RowIter it(n);
  for (int k = 0; k < 2; ++k) {
    const int cc = it.c + k;
    if (c0 + cc >= n) continue;
    const double mean = project ? sums[cc] / n : 0.0;
    for (int i = it.r0; i < it.r1; i += BCG_RLANES) {
      const double v = X[(size_t)i * W + cc] - mean;
      const float h = (float)v;
      Xhi[(size_t)i * ld + c0 + cc] = h;
      Xlo[(size_t)i * ld + c0 + cc] = (float)(v - (double)h);
    }
  }
}

// Xd[i, c0 + c] = X[i, c] - mean_c + 1/n  (an approximation of (L + 1 1^T / n)^{-1}, FP64)
__global__ void bcg_store_f64_kernel(int n, int W, int c0, long long ld, const double* __restrict__ X,
                                     const double* __restrict__ sums, double* __restrict__ Xd) {
  RF_COUNT_LAUNCH();
  RowIter it(n);
  for (int k = 0; k < 2; ++k) {
    const int cc = it.c + k;
    if (c0 + cc >= n) continue;
    const double shift = 1.0 / n - sums[cc] / n;
    for (int i = it.r0; i < it.r1; i += BCG_RLANES) Xd[(size_t)i * ld + c0 + cc] = X[(size_t)i * W + cc] + shift;
  }
}

struct DevLevel {
  int n = 0, nc = 0;
  double omega = 0.0;
  double* diag = nullptr;
  int32_t *A_ptr = nullptr, *A_col = nullptr, *P_ptr = nullptr, *P_col = nullptr, *R_ptr = nullptr, *R_col = nullptr;
  double *A_val = nullptr, *P_val = nullptr, *R_val = nullptr;
  double *B = nullptr, *X = nullptr, *T = nullptr;  // n x W work arrays (level 0 uses the CG arrays)
};

template <class T>
cudaError_t up(T** d, const std::vector<T>& h, std::vector<void*>& own) {
  cudaError_t e = dev_malloc(d, std::max<size_t>(1, h.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  own.push_back(*d);
  if (!h.empty()) e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

inline dim3 bgrid(int n, int w) { return dim3((w + BCG_COLS - 1) / BCG_COLS, (n + BCG_ROWS - 1) / BCG_ROWS); }
// every kernel of a column block runs over all W columns of the (padded) stride

}  // namespace

cudaError_t dense_inverse_block_cg(const int32_t* ptr, const int32_t* col, const double* val, int n, bool project,
                                   const AmgHierarchy* H, double tol, int max_iter, float* Xhi, float* Xlo,
                                   int* iters, cudaStream_t s, double* Xd) {
  const int ld = padded_ld(n);
  std::vector<void*> own;
  cudaError_t err = cudaSuccess;
  auto fail = [&](cudaError_t e) {
    for (void* p : own) dev_free(p);
    return e;
  };
  // device hierarchy
  std::vector<DevLevel> L;
  double* Cinv = nullptr;
  int m = 0;
  size_t coarse_rows = 0;  // sum of the rows of levels 1.. (plus the coarsest) for the work arrays
  if (H && !H->levels.empty()) {
    for (const AmgLevelHost& h : H->levels) {
      DevLevel d;
      d.n = h.n;
      d.nc = h.nc;
      d.omega = h.omega;
      if ((err = up(&d.diag, h.diag, own)) != cudaSuccess) return fail(err);
      if ((err = up(&d.A_ptr, h.A_ptr, own)) != cudaSuccess) return fail(err);
      if ((err = up(&d.A_col, h.A_col, own)) != cudaSuccess) return fail(err);
      if ((err = up(&d.A_val, h.A_val, own)) != cudaSuccess) return fail(err);
      if ((err = up(&d.P_ptr, h.P_ptr, own)) != cudaSuccess) return fail(err);
      if ((err = up(&d.P_col, h.P_col, own)) != cudaSuccess) return fail(err);
      if ((err = up(&d.P_val, h.P_val, own)) != cudaSuccess) return fail(err);
      if ((err = up(&d.R_ptr, h.R_ptr, own)) != cudaSuccess) return fail(err);
      if ((err = up(&d.R_col, h.R_col, own)) != cudaSuccess) return fail(err);
      if ((err = up(&d.R_val, h.R_val, own)) != cudaSuccess) return fail(err);
      L.push_back(d);
      coarse_rows += (size_t)h.nc;
    }
    m = H->coarse_n;
    if ((err = up(&Cinv, H->coarse_inv, own)) != cudaSuccess) return fail(err);
  }
  const bool mg = !L.empty();
  // column block width: bound the work arrays to about 24 GB
  const size_t fine_arrays = mg ? 6 : 4;
  const size_t per_col = sizeof(double) * (fine_arrays * (size_t)n + 3 * coarse_rows);
  const size_t cap = (size_t)24 << 30;
  const int n_pad = (n + BCG_COLS - 1) / BCG_COLS * BCG_COLS;  // all columns in one block when they fit
  int W = n_pad;
  if ((size_t)W * per_col > cap) W = std::max<int>(BCG_COLS, (int)(cap / per_col) / BCG_COLS * BCG_COLS);
  const size_t bytes = (size_t)n * W * sizeof(double);
  double *X, *R, *P = nullptr, *AP = nullptr, *Z = nullptr, *T0 = nullptr, *sc;
  const bool iterate = !(mg && max_iter == 0);  // max_iter 0 with a hierarchy: one V-cycle, no CG
  for (double** p : {&X, &R, &P, &AP}) {
    if (!iterate && (p == &P || p == &AP)) continue;
    if ((err = dev_malloc(p, bytes)) != cudaSuccess) return fail(err);
    own.push_back(*p);
  }
  if (mg) {
    for (double** p : {&Z, &T0}) {
      if ((err = dev_malloc(p, bytes)) != cudaSuccess) return fail(err);
      own.push_back(*p);
    }
    // levels 1.. hold B, X, T; the coarsest rhs / solution live in the last level's extra slots
    for (size_t l = 1; l < L.size(); ++l)
      for (double** p : {&L[l].B, &L[l].X, &L[l].T}) {
        if ((err = dev_malloc(p, (size_t)L[l].n * W * sizeof(double))) != cudaSuccess) return fail(err);
        own.push_back(*p);
      }
  }
  // coarsest arrays (m x W): rhs and solution
  double *Bc = nullptr, *Xc = nullptr;
  if (mg) {
    for (double** p : {&Bc, &Xc}) {
      if ((err = dev_malloc(p, (size_t)m * W * sizeof(double))) != cudaSuccess) return fail(err);
      own.push_back(*p);
    }
  }
  // scalars: rz ring (3W), rr ring (3W), pAp, bb, sums
  if ((err = dev_malloc(&sc, sizeof(double) * W * 9)) != cudaSuccess) return fail(err);
  own.push_back(sc);
  double* rzr = sc;
  double* rrr = sc + 3 * (size_t)W;
  double* pAp = sc + 6 * (size_t)W;
  double* bb = sc + 7 * (size_t)W;
  double* sums = sc + 8 * (size_t)W;
  std::vector<double> h_rr(W), h_bb(W);
  int worst_iters = 0;
  const double tol2 = tol * tol;
  for (int c0 = 0; c0 < n; c0 += W) {
    const int w = W;  // padding columns (c0 + c >= n) carry b = 0 and stay frozen
    const int wlive = std::min(W, n - c0);
    dim3 grid = bgrid(n, w);
    if ((err = cudaMemsetAsync(sc, 0, sizeof(double) * W * 9, s)) != cudaSuccess) return fail(err);
    bcg_init_kernel<<<grid, BCG_THREADS, 0, s>>>(n, w, c0, project, X, R, rrr);
    if ((err = cudaMemcpyAsync(bb, rrr, sizeof(double) * w, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return fail(err);
    if ((err = cudaMemcpyAsync(h_bb.data(), rrr, sizeof(double) * w, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return fail(err);
    // z0 = M r0 (one V(1,1) cycle; Z = R without a hierarchy), rz0 = r0.z0, p0 = z0
    auto precond = [&](double* Rin) -> double* {
      if (!mg) return Rin;
      ProfScope prof("factor_mg_vcycle", 0.0, 0.0, s);
      // levels: l = 0 .. nl-1 have operators; the coarse solve sits after the last
      const size_t nl = L.size();
      std::vector<double*> Bs(nl + 1), Xs(nl + 1), Ts(nl);
      for (size_t l = 0; l < nl; ++l) {
        Bs[l] = l == 0 ? Rin : L[l].B;
        Xs[l] = l == 0 ? Z : L[l].X;
        Ts[l] = l == 0 ? T0 : L[l].T;
      }
      Bs[nl] = Bc;
      Xs[nl] = Xc;
      for (size_t l = 0; l < nl; ++l) {
        DevLevel& v = L[l];
        mg_smooth0_kernel<<<bgrid(v.n, w), BCG_THREADS, 0, s>>>(v.n, w, v.omega, v.diag, Bs[l], Xs[l]);
        mg_resid_kernel<<<bgrid(v.n, w), BCG_THREADS, 0, s>>>(v.A_ptr, v.A_col, v.A_val, v.diag, v.n, w, v.omega,
                                                             0, Bs[l], Xs[l], Ts[l]);
        bcg_spmm_kernel<<<bgrid(v.nc, w), BCG_THREADS, 0, s>>>(v.R_ptr, v.R_col, v.R_val, v.nc, w, Ts[l], Bs[l + 1],
                                                               0, nullptr);
      }
      {
        dim3 g((w + 127) / 128, m);
        mg_coarse_kernel<<<g, 128, 0, s>>>(m, w, Cinv, Bs[nl], Xs[nl]);
      }
      for (size_t li = nl; li-- > 0;) {
        DevLevel& v = L[li];
        bcg_spmm_kernel<<<bgrid(v.n, w), BCG_THREADS, 0, s>>>(v.P_ptr, v.P_col, v.P_val, v.n, w, Xs[li + 1], Xs[li],
                                                              1, nullptr);
        mg_resid_kernel<<<bgrid(v.n, w), BCG_THREADS, 0, s>>>(v.A_ptr, v.A_col, v.A_val, v.diag, v.n, w, v.omega,
                                                             1, Bs[li], Xs[li], Ts[li]);
        // the smoothed iterate is in Ts[li]: swap the roles of the two arrays of this level
        if (li == 0) {
          std::swap(Z, T0);
        } else {
          std::swap(L[li].X, L[li].T);
        }
        Xs[li] = li == 0 ? Z : L[li].X;
      }
      return Z;
    };
    double* Zp = precond(R);
    double* Xres = X;  // the block stored below
    if (!iterate) Xres = Zp;  // no iteration: the result is one V-cycle applied to R0
    else {
      bcg_dot_kernel<<<grid, BCG_THREADS, 0, s>>>(n, w, R, Zp, rzr);
      if ((err = cudaMemcpyAsync(P, Zp, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return fail(err);
    }
    int it = 0;
    bool done = false;
    while (iterate && !done && it < max_iter) {
      double* rz = rzr + (size_t)(it % 3) * W;
      double* rz_new = rzr + (size_t)((it + 1) % 3) * W;
      double* rz_next = rzr + (size_t)((it + 2) % 3) * W;
      double* rr = rrr + (size_t)(it % 3) * W;
      double* rr_new = rrr + (size_t)((it + 1) % 3) * W;
      double* rr_next = rrr + (size_t)((it + 2) % 3) * W;
      {
        ProfScope prof("factor_bcg_spmm", 16.0 * n * w, 0.0, s);
        bcg_spmm_kernel<<<grid, BCG_THREADS, 0, s>>>(ptr, col, val, n, w, P, AP, 0, pAp);
      }
      {
        ProfScope prof("factor_bcg_update", 48.0 * n * w, 0.0, s);
        bcg_update_kernel<<<grid, BCG_THREADS, 0, s>>>(n, w, rz, rr, pAp, bb, tol2, X, R, P, AP, rr_new);
      }
      double* Zi = precond(R);
      bcg_dot_kernel<<<grid, BCG_THREADS, 0, s>>>(n, w, R, Zi, rz_new);
      {
        ProfScope prof("factor_bcg_direction", 24.0 * n * w, 0.0, s);
        bcg_direction_kernel<<<grid, BCG_THREADS, 0, s>>>(n, w, rz, rz_new, rr_new, bb, tol2, Zi, P, pAp, rz_next,
                                                          rr_next);
      }
      ++it;
      if (it % 8 == 0 || it == max_iter) {
        if ((err = cudaMemcpyAsync(h_rr.data(), rr_new, sizeof(double) * w, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
          return fail(err);
        if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return fail(err);
        double worst = 0.0;
        for (int c = 0; c < wlive; ++c) worst = std::max(worst, std::sqrt(h_rr[c] / std::max(h_bb[c], 1e-300)));
        done = worst <= tol;
      }
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return fail(err);
    worst_iters = std::max(worst_iters, it);
    if (project) {
      if ((err = cudaMemsetAsync(sums, 0, sizeof(double) * W, s)) != cudaSuccess) return fail(err);
      bcg_colsum_kernel<<<grid, BCG_THREADS, 0, s>>>(n, w, Xres, sums);
    }
    if (Xd && project)
      bcg_store_f64_kernel<<<grid, BCG_THREADS, 0, s>>>(n, w, c0, ld, Xres, sums, Xd);
    else
      bcg_store_kernel<<<grid, BCG_THREADS, 0, s>>>(n, w, c0, ld, Xres, sums, project, Xhi, Xlo);
    if ((err = cudaGetLastError()) != cudaSuccess) return fail(err);
  }
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return fail(err);
  *iters = worst_iters;
  return fail(cudaSuccess);
}

RF_LAUNCH_READER(launches_linalg)

}  // namespace rfcmp
