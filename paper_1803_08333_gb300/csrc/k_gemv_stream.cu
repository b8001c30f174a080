// Streaming GEMV: y = op(M) x for one or two FP32-mode columns with the matrix moved by the
// bulk-copy engine.
//
// The operator products of a single-right-hand-side solve are HBM bound: each application
// streams T_A, V and the factors once.  A register-pipelined GEMV keeps only as many bytes in
// flight as its unrolled loads allow; here one producer thread per CTA issues cp.async.bulk
// copies of whole row segments (8 rows x 512 complex64 or 1024 FP32 values, 32 KB per stage)
// together with the matching segment of x into a 4-stage shared-memory ring, so about 180 KB per
// SM are in flight whatever the consumers do.  Eight consumer warps each take one row of a
// stage, read it and x from shared memory (no global-memory latency on the consumer side),
// accumulate in FP32 within the segment and in compensated FP32 across segments, and release
// the stage through an mbarrier.  Work units (row block, column segment) are dealt to
// the persistent CTAs in contiguous ranges of equal size; a row block split between CTAs is
// combined by FP64 atomics.  Every wait is bounded and records an error code on timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "rfcmp_internal.h"
#include "tc_common.cuh"

namespace rfcmp {

namespace {

using tc::mbar_arrive;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::smem_u32;

constexpr int SROWS = 8;                 // rows per stage (one consumer warp each)
constexpr int SBYTES_ROW = 4096;         // bytes per row segment
constexpr int SSTAGES = 4;
constexpr int SMAT = SROWS * SBYTES_ROW;    // 32 KB of matrix per stage
constexpr int SXMAX = 2 * 8192;             // x segments per stage: up to 2 columns x 1024 complex
constexpr int SXI = 2 * 64;                 // x of the stage's 8 rows (symmetric kernel), up to 2 columns
constexpr int SSTAGE = SMAT + SXMAX + SXI;  // 48 KB + 128 B
constexpr int STHREADS = (SROWS + 1) * 32;  // consumers + producer warp
constexpr int SSMEM = SSTAGES * SSTAGE + 128;

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// REAL: M is FP32 (n x ld), else complex64; CONJ: conj(M) (complex only)
template <int NR, bool REAL, bool CONJ>
__global__ void __launch_bounds__(STHREADS, 1)
gemv_stream_kernel(const void* __restrict__ Mv, int ld, int n, const float2* __restrict__ xh,
                   double2* __restrict__ out, long long units, int upr, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SSTAGES * SSTAGE);
  uint64_t* empty = full + SSTAGES;
  constexpr int ESZ = REAL ? 4 : 8;          // bytes per matrix element
  constexpr int SEG = SBYTES_ROW / ESZ;      // elements per row segment
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < SSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], SROWS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const char* M = reinterpret_cast<const char*>(Mv);

  if (warp == SROWS) {
    if (lane == 0) {
      for (long long u = u0; u < u1; ++u) {
        const long long i = u - u0;
        const int s = (int)(i % SSTAGES);
        const long long round = i / SSTAGES;
        if (round > 0 && !mbar_wait(&empty[s], (uint32_t)((round - 1) & 1))) {
          atomicExch(err, 21);
          break;
        }
        const int rb = (int)(u / upr), cb = (int)(u % upr) * SEG;
        const int row0 = rb * SROWS, rows = min(SROWS, n - row0);
        const int cols = min(SEG, ld - cb);
        const uint32_t bytes = (uint32_t)cols * ESZ, xbytes = (uint32_t)cols * 8;
        mbar_expect_tx(&full[s], bytes * rows + xbytes * NR);
        uint8_t* st = smem + s * SSTAGE;
        for (int r = 0; r < rows; ++r)
          bulk_load(st + r * SBYTES_ROW, M + ((size_t)(row0 + r) * ld + cb) * ESZ, bytes, &full[s]);
        for (int r = 0; r < NR; ++r)
          bulk_load(st + SMAT + r * (SXMAX / 2), xh + (size_t)r * ld + cb, xbytes, &full[s]);
      }
      // the CTA must not end with copies into its shared memory in flight: wait (bounded) for
      // the last stages issued
      const long long cnt = u1 - u0;
      for (long long i = cnt > SSTAGES ? cnt - SSTAGES : 0; i < cnt; ++i)
        if (!mbar_wait(&full[i % SSTAGES], (uint32_t)((i / SSTAGES) & 1))) atomicExch(err, 23);
    }
    return;
  }

  // consumer warp: row `warp` of every stage.  Segment sums are FP32; across segments they are
  // added into an FP32 pair (hi, compensation) by an error-free two-sum, so the row sum keeps
  // about twice FP32 precision without FP64 arithmetic in the loop (GB300's FP64 pipe runs at
  // a small fraction of the FP32 rate); FP64 enters only at the per-row flush.
  float acc[NR][2], cmp[NR][2];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r][0] = acc[r][1] = cmp[r][0] = cmp[r][1] = 0.f;
  long long cur_rb = -1;
  bool ok = true;
  for (long long u = u0; u < u1 && ok; ++u) {
    const long long i = u - u0;
    const int s = (int)(i % SSTAGES);
    const uint32_t parity = (uint32_t)((i / SSTAGES) & 1);
    const int rb = (int)(u / upr), cb = (int)(u % upr) * SEG;
    if (rb != cur_rb) {
      if (cur_rb >= 0) {
        const int row = (int)cur_rb * SROWS + warp;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const double re = warp_sum_d((double)acc[r][0] + (double)cmp[r][0]);
          const double im = warp_sum_d((double)acc[r][1] + (double)cmp[r][1]);
          acc[r][0] = acc[r][1] = cmp[r][0] = cmp[r][1] = 0.f;
          if (lane == 0 && row < n) {
            double* o = reinterpret_cast<double*>(out + (size_t)r * n + row);
            atomicAdd(o, re);
            atomicAdd(o + 1, im);
          }
        }
      }
      cur_rb = rb;
    }
    ok = __all_sync(0xffffffffu, mbar_wait(&full[s], parity));
    if (!ok) {
      if (lane == 0) atomicExch(err, 22);
      break;
    }
    const int row = rb * SROWS + warp;
    if (row < n) {
      const float4* srow = reinterpret_cast<const float4*>(smem + s * SSTAGE + warp * SBYTES_ROW);
      const float4* sx = reinterpret_cast<const float4*>(smem + s * SSTAGE + SMAT);
      const int nq = min(SEG, ld - cb) * ESZ / 16;  // float4 per segment row
      float f[NR][2];
#pragma unroll
      for (int r = 0; r < NR; ++r) f[r][0] = f[r][1] = 0.f;
#pragma unroll 4
      for (int q = lane; q < nq; q += 32) {
        const float4 m = srow[q];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const float4* xr = sx + r * (SXMAX / 32);
          if (REAL) {
            // four real entries times four complex x values
            const float4 x0 = xr[2 * q];
            const float4 x1 = xr[2 * q + 1];
            float re = f[r][0], im = f[r][1];
            re = fmaf(m.x, x0.x, re);
            im = fmaf(m.x, x0.y, im);
            re = fmaf(m.y, x0.z, re);
            im = fmaf(m.y, x0.w, im);
            re = fmaf(m.z, x1.x, re);
            im = fmaf(m.z, x1.y, im);
            re = fmaf(m.w, x1.z, re);
            im = fmaf(m.w, x1.w, im);
            f[r][0] = re;
            f[r][1] = im;
          } else {
            // two complex entries (m.x + i m.y, m.z + i m.w) times two complex x values
            const float4 x4 = xr[q];
            const float my = CONJ ? -m.y : m.y, mw = CONJ ? -m.w : m.w;
            float re = f[r][0], im = f[r][1];
            re = fmaf(m.x, x4.x, re);
            re = fmaf(-my, x4.y, re);
            re = fmaf(m.z, x4.z, re);
            re = fmaf(-mw, x4.w, re);
            im = fmaf(m.x, x4.y, im);
            im = fmaf(my, x4.x, im);
            im = fmaf(m.z, x4.w, im);
            im = fmaf(mw, x4.z, im);
            f[r][0] = re;
            f[r][1] = im;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {  // two-sum: acc + f = t + e exactly
          const float a = acc[r][c], b = f[r][c], t = a + b, bb = t - a;
          cmp[r][c] += (a - (t - bb)) + (b - bb);
          acc[r][c] = t;
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  if (ok && cur_rb >= 0) {
    const int row = (int)cur_rb * SROWS + warp;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const double re = warp_sum_d((double)acc[r][0] + (double)cmp[r][0]);
      const double im = warp_sum_d((double)acc[r][1] + (double)cmp[r][1]);
      if (lane == 0 && row < n) {
        double* o = reinterpret_cast<double*>(out + (size_t)r * n + row);
        atomicAdd(o, re);
        atomicAdd(o + 1, im);
      }
    }
  }
}

// ---------------------------------------------------------------- symmetric matrices
// For a symmetric M (T_A, V and the factors all are) only the tiles that reach the diagonal or
// lie above it are read: a tile of 8 rows I x one segment J contributes y_I += M_IJ x_J (row part,
// entries j >= i) and y_J += M_IJ^T x_I (column part, entries j > i), so half the matrix bytes
// leave HBM.  Units run column-major over the upper triangle: segment c holds the row blocks
// 0 .. min(RB, P (c + 1)) - 1 (P = segment width / 8 rows), so the column part of a warp stays in
// registers across the row blocks of a segment and reaches y once per segment; the row part of a
// unit is reduced across the warp and added at once.  Warp w takes row w for the row part and the
// w-th eighth of the segment's columns (one float4 per lane and row) for the column part.
struct SymGeom {
  long long RB, P, S, cstar, base;  // row blocks, row blocks per segment step, segments, off() knee
  __host__ __device__ long long nrb(long long c) const { return c < cstar ? P * (c + 1) : RB; }
  // units before segment c
  __host__ __device__ long long off(long long c) const {
    return c <= cstar ? P * c * (c + 1) / 2 : base + (c - cstar) * RB;
  }
};

__host__ __device__ inline SymGeom sym_geom(int n, int ld, int seg) {
  SymGeom g;
  g.RB = (n + SROWS - 1) / SROWS;
  g.P = seg / SROWS;
  g.S = (ld + seg - 1) / seg;
  g.cstar = g.RB / g.P;  // segments c < cstar hold P (c + 1) <= RB row blocks
  g.base = g.P * g.cstar * (g.cstar + 1) / 2;
  return g;
}

template <int NR, bool REAL, bool CONJ>
__global__ void __launch_bounds__(STHREADS, 1)
gemv_sym_kernel(const void* __restrict__ Mv, int ld, int n, const float2* __restrict__ xh,
                double2* __restrict__ out, long long units, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SSTAGES * SSTAGE);
  uint64_t* empty = full + SSTAGES;
  constexpr int ESZ = REAL ? 4 : 8;
  constexpr int SEG = SBYTES_ROW / ESZ;
  constexpr int EPQ = 16 / ESZ;  // matrix entries per float4
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const SymGeom G = sym_geom(n, ld, SEG);
  const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < SSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], SROWS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (u0 >= u1) return;
  // segment and row block of unit u0 (binary search on off())
  long long c0 = 0;
  {
    long long lo = 0, hi = G.S - 1;
    while (lo < hi) {
      const long long mid = (lo + hi + 1) / 2;
      if (G.off(mid) <= u0) lo = mid;
      else hi = mid - 1;
    }
    c0 = lo;
  }
  const long long rb0 = u0 - G.off(c0);
  const char* M = reinterpret_cast<const char*>(Mv);

  if (warp == SROWS) {
    if (lane == 0) {
      long long c = c0, rb = rb0;
      for (long long u = u0; u < u1; ++u) {
        const long long i = u - u0;
        const int s = (int)(i % SSTAGES);
        const long long round = i / SSTAGES;
        if (round > 0 && !mbar_wait(&empty[s], (uint32_t)((round - 1) & 1))) {
          atomicExch(err, 24);
          break;
        }
        const int cb = (int)(c * SEG), row0 = (int)(rb * SROWS), rows = min(SROWS, n - row0);
        const int cols = min(SEG, ld - cb);
        const uint32_t bytes = (uint32_t)cols * ESZ, xbytes = (uint32_t)cols * 8;
        mbar_expect_tx(&full[s], bytes * rows + (xbytes + 64) * NR);
        uint8_t* st = smem + s * SSTAGE;
        for (int r = 0; r < rows; ++r)
          bulk_load(st + r * SBYTES_ROW, M + ((size_t)(row0 + r) * ld + cb) * ESZ, bytes, &full[s]);
        for (int r = 0; r < NR; ++r) {
          bulk_load(st + SMAT + r * (SXMAX / 2), xh + (size_t)r * ld + cb, xbytes, &full[s]);
          bulk_load(st + SMAT + SXMAX + r * 64, xh + (size_t)r * ld + row0, 64, &full[s]);  // x of the 8 rows
        }
        if (++rb == G.nrb(c)) {
          ++c;
          rb = 0;
        }
      }
      const long long cnt = u1 - u0;
      for (long long i = cnt > SSTAGES ? cnt - SSTAGES : 0; i < cnt; ++i)
        if (!mbar_wait(&full[i % SSTAGES], (uint32_t)((i / SSTAGES) & 1))) atomicExch(err, 25);
    }
    return;
  }

  // column part: lane's float4 q = 32 warp + lane of every row, EPQ entries, NR columns
  float ca[NR][EPQ][2], cc[NR][EPQ][2];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int e = 0; e < EPQ; ++e) ca[r][e][0] = ca[r][e][1] = cc[r][e][0] = cc[r][e][1] = 0.f;
  const int qc = 32 * warp + lane;
  auto flush_cols = [&](long long c) {
    const int j0 = (int)(c * SEG) + EPQ * qc;
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int e = 0; e < EPQ; ++e) {
        if (j0 + e < n) {
          double* o = reinterpret_cast<double*>(out + (size_t)r * n + j0 + e);
          atomicAdd(o, (double)ca[r][e][0] + (double)cc[r][e][0]);
          atomicAdd(o + 1, (double)ca[r][e][1] + (double)cc[r][e][1]);
        }
        ca[r][e][0] = ca[r][e][1] = cc[r][e][0] = cc[r][e][1] = 0.f;
      }
  };
  long long c = c0, rb = rb0;
  bool ok = true;
  for (long long u = u0; u < u1; ++u) {
    const long long i = u - u0;
    const int s = (int)(i % SSTAGES);
    const uint32_t parity = (uint32_t)((i / SSTAGES) & 1);
    ok = __all_sync(0xffffffffu, mbar_wait(&full[s], parity));
    if (!ok) {
      if (lane == 0) atomicExch(err, 26);
      break;
    }
    const int cb = (int)(c * SEG), row0 = (int)(rb * SROWS);
    const bool diag = row0 + SROWS > cb;  // the segment reaches the diagonal of this row block
    const uint8_t* st = smem + s * SSTAGE;
    const float4* sx = reinterpret_cast<const float4*>(st + SMAT);
    const int nq = min(SEG, ld - cb) * ESZ / 16;
    // row part: row `warp`, entries j >= i
    {
      const int row = row0 + warp;
      float f[NR][2];
#pragma unroll
      for (int r = 0; r < NR; ++r) f[r][0] = f[r][1] = 0.f;
      if (row < n) {
        const float4* srow = reinterpret_cast<const float4*>(st + warp * SBYTES_ROW);
#pragma unroll 4
        for (int q = lane; q < nq; q += 32) {
          float4 m = srow[q];
          if (diag) {  // zero the entries left of the diagonal
            const int j = cb + EPQ * q;
            if (REAL) {
              if (j < row) m.x = 0.f;
              if (j + 1 < row) m.y = 0.f;
              if (j + 2 < row) m.z = 0.f;
              if (j + 3 < row) m.w = 0.f;
            } else {
              if (j < row) m.x = m.y = 0.f;
              if (j + 1 < row) m.z = m.w = 0.f;
            }
          }
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const float4* xr = sx + r * (SXMAX / 32);
            float re = f[r][0], im = f[r][1];
            if (REAL) {
              const float4 x0 = xr[2 * q], x1 = xr[2 * q + 1];
              re = fmaf(m.x, x0.x, re);
              im = fmaf(m.x, x0.y, im);
              re = fmaf(m.y, x0.z, re);
              im = fmaf(m.y, x0.w, im);
              re = fmaf(m.z, x1.x, re);
              im = fmaf(m.z, x1.y, im);
              re = fmaf(m.w, x1.z, re);
              im = fmaf(m.w, x1.w, im);
            } else {
              const float4 x4 = xr[q];
              const float my = CONJ ? -m.y : m.y, mw = CONJ ? -m.w : m.w;
              re = fmaf(m.x, x4.x, re);
              re = fmaf(-my, x4.y, re);
              re = fmaf(m.z, x4.z, re);
              re = fmaf(-mw, x4.w, re);
              im = fmaf(m.x, x4.y, im);
              im = fmaf(my, x4.x, im);
              im = fmaf(m.z, x4.w, im);
              im = fmaf(mw, x4.z, im);
            }
            f[r][0] = re;
            f[r][1] = im;
          }
        }
      }
      // FP32 warp reduction (FP64 arithmetic in every unit would saturate GB300's FP64 pipe);
      // the units of a row meet in the FP64 accumulator
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        float re = f[r][0], im = f[r][1];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          re += __shfl_xor_sync(0xffffffffu, re, off);
          im += __shfl_xor_sync(0xffffffffu, im, off);
        }
        if (lane == 0 && row < n) {
          double* o = reinterpret_cast<double*>(out + (size_t)r * n + row);
          atomicAdd(o, (double)re);
          atomicAdd(o + 1, (double)im);
        }
      }
    }
    // column part: entries j > i of the 8 rows, the lane's float4 column slot qc
    if (qc < nq) {
      float t[NR][EPQ][2];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int e = 0; e < EPQ; ++e) t[r][e][0] = t[r][e][1] = 0.f;
      const int j = cb + EPQ * qc;
      const float2* sxi = reinterpret_cast<const float2*>(st + SMAT + SXMAX);
#pragma unroll
      for (int rr = 0; rr < SROWS; ++rr) {
        const int row = row0 + rr;
        float4 m = row < n ? reinterpret_cast<const float4*>(st + rr * SBYTES_ROW)[qc] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (diag) {  // keep only j > i
          if (REAL) {
            if (j <= row) m.x = 0.f;
            if (j + 1 <= row) m.y = 0.f;
            if (j + 2 <= row) m.z = 0.f;
            if (j + 3 <= row) m.w = 0.f;
          } else {
            if (j <= row) m.x = m.y = 0.f;
            if (j + 1 <= row) m.z = m.w = 0.f;
          }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const float2 xi = sxi[r * 8 + rr];
          if (REAL) {
            const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
            for (int e = 0; e < EPQ; ++e) {
              t[r][e][0] = fmaf(mv[e], xi.x, t[r][e][0]);
              t[r][e][1] = fmaf(mv[e], xi.y, t[r][e][1]);
            }
          } else {
            const float ar[2] = {m.x, m.z};
            const float ai[2] = {CONJ ? -m.y : m.y, CONJ ? -m.w : m.w};
#pragma unroll
            for (int e = 0; e < EPQ; ++e) {
              t[r][e][0] = fmaf(ar[e], xi.x, fmaf(-ai[e], xi.y, t[r][e][0]));
              t[r][e][1] = fmaf(ar[e], xi.y, fmaf(ai[e], xi.x, t[r][e][1]));
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int e = 0; e < EPQ; ++e)
#pragma unroll
          for (int z = 0; z < 2; ++z) {  // two-sum into the running column sums
            const float a = ca[r][e][z], b = t[r][e][z], tt = a + b, bb = tt - a;
            cc[r][e][z] += (a - (tt - bb)) + (b - bb);
            ca[r][e][z] = tt;
          }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (++rb == G.nrb(c)) {
      flush_cols(c);
      ++c;
      rb = 0;
    }
  }
  if (ok && rb > 0) flush_cols(c);
}

template <int NR, bool REAL, bool CONJ>
cudaError_t launch_sym(const void* M, int ld, int n, GemvScratch& w, cudaStream_t s) {
  constexpr int SEG = SBYTES_ROW / (REAL ? 4 : 8);
  auto k = gemv_sym_kernel<NR, REAL, CONJ>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  static int sms = 0;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SSMEM);
    int dev = 0;
    if (attr == cudaSuccess) attr = cudaGetDevice(&dev);
    if (attr == cudaSuccess) attr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  if (attr != cudaSuccess) return attr;
  if (!w.err) return cudaErrorInvalidValue;
  const SymGeom G = sym_geom(n, ld, SEG);
  const long long units = G.off(G.S);
  const int grid = (int)std::max(1LL, std::min<long long>(units, sms));
  k<<<grid, STHREADS, SSMEM, s>>>(M, ld, n, w.xh, w.acc, units, w.err);
  return cudaGetLastError();
}

template <int NR, bool REAL, bool CONJ>
cudaError_t launch_stream(const void* M, int ld, int n, GemvScratch& w, cudaStream_t s) {
  constexpr int SEG = SBYTES_ROW / (REAL ? 4 : 8);
  auto k = gemv_stream_kernel<NR, REAL, CONJ>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  static int sms = 0;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SSMEM);
    int dev = 0;
    if (attr == cudaSuccess) attr = cudaGetDevice(&dev);
    if (attr == cudaSuccess) attr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  if (attr != cudaSuccess) return attr;
  if (!w.err) return cudaErrorInvalidValue;
  const int upr = (ld + SEG - 1) / SEG;
  const long long units = (long long)((n + SROWS - 1) / SROWS) * upr;
  const int grid = (int)std::max(1LL, std::min<long long>(units, sms));
  k<<<grid, STHREADS, SSMEM, s>>>(M, ld, n, w.xh, w.acc, units, upr, w.err);
  return cudaGetLastError();
}

}  // namespace

template <int NR>
cudaError_t gemv_stream_c64(const float2* M, int ld, int n, bool conj, GemvScratch& w, cudaStream_t s) {
  if (w.symmetric)
    return conj ? launch_sym<NR, false, true>(M, ld, n, w, s) : launch_sym<NR, false, false>(M, ld, n, w, s);
  return conj ? launch_stream<NR, false, true>(M, ld, n, w, s) : launch_stream<NR, false, false>(M, ld, n, w, s);
}
template <int NR>
cudaError_t gemv_stream_r32(const float* M, int ld, int n, GemvScratch& w, cudaStream_t s) {
  if (w.symmetric) return launch_sym<NR, true, false>(M, ld, n, w, s);
  return launch_stream<NR, true, false>(M, ld, n, w, s);
}
template cudaError_t gemv_stream_c64<1>(const float2*, int, int, bool, GemvScratch&, cudaStream_t);
template cudaError_t gemv_stream_c64<2>(const float2*, int, int, bool, GemvScratch&, cudaStream_t);
template cudaError_t gemv_stream_r32<1>(const float*, int, int, GemvScratch&, cudaStream_t);
template cudaError_t gemv_stream_r32<2>(const float*, int, int, GemvScratch&, cudaStream_t);

}  // namespace rfcmp
