// Streaming GEMV: y = op(M) x for one or two columns with the matrix moved by the bulk-copy
// engine.
//
// The operator products of a single-right-hand-side solve are HBM bound: each application
// streams T_A, V and the factors once.  A register-pipelined GEMV keeps only as many bytes in
// flight as its unrolled loads allow; here one producer thread per CTA issues cp.async.bulk
// copies of whole row segments (8 rows x 512 complex64 or 1024 FP32 values, 32 KB per stage)
// together with the matching segment of x into shared-memory rings of four to six stages per SM
// (one CTA with four stages, or two CTAs with two or three where the registers allow twice the
// warps), so 128 to 192 KB of matrix per SM are in flight whatever the consumers do; consumers read the matrix and x from
// shared memory only and release a stage through an mbarrier.  Two kernels:
//   * gemv_sym_kernel (FP32 mode, symmetric M: T_A, V and the factors): reads only the tiles on
//     and above the diagonal and forms both the row and the mirrored column product;
//   * gemv_stream_ff_kernel (float-float, one column of a complex64 M): the accurate products,
//     one consumer warp per row of a stage.
// Work units are dealt to persistent CTAs in contiguous ranges of equal size; partial sums meet
// in FP64 atomics.  Every wait is bounded and records an error code on timeout.
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
constexpr int SXMAX = 2 * 8192;             // x per stage of the float-float kernel: hi and lo segments
constexpr int SSTAGE = SMAT + SXMAX;        // 48 KB: a stage of the float-float kernel
constexpr int STHREADS = (SROWS + 1) * 32;  // consumers + producer warp

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

// ---------------------------------------------------------------- float-float, one column
// The accurate products (right-hand side, refinement residuals) of a complex64 matrix in the
// streaming layout: x is split into FP32 hi + lo, every product m * x_hi is exact as (p, e) by an
// FMA residual, p enters a float-float (hi, lo) accumulator by an error-free two-sum and
// e + m * x_lo its low word (about 1e-14 of sum |terms|).
// two CTAs per SM, two stages each: twice the consumer warps to hide the two-sum chains
constexpr int FF_NCTA = 2;
constexpr int FF_NST = 2;
static_assert(FF_NCTA * (FF_NST * SSTAGE + 256 + 1024) <= 233472, "the SM holds FF_NCTA float-float CTAs");

__device__ __forceinline__ void ff_acc(float& hi, float& lo, float a, float bh, float bl) {
  const float p = a * bh;
  const float e = fmaf(a, bh, -p);
  const float c = fmaf(a, bl, e);
  const float s = hi + p;
  const float bb = s - hi;
  lo += ((hi - (s - bb)) + (p - bb)) + c;
  hi = s;
}

template <bool CONJ>
__global__ void __launch_bounds__(STHREADS, FF_NCTA)
gemv_stream_ff_kernel(const float2* __restrict__ M, int ld, int n, const float2* __restrict__ xh,
                      const float2* __restrict__ xl, double2* __restrict__ out, double scale, long long units,
                      int upr, int* __restrict__ err) {
  RF_COUNT_LAUNCH();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + FF_NST * SSTAGE);
  uint64_t* empty = full + FF_NST;
  constexpr int SEG = SBYTES_ROW / 8;  // 512 complex entries per row segment
  static_assert(SEG * 8 <= SXMAX / 2, "x hi and lo segments fit the stage");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < FF_NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], SROWS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == SROWS) {
    if (lane == 0) {
      for (long long u = u0; u < u1; ++u) {
        const long long i = u - u0;
        const int s = (int)(i % FF_NST);
        const long long round = i / FF_NST;
        if (round > 0 && !mbar_wait(&empty[s], (uint32_t)((round - 1) & 1))) {
          atomicExch(err, 31);
          break;
        }
        const int rb = (int)(u / upr), cb = (int)(u % upr) * SEG;
        const int row0 = rb * SROWS, rows = min(SROWS, n - row0);
        const int cols = min(SEG, ld - cb);
        const uint32_t bytes = (uint32_t)cols * 8;
        mbar_expect_tx(&full[s], bytes * rows + 2 * bytes);
        uint8_t* st = smem + s * SSTAGE;
        for (int r = 0; r < rows; ++r)
          bulk_load(st + r * SBYTES_ROW, M + (size_t)(row0 + r) * ld + cb, bytes, &full[s]);
        bulk_load(st + SMAT, xh + cb, bytes, &full[s]);
        bulk_load(st + SMAT + SXMAX / 2, xl + cb, bytes, &full[s]);
      }
      const long long cnt = u1 - u0;
      for (long long i = cnt > FF_NST ? cnt - FF_NST : 0; i < cnt; ++i)
        if (!mbar_wait(&full[i % FF_NST], (uint32_t)((i / FF_NST) & 1))) atomicExch(err, 33);
    }
    return;
  }

  float fh[2] = {0.f, 0.f}, fl[2] = {0.f, 0.f};  // (re, im) float-float sums of row `warp`
  auto flush = [&](long long rb) {
    const int row = (int)rb * SROWS + warp;
    const double re = warp_sum_d((double)fh[0] + (double)fl[0]);
    const double im = warp_sum_d((double)fh[1] + (double)fl[1]);
    fh[0] = fh[1] = fl[0] = fl[1] = 0.f;
    if (lane == 0 && row < n) {
      double* o = reinterpret_cast<double*>(out + row);
      atomicAdd(o, scale * re);
      atomicAdd(o + 1, scale * im);
    }
  };
  long long cur_rb = -1;
  bool ok = true;
  for (long long u = u0; u < u1 && ok; ++u) {
    const long long i = u - u0;
    const int s = (int)(i % FF_NST);
    const uint32_t parity = (uint32_t)((i / FF_NST) & 1);
    const int rb = (int)(u / upr), cb = (int)(u % upr) * SEG;
    if (rb != cur_rb) {
      if (cur_rb >= 0) flush(cur_rb);
      cur_rb = rb;
    }
    ok = __all_sync(0xffffffffu, mbar_wait(&full[s], parity));
    if (!ok) {
      if (lane == 0) atomicExch(err, 32);
      break;
    }
    const int row = rb * SROWS + warp;
    if (row < n) {
      const uint8_t* st = smem + s * SSTAGE;
      const float4* sxh = reinterpret_cast<const float4*>(st + SMAT);
      const float4* sxl = reinterpret_cast<const float4*>(st + SMAT + SXMAX / 2);
      const float4* srow = reinterpret_cast<const float4*>(st + warp * SBYTES_ROW);
      const int nq = min(SEG, ld - cb) / 2;  // two complex entries per float4
#pragma unroll 2
      for (int q = lane; q < nq; q += 32) {
        const float4 m = srow[q], x4 = sxh[q], l4 = sxl[q];
        const float my = CONJ ? -m.y : m.y, mw = CONJ ? -m.w : m.w;
        ff_acc(fh[0], fl[0], m.x, x4.x, l4.x);
        ff_acc(fh[0], fl[0], -my, x4.y, l4.y);
        ff_acc(fh[0], fl[0], m.z, x4.z, l4.z);
        ff_acc(fh[0], fl[0], -mw, x4.w, l4.w);
        ff_acc(fh[1], fl[1], m.x, x4.y, l4.y);
        ff_acc(fh[1], fl[1], my, x4.x, l4.x);
        ff_acc(fh[1], fl[1], m.z, x4.w, l4.w);
        ff_acc(fh[1], fl[1], mw, x4.z, l4.z);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  if (ok && cur_rb >= 0) flush(cur_rb);
}

// ---------------------------------------------------------------- symmetric matrices
// For a symmetric M (T_A, V and the factors all are) only the tiles that reach the diagonal or
// lie above it are read: a tile of 8 rows I x one segment J contributes y_I += M_IJ x_J (row part,
// entries j >= i) and y_J += M_IJ^T x_I (column part, entries j > i), so half the matrix bytes
// leave HBM.  Units run column-major over the upper triangle: segment c holds the row blocks
// 0 .. min(RB, P (c + 1)) - 1 (P = segment width / 8 rows), so the column part stays in registers
// across the row blocks of a segment and reaches y once per segment.
//
// Both parts come from one read of the tile: consumer thread t owns float4 column slot t of the
// segment (256 slots = the 8 consumer warps x 32 lanes) in all 8 rows.  For each row it adds
// M_ij x_j into that row's partial (x_j of its slot held in registers) and M_ij x_i into its
// column sums (x_i a shared-memory broadcast).  The 8 x NR complex row partials of a warp are
// reduce-scattered across its lanes (each exchange halves the values a lane holds), the 8 warps'
// results meet in shared memory, and one warp per unit (rotating) adds them and issues the FP64
// atomics of the row part.
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

// Reduce-scatter of V = 16 or 32 per-lane values over the warp: on return v[0] of lane l is the
// warp sum of value l * V / 32 (for V = 16 lanes l and l ^ 1 hold the same sum).
template <int V>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[V], int lane) {
#pragma unroll
  for (int step = 0; step < 5; ++step) {
    const int off = 16 >> step;
    const int h = V >> (step + 1);  // values kept after this exchange (0: plain reduction)
    if (h == 0) {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
    } else {
      const bool upper = (lane & off) != 0;
#pragma unroll
      for (int k = 0; k < h; ++k) {
        const float send = upper ? v[k] : v[k + h];
        const float keep = upper ? v[k + h] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
  }
}

// Stage layout of the symmetric kernel: the 8 row segments, the x segments of its NR columns,
// x of the 8 rows, and the consumer warps' row partials, rounded to 128 bytes.  With two CTAs
// per SM a CTA takes three stages where both rings fit the SM's 228 KB of shared memory
// (1 KB per CTA reserved by the system): the one-column complex product (37.5 KB stages);
// the others take two.
template <int NR, bool REAL, int NCTA>
struct SymStage {
  static constexpr int SEG = SBYTES_ROW / (REAL ? 4 : 8);
  static constexpr int XB = NR * SEG * 8;  // x segments of the stage (complex FP32)
  static constexpr int BYTES = ((SMAT + XB + NR * 64 + 8 * (SROWS * NR * 2) * 4) + 127) / 128 * 128;
  static constexpr int NST = NCTA == 1 ? SSTAGES : ((2 * (3 * BYTES + 256 + 1024) <= 233472) ? 3 : 2);
  static constexpr int SMEM = NST * BYTES + 256;  // + alignment slack and the mbarriers
  static_assert(SMEM <= 232448, "dynamic shared memory of one CTA");
  static_assert(NCTA * (SMEM + 1024) <= 233472, "the SM holds NCTA such CTAs");
  static_assert(BYTES % 128 == 0 && (SMAT + XB) % 16 == 0, "bulk-copy destinations stay 16-byte aligned");
};

// The 8 rows of one tile for column slot qc (entries j .. j + EPQ - 1): row partials v gain
// M_ij x_j (j >= i), column partials t gain M_ij x_i (j > i).  DIAG: the tile reaches the
// diagonal and the entries outside those ranges are dropped.
template <int NR, bool REAL, bool CONJ, bool DIAG, int XB, int EPQ = (REAL ? 4 : 2)>
__device__ __forceinline__ void sym_tile(const uint8_t* st, int qc, int row0, int n, int j, const float2 (&xj)[NR][EPQ],
                                         float (&v)[SROWS * NR * 2], float (&t)[NR][EPQ][2]) {
  const float2* sxi = reinterpret_cast<const float2*>(st + SMAT + XB);
#pragma unroll
  for (int rr = 0; rr < SROWS; ++rr) {
    const int row = row0 + rr;
    const float4 m = row < n ? reinterpret_cast<const float4*>(st + rr * SBYTES_ROW)[qc] : make_float4(0.f, 0.f, 0.f, 0.f);
    float er[EPQ], ei[EPQ];  // entries as (re, im)
    if constexpr (REAL) {
      er[0] = m.x, er[1] = m.y, er[2] = m.z, er[3] = m.w;
#pragma unroll
      for (int e = 0; e < EPQ; ++e) ei[e] = 0.f;
    } else {
      er[0] = m.x, ei[0] = CONJ ? -m.y : m.y;
      er[1] = m.z, ei[1] = CONJ ? -m.w : m.w;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const float2 xi = sxi[r * SROWS + rr];
      float pre = v[(rr * NR + r) * 2], pim = v[(rr * NR + r) * 2 + 1];
#pragma unroll
      for (int e = 0; e < EPQ; ++e) {
        float ar = er[e], ai = ei[e], br = er[e], bi = ei[e];
        if constexpr (DIAG) {
          if (j + e < row) ar = ai = 0.f;
          if (j + e <= row) br = bi = 0.f;
        }
        if constexpr (REAL) {
          pre = fmaf(ar, xj[r][e].x, pre);
          pim = fmaf(ar, xj[r][e].y, pim);
          t[r][e][0] = fmaf(br, xi.x, t[r][e][0]);
          t[r][e][1] = fmaf(br, xi.y, t[r][e][1]);
        } else {
          pre = fmaf(ar, xj[r][e].x, fmaf(-ai, xj[r][e].y, pre));
          pim = fmaf(ar, xj[r][e].y, fmaf(ai, xj[r][e].x, pim));
          t[r][e][0] = fmaf(br, xi.x, fmaf(-bi, xi.y, t[r][e][0]));
          t[r][e][1] = fmaf(br, xi.y, fmaf(bi, xi.x, t[r][e][1]));
        }
      }
      v[(rr * NR + r) * 2] = pre;
      v[(rr * NR + r) * 2 + 1] = pim;
    }
  }
}

template <int NR, bool REAL, bool CONJ, int NCTA>
__global__ void __launch_bounds__(STHREADS, NCTA)
gemv_sym_kernel(const void* __restrict__ Mv, int ld, int n, const float2* __restrict__ xh,
                double2* __restrict__ out, double scale, long long units, int* __restrict__ err) {
  RF_COUNT_LAUNCH();
  constexpr int NST = SymStage<NR, REAL, NCTA>::NST;
  constexpr int STG = SymStage<NR, REAL, NCTA>::BYTES;
  constexpr int XB = SymStage<NR, REAL, NCTA>::XB;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * STG);
  uint64_t* empty = full + NST;
  uint64_t* rfull = empty + NST;  // the 8 warps' row partials of a stage are in shared memory
  constexpr int ESZ = REAL ? 4 : 8;
  constexpr int SEG = SBYTES_ROW / ESZ;
  constexpr int EPQ = 16 / ESZ;       // matrix entries per float4
  constexpr int V = SROWS * NR * 2;   // row partials per lane: 8 rows x NR columns x (re, im)
  static_assert(SBYTES_ROW / 16 == SROWS * 32, "one float4 column slot per consumer thread");
  static_assert(V == 16 || V == 32, "reduce-scatter of 16 or 32 values");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const SymGeom G = sym_geom(n, ld, SEG);
  const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], SROWS);
      mbar_init(&rfull[s], SROWS);
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
        const int s = (int)(i % NST);
        const long long round = i / NST;
        if (round > 0 && !mbar_wait(&empty[s], (uint32_t)((round - 1) & 1))) {
          atomicExch(err, 24);
          break;
        }
        const int cb = (int)(c * SEG), row0 = (int)(rb * SROWS), rows = min(SROWS, n - row0);
        const int cols = min(SEG, ld - cb);
        const uint32_t bytes = (uint32_t)cols * ESZ, xbytes = (uint32_t)cols * 8;
        mbar_expect_tx(&full[s], bytes * rows + (xbytes + 64) * NR);
        uint8_t* st = smem + s * STG;
        for (int r = 0; r < rows; ++r)
          bulk_load(st + r * SBYTES_ROW, M + ((size_t)(row0 + r) * ld + cb) * ESZ, bytes, &full[s]);
        for (int r = 0; r < NR; ++r) {
          bulk_load(st + SMAT + r * (XB / NR), xh + (size_t)r * ld + cb, xbytes, &full[s]);
          bulk_load(st + SMAT + XB + r * 64, xh + (size_t)r * ld + row0, 64, &full[s]);  // x of the 8 rows
        }
        if (++rb == G.nrb(c)) {
          ++c;
          rb = 0;
        }
      }
      const long long cnt = u1 - u0;
      for (long long i = cnt > NST ? cnt - NST : 0; i < cnt; ++i)
        if (!mbar_wait(&full[i % NST], (uint32_t)((i / NST) & 1))) atomicExch(err, 25);
    }
    return;
  }

  // column sums of slot qc (EPQ entries, NR columns) in compensated FP32
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
          atomicAdd(o, scale * ((double)ca[r][e][0] + (double)cc[r][e][0]));
          atomicAdd(o + 1, scale * ((double)ca[r][e][1] + (double)cc[r][e][1]));
        }
        ca[r][e][0] = ca[r][e][1] = cc[r][e][0] = cc[r][e][1] = 0.f;
      }
  };
  long long c = c0, rb = rb0;
  bool ok = true;
  for (long long u = u0; u < u1; ++u) {
    const long long i = u - u0;
    const int s = (int)(i % NST);
    const uint32_t parity = (uint32_t)((i / NST) & 1);
    ok = __all_sync(0xffffffffu, mbar_wait(&full[s], parity));
    if (!ok) {
      if (lane == 0) atomicExch(err, 26);
      break;
    }
    const int cb = (int)(c * SEG), row0 = (int)(rb * SROWS);
    const bool diag = row0 + SROWS > cb;  // the segment reaches the diagonal of this row block
    uint8_t* st = smem + s * STG;
    const int nq = min(SEG, ld - cb) * ESZ / 16;
    float v[V];  // row partials, index (rr * NR + r) * 2 + (re, im)
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = 0.f;
    if (qc < nq) {
      // x_j of the slot, NR columns
      float2 xj[NR][EPQ];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const float4* xr = reinterpret_cast<const float4*>(st + SMAT + r * (XB / NR));
#pragma unroll
        for (int h = 0; h < EPQ / 2; ++h) {
          const float4 x4 = xr[(EPQ / 2) * qc + h];
          xj[r][2 * h] = make_float2(x4.x, x4.y);
          xj[r][2 * h + 1] = make_float2(x4.z, x4.w);
        }
      }
      const int j = cb + EPQ * qc;
      float t[NR][EPQ][2];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int e = 0; e < EPQ; ++e) t[r][e][0] = t[r][e][1] = 0.f;
      if (diag) sym_tile<NR, REAL, CONJ, true, XB>(st, qc, row0, n, j, xj, v, t);
      else sym_tile<NR, REAL, CONJ, false, XB>(st, qc, row0, n, j, xj, v, t);
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
    // row part: reduce-scatter over the warp, then the 8 warps meet in shared memory
    warp_reduce_scatter<V>(v, lane);
    float* red = reinterpret_cast<float*>(st + SMAT + XB + NR * 64);  // [SROWS warps][V]
    if (V == 32 || (lane & 1) == 0) red[warp * V + lane * V / 32] = v[0];
    __syncwarp();
    if (lane == 0) mbar_arrive(&rfull[s]);
    if (warp == (int)(i % SROWS)) {
      const bool got = __all_sync(0xffffffffu, mbar_wait(&rfull[s], parity));
      if (!got) {
        if (lane == 0) atomicExch(err, 27);
        ok = false;
        break;
      }
      if (lane < V) {
        float sum = 0.f;
#pragma unroll
        for (int w2 = 0; w2 < SROWS; ++w2) sum += red[w2 * V + lane];
        const int rr = lane / (2 * NR), r = (lane / 2) % NR, z = lane & 1;
        const int row = row0 + rr;
        if (row < n) atomicAdd(reinterpret_cast<double*>(out + (size_t)r * n + row) + z, scale * (double)sum);
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

// Two CTAs per SM where the registers allow (the real two-column variant needs more than half
// the register file): twice the warps to hide the consumers' latency (complex T_A product at
// N = 30720: 0.659 ms with one CTA of four stages, 0.585 ms with two CTAs of two stages,
// 0.557 ms with two CTAs of three stages: the measured copy bandwidth).
template <int NR, bool REAL, bool CONJ>
cudaError_t launch_sym(const void* M, int ld, int n, GemvScratch& w, cudaStream_t s) {
  constexpr int SEG = SBYTES_ROW / (REAL ? 4 : 8);
  constexpr int NCTA = REAL && NR == 2 ? 1 : 2;
  constexpr int SMEM = SymStage<NR, REAL, NCTA>::SMEM;
  auto k = gemv_sym_kernel<NR, REAL, CONJ, NCTA>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  static int sms = 0;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    int dev = 0;
    if (attr == cudaSuccess) attr = cudaGetDevice(&dev);
    if (attr == cudaSuccess) attr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  if (attr != cudaSuccess) return attr;
  if (!w.err) return cudaErrorInvalidValue;
  const SymGeom G = sym_geom(n, ld, SEG);
  const long long units = G.off(G.S);
  const int grid = (int)std::max(1LL, std::min<long long>(units, (long long)NCTA * sms));
  k<<<grid, STHREADS, SMEM, s>>>(M, ld, n, w.xh, w.out, w.scale, units, w.err);
  return cudaGetLastError();
}

template <bool CONJ>
cudaError_t launch_stream_ff(const float2* M, int ld, int n, GemvScratch& w, cudaStream_t s) {
  constexpr int SEG = SBYTES_ROW / 8;
  auto k = gemv_stream_ff_kernel<CONJ>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  static int sms = 0;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, FF_NST * SSTAGE + 256);
    int dev = 0;
    if (attr == cudaSuccess) attr = cudaGetDevice(&dev);
    if (attr == cudaSuccess) attr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  if (attr != cudaSuccess) return attr;
  if (!w.err || !w.xl) return cudaErrorInvalidValue;
  const int upr = (ld + SEG - 1) / SEG;
  const long long units = (long long)((n + SROWS - 1) / SROWS) * upr;
  const int grid = (int)std::max(1LL, std::min<long long>(units, (long long)FF_NCTA * sms));
  k<<<grid, STHREADS, FF_NST * SSTAGE + 256, s>>>(M, ld, n, w.xh, w.xl, w.out, w.scale, units, upr, w.err);
  return cudaGetLastError();
}

}  // namespace

template <int NR>
cudaError_t gemv_stream_c64(const float2* M, int ld, int n, bool conj, GemvScratch& w, cudaStream_t s) {
  if (!w.symmetric) return cudaErrorInvalidValue;
  return conj ? launch_sym<NR, false, true>(M, ld, n, w, s) : launch_sym<NR, false, false>(M, ld, n, w, s);
}
template <int NR>
cudaError_t gemv_stream_r32(const float* M, int ld, int n, GemvScratch& w, cudaStream_t s) {
  if (!w.symmetric) return cudaErrorInvalidValue;
  return launch_sym<NR, true, false>(M, ld, n, w, s);
}
cudaError_t gemv_stream_c64_ff(const float2* M, int ld, int n, bool conj, GemvScratch& w, cudaStream_t s) {
  return conj ? launch_stream_ff<true>(M, ld, n, w, s) : launch_stream_ff<false>(M, ld, n, w, s);
}
template cudaError_t gemv_stream_c64<1>(const float2*, int, int, bool, GemvScratch&, cudaStream_t);
template cudaError_t gemv_stream_c64<2>(const float2*, int, int, bool, GemvScratch&, cudaStream_t);
template cudaError_t gemv_stream_r32<1>(const float*, int, int, GemvScratch&, cudaStream_t);
template cudaError_t gemv_stream_r32<2>(const float*, int, int, GemvScratch&, cudaStream_t);

RF_LAUNCH_READER(launches_gemv_stream)

}  // namespace rfcmp
