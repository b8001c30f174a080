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
#include <vector>

#include "rfcmp_internal.h"

namespace rfcmp {

namespace {

constexpr int GEMV_ROWS_PER_WARP = 4;
constexpr int GEMV_WARPS = 8;
constexpr int GEMV_ROWS = GEMV_ROWS_PER_WARP * GEMV_WARPS;  // 32 rows per block
constexpr int GEMV_CHUNK = 1024;                            // columns staged per pass

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

// ---------------------------------------------------------------- complex64 GEMV
template <int NR, bool FF, bool CONJ>
__global__ void __launch_bounds__(GEMV_WARPS * 32)
gemv_c64_kernel(const float2* __restrict__ M, int ld, int n, const double2* __restrict__ x, double2* __restrict__ y,
                double2 scale, int accumulate) {
  __shared__ float4 xs_hi[NR][GEMV_CHUNK / 2];
  __shared__ float4 xs_lo[FF ? NR : 1][FF ? GEMV_CHUNK / 2 : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * GEMV_ROWS + warp * GEMV_ROWS_PER_WARP;
  double acc[GEMV_ROWS_PER_WARP][NR][2];
#pragma unroll
  for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[a][r][0] = acc[a][r][1] = 0.0;

  for (int cb = 0; cb < ld; cb += GEMV_CHUNK) {
    const int clen = min(GEMV_CHUNK, ld - cb);  // multiple of 64
    __syncthreads();
    for (int idx = threadIdx.x; idx < NR * (GEMV_CHUNK / 2); idx += blockDim.x) {
      const int r = idx / (GEMV_CHUNK / 2), p = idx % (GEMV_CHUNK / 2);
      const int c0 = cb + 2 * p;
      double2 v0 = make_double2(0.0, 0.0), v1 = make_double2(0.0, 0.0);
      if (c0 < n) v0 = x[(size_t)r * n + c0];
      if (c0 + 1 < n) v1 = x[(size_t)r * n + c0 + 1];
      float4 h = make_float4((float)v0.x, (float)v0.y, (float)v1.x, (float)v1.y);
      xs_hi[r][p] = h;
      if (FF)
        xs_lo[r][p] = make_float4((float)(v0.x - (double)h.x), (float)(v0.y - (double)h.y),
                                  (float)(v1.x - (double)h.z), (float)(v1.y - (double)h.w));
    }
    __syncthreads();
    float fh[GEMV_ROWS_PER_WARP][NR][2], fl[GEMV_ROWS_PER_WARP][NR][2];
#pragma unroll
    for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
      for (int r = 0; r < NR; ++r) fh[a][r][0] = fh[a][r][1] = fl[a][r][0] = fl[a][r][1] = 0.f;
    const int npair = clen / 2;
#pragma unroll 4
    for (int p = lane; p < npair; p += 32) {
      float4 m[GEMV_ROWS_PER_WARP];
#pragma unroll
      for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
        const int row = row0 + a;
        m[a] = row < n ? __ldg(reinterpret_cast<const float4*>(M + (size_t)row * ld + cb) + p)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        if (CONJ) {
          m[a].y = -m[a].y;
          m[a].w = -m[a].w;
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const float4 xh = xs_hi[r][p];
        if (!FF) {
#pragma unroll
          for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
            float re = fh[a][r][0], im = fh[a][r][1];
            re = fmaf(m[a].x, xh.x, re);
            re = fmaf(-m[a].y, xh.y, re);
            re = fmaf(m[a].z, xh.z, re);
            re = fmaf(-m[a].w, xh.w, re);
            im = fmaf(m[a].x, xh.y, im);
            im = fmaf(m[a].y, xh.x, im);
            im = fmaf(m[a].z, xh.w, im);
            im = fmaf(m[a].w, xh.z, im);
            fh[a][r][0] = re;
            fh[a][r][1] = im;
          }
        } else {
          const float4 xl = xs_lo[r][p];
#pragma unroll
          for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
            ff_mac(fh[a][r][0], fl[a][r][0], m[a].x, xh.x, xl.x);
            ff_mac(fh[a][r][0], fl[a][r][0], -m[a].y, xh.y, xl.y);
            ff_mac(fh[a][r][0], fl[a][r][0], m[a].z, xh.z, xl.z);
            ff_mac(fh[a][r][0], fl[a][r][0], -m[a].w, xh.w, xl.w);
            ff_mac(fh[a][r][1], fl[a][r][1], m[a].x, xh.y, xl.y);
            ff_mac(fh[a][r][1], fl[a][r][1], m[a].y, xh.x, xl.x);
            ff_mac(fh[a][r][1], fl[a][r][1], m[a].z, xh.w, xl.w);
            ff_mac(fh[a][r][1], fl[a][r][1], m[a].w, xh.z, xl.z);
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
#pragma unroll
  for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
    const int row = row0 + a;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const double re = warp_sum(acc[a][r][0]);
      const double im = warp_sum(acc[a][r][1]);
      if (lane == 0 && row < n) {
        double2 out = make_double2(scale.x * re - scale.y * im, scale.x * im + scale.y * re);
        double2* dst = y + (size_t)r * n + row;
        if (accumulate) {
          out.x += dst->x;
          out.y += dst->y;
        }
        *dst = out;
      }
    }
  }
}

// ---------------------------------------------------------------- real (hi + lo) GEMV
template <int NR, bool FF>
__global__ void __launch_bounds__(GEMV_WARPS * 32)
gemv_r32_kernel(const float* __restrict__ Mhi, const float* __restrict__ Mlo, int ld, int n,
                const double2* __restrict__ x, double2* __restrict__ y, double scale, int accumulate) {
  // x chunk as 4 complex per float4 pair: xs[r][q] holds complex 2q, 2q+1
  __shared__ float4 xs_hi[NR][GEMV_CHUNK / 2];
  __shared__ float4 xs_lo[FF ? NR : 1][FF ? GEMV_CHUNK / 2 : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * GEMV_ROWS + warp * GEMV_ROWS_PER_WARP;
  double acc[GEMV_ROWS_PER_WARP][NR][2];
#pragma unroll
  for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[a][r][0] = acc[a][r][1] = 0.0;

  for (int cb = 0; cb < ld; cb += GEMV_CHUNK) {
    const int clen = min(GEMV_CHUNK, ld - cb);
    __syncthreads();
    for (int idx = threadIdx.x; idx < NR * (GEMV_CHUNK / 2); idx += blockDim.x) {
      const int r = idx / (GEMV_CHUNK / 2), p = idx % (GEMV_CHUNK / 2);
      const int c0 = cb + 2 * p;
      double2 v0 = make_double2(0.0, 0.0), v1 = make_double2(0.0, 0.0);
      if (c0 < n) v0 = x[(size_t)r * n + c0];
      if (c0 + 1 < n) v1 = x[(size_t)r * n + c0 + 1];
      float4 h = make_float4((float)v0.x, (float)v0.y, (float)v1.x, (float)v1.y);
      xs_hi[r][p] = h;
      if (FF)
        xs_lo[r][p] = make_float4((float)(v0.x - (double)h.x), (float)(v0.y - (double)h.y),
                                  (float)(v1.x - (double)h.z), (float)(v1.y - (double)h.w));
    }
    __syncthreads();
    float fh[GEMV_ROWS_PER_WARP][NR][2], fl[GEMV_ROWS_PER_WARP][NR][2];
#pragma unroll
    for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a)
#pragma unroll
      for (int r = 0; r < NR; ++r) fh[a][r][0] = fh[a][r][1] = fl[a][r][0] = fl[a][r][1] = 0.f;
    const int nquad = clen / 4;
#pragma unroll 4
    for (int q = lane; q < nquad; q += 32) {
      float4 mh[GEMV_ROWS_PER_WARP], ml[GEMV_ROWS_PER_WARP];
#pragma unroll
      for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
        const int row = row0 + a;
        const bool ok = row < n;
        mh[a] = ok ? __ldg(reinterpret_cast<const float4*>(Mhi + (size_t)row * ld + cb) + q)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
        if (FF)
          ml[a] = ok ? __ldg(reinterpret_cast<const float4*>(Mlo + (size_t)row * ld + cb) + q)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const float4 x0 = xs_hi[r][2 * q], x1 = xs_hi[r][2 * q + 1];
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
          const float4 l0 = xs_lo[r][2 * q], l1 = xs_lo[r][2 * q + 1];
#pragma unroll
          for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
            // (mh + ml)(xh + xl): mh*xh exact in ff, mh*xl + ml*xh folded into the low word
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
#pragma unroll
  for (int a = 0; a < GEMV_ROWS_PER_WARP; ++a) {
    const int row = row0 + a;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const double re = warp_sum(acc[a][r][0]);
      const double im = warp_sum(acc[a][r][1]);
      if (lane == 0 && row < n) {
        double2 out = make_double2(scale * re, scale * im);
        double2* dst = y + (size_t)r * n + row;
        if (accumulate) {
          out.x += dst->x;
          out.y += dst->y;
        }
        *dst = out;
      }
    }
  }
}

template <int NR>
cudaError_t gemv_c64_dispatch(const float2* M, int ld, int n, const double2* x, double2* y, bool conj, double2 scale,
                              bool acc, GemvMode mode, cudaStream_t s) {
  const int blocks = (n + GEMV_ROWS - 1) / GEMV_ROWS;
  const int a = acc ? 1 : 0;
  ProfScope prof(mode == GEMV_FF ? "gemv_c64_ff" : "gemv_c64_f32", 8.0 * n * n + 32.0 * n * NR,
                 8.0 * n * n * NR, s);
  if (mode == GEMV_FF) {
    if (conj)
      gemv_c64_kernel<NR, true, true><<<blocks, GEMV_WARPS * 32, 0, s>>>(M, ld, n, x, y, scale, a);
    else
      gemv_c64_kernel<NR, true, false><<<blocks, GEMV_WARPS * 32, 0, s>>>(M, ld, n, x, y, scale, a);
  } else {
    if (conj)
      gemv_c64_kernel<NR, false, true><<<blocks, GEMV_WARPS * 32, 0, s>>>(M, ld, n, x, y, scale, a);
    else
      gemv_c64_kernel<NR, false, false><<<blocks, GEMV_WARPS * 32, 0, s>>>(M, ld, n, x, y, scale, a);
  }
  return cudaGetLastError();
}

template <int NR>
cudaError_t gemv_r32_dispatch(const float* Mhi, const float* Mlo, int ld, int n, const double2* x, double2* y,
                              double scale, bool acc, GemvMode mode, cudaStream_t s) {
  const int blocks = (n + GEMV_ROWS - 1) / GEMV_ROWS;
  const int a = acc ? 1 : 0;
  ProfScope prof(mode == GEMV_FF ? "gemv_r32_ff" : "gemv_r32_f32",
                 (mode == GEMV_FF ? 8.0 : 4.0) * n * n + 32.0 * n * NR, 4.0 * n * n * NR, s);
  if (mode == GEMV_FF)
    gemv_r32_kernel<NR, true><<<blocks, GEMV_WARPS * 32, 0, s>>>(Mhi, Mlo, ld, n, x, y, scale, a);
  else
    gemv_r32_kernel<NR, false><<<blocks, GEMV_WARPS * 32, 0, s>>>(Mhi, Mlo, ld, n, x, y, scale, a);
  return cudaGetLastError();
}

}  // namespace

int padded_ld(int n) { return (n + 63) / 64 * 64; }

cudaError_t gemv_c64(const float2* M, int n, const double2* x, double2* y, int nrhs, bool conjugate, double2 scale,
                     bool accumulate, GemvMode mode, cudaStream_t s) {
  const int ld = padded_ld(n);
  int r = 0;
  cudaError_t err = cudaSuccess;
  while (r < nrhs && err == cudaSuccess) {
    const int left = nrhs - r;
    const double2* xr = x + (size_t)r * n;
    double2* yr = y + (size_t)r * n;
    if (left >= 4) {
      err = gemv_c64_dispatch<4>(M, ld, n, xr, yr, conjugate, scale, accumulate, mode, s);
      r += 4;
    } else if (left >= 2) {
      err = gemv_c64_dispatch<2>(M, ld, n, xr, yr, conjugate, scale, accumulate, mode, s);
      r += 2;
    } else {
      err = gemv_c64_dispatch<1>(M, ld, n, xr, yr, conjugate, scale, accumulate, mode, s);
      r += 1;
    }
  }
  return err;
}

cudaError_t gemv_r32(const float* Mhi, const float* Mlo, int n, const double2* x, double2* y, int nrhs, double scale,
                     bool accumulate, GemvMode mode, cudaStream_t s) {
  const int ld = padded_ld(n);
  int r = 0;
  cudaError_t err = cudaSuccess;
  while (r < nrhs && err == cudaSuccess) {
    const int left = nrhs - r;
    const double2* xr = x + (size_t)r * n;
    double2* yr = y + (size_t)r * n;
    if (left >= 4) {
      err = gemv_r32_dispatch<4>(Mhi, Mlo, ld, n, xr, yr, scale, accumulate, mode, s);
      r += 4;
    } else if (left >= 2) {
      err = gemv_r32_dispatch<2>(Mhi, Mlo, ld, n, xr, yr, scale, accumulate, mode, s);
      r += 2;
    } else {
      err = gemv_r32_dispatch<1>(Mhi, Mlo, ld, n, xr, yr, scale, accumulate, mode, s);
      r += 1;
    }
  }
  return err;
}

// ---------------------------------------------------------------- sparse transforms
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void sigma_t_kernel(const int32_t* __restrict__ cell_edges, const int8_t* __restrict__ cell_sign, int nc,
                               int ne, const double2* __restrict__ x, double2* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= nc) return;
  const double2* xr = x + (size_t)r * ne;
  double2 acc = make_double2(0.0, 0.0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double sg = (double)cell_sign[3 * c + i];
    const double2 v = xr[cell_edges[3 * c + i]];
    acc.x += sg * v.x;
    acc.y += sg * v.y;
  }
  out[(size_t)r * nc + c] = acc;
}

__global__ void lambda_t_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ edge,
                                const int8_t* __restrict__ sign, int nv, int ne, const double2* __restrict__ x,
                                double2* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (v >= nv) return;
  const double2* xr = x + (size_t)r * ne;
  double2 acc = make_double2(0.0, 0.0);
  for (int q = ptr[v]; q < ptr[v + 1]; ++q) {
    const double sg = (double)sign[q];
    const double2 val = xr[edge[q]];
    acc.x += sg * val.x;
    acc.y += sg * val.y;
  }
  out[(size_t)r * nv + v] = acc;
}

__global__ void lap_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, int nc,
                           const double2* __restrict__ z, double2* __restrict__ out) {
  // Sigma^T Sigma z: 3 z_c - sum over edge-neighbours (values are +-1 and 3 by construction)
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= nc) return;
  const double2* zr = z + (size_t)r * nc;
  double2 acc = make_double2(0.0, 0.0);
  for (int q = ptr[c]; q < ptr[c + 1]; ++q) {
    const int d = col[q];
    const double w = d == c ? 3.0 : -1.0;
    acc.x += w * zr[d].x;
    acc.y += w * zr[d].y;
  }
  out[(size_t)r * nc + c] = acc;
}

__global__ void edge_combo_kernel(const int32_t* __restrict__ edge_cells, const int32_t* __restrict__ edge_verts,
                                  int ne, int nc, int nv, EdgeCombo cb, double2* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (n >= ne) return;
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
    const int v1 = edge_verts[2 * n], v2 = edge_verts[2 * n + 1];
    const double2 p = cb.zl[(size_t)r * nv + v1], m = cb.zl[(size_t)r * nv + v2];
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
}

__global__ void column_sum_kernel(const double2* __restrict__ w, int n, double* __restrict__ sums) {
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
                                   double2* __restrict__ q) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= nc) return;
  const size_t o = (size_t)r * nc + c;
  double2 v = z[o];
  if (w) {
    const double mx = sums[2 * r] / nc, my = sums[2 * r + 1] / nc;
    v.x += w[o].x - mx;
    v.y += w[o].y - my;
  }
  const double f = scale * area[c];
  q[o] = make_double2(f * v.x, f * v.y);
}

}  // namespace

cudaError_t sigma_t(const DeviceGeometry& g, const double2* x, double2* out, int nrhs, cudaStream_t s) {
  dim3 grid((g.nc + 255) / 256, nrhs);
  sigma_t_kernel<<<grid, 256, 0, s>>>(g.cell_edges, g.cell_sign, g.nc, g.ne, x, out);
  return cudaGetLastError();
}

cudaError_t lambda_t(const DeviceGeometry& g, const double2* x, double2* out, int nrhs, cudaStream_t s) {
  dim3 grid((g.nv + 255) / 256, nrhs);
  lambda_t_kernel<<<grid, 256, 0, s>>>(g.vtx_ptr, g.vtx_edge, g.vtx_sign, g.nv, g.ne, x, out);
  return cudaGetLastError();
}

cudaError_t lap_apply(const DeviceGeometry& g, const double2* z, double2* out, int nrhs, cudaStream_t s) {
  dim3 grid((g.nc + 255) / 256, nrhs);
  lap_kernel<<<grid, 256, 0, s>>>(g.lap_ptr, g.lap_col, g.nc, z, out);
  return cudaGetLastError();
}

cudaError_t edge_combo(const DeviceGeometry& g, const EdgeCombo& c, double2* out, int nrhs, cudaStream_t s) {
  dim3 grid((g.ne + 255) / 256, nrhs);
  edge_combo_kernel<<<grid, 256, 0, s>>>(g.edge_cells, g.edge_verts, g.ne, g.nc, g.nv, c, out);
  return cudaGetLastError();
}

cudaError_t star_middle(const DeviceGeometry& g, const double2* z, const double2* w, double scale, double2* q,
                        int nrhs, double* scratch_mean, cudaStream_t s) {
  if (w) {
    cudaError_t e = cudaMemsetAsync(scratch_mean, 0, sizeof(double) * 2 * nrhs, s);
    if (e != cudaSuccess) return e;
    dim3 grid(std::min(64, (g.nc + 255) / 256), nrhs);
    column_sum_kernel<<<grid, 256, 0, s>>>(w, g.nc, scratch_mean);
  }
  dim3 grid((g.nc + 255) / 256, nrhs);
  star_middle_kernel<<<grid, 256, 0, s>>>(g.area64, g.nc, z, w, scratch_mean, scale, q);
  return cudaGetLastError();
}

namespace {
__global__ void area_center_kernel(const double* __restrict__ area, int nc, const double2* __restrict__ w,
                                   const double* __restrict__ sums, double2* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= nc) return;
  const size_t o = (size_t)r * nc + c;
  const double mx = sums[2 * r] / nc, my = sums[2 * r + 1] / nc;
  out[o] = make_double2(area[c] * (w[o].x - mx), area[c] * (w[o].y - my));
}
__global__ void center_kernel(int nc, const double* __restrict__ sums, double2* __restrict__ out) {
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
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i];
}

__global__ void scale_kernel(double2* __restrict__ y, double2 a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = y[i];
    y[i] = make_double2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x);
  }
}

__global__ void cg_alpha_kernel(const double* __restrict__ rr, const double2* __restrict__ pAp,
                                double* __restrict__ alpha, const int* __restrict__ active, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const double d = pAp[r].x;
  alpha[r] = (active && !active[r]) || d == 0.0 ? 0.0 : rr[r] / d;
}

__global__ void cg_beta_kernel(const double2* __restrict__ rr_new2, double* __restrict__ rr, double* __restrict__ beta,
                               const int* __restrict__ active, int nrhs) {
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

// ---------------------------------------------------------------- dense inverse by block CG
// X = A^{-1} B for the sparse SPD A (or, with project, the graph Laplacian
// restricted to 1^perp: B = I - 1 1^T / n, X = A^+ by Sec. 3.2), W columns at a
// time; every column runs plain CG with its own scalars.  Arrays are row-major
// n x W so that consecutive threads read consecutive columns.
namespace {

constexpr int BCG_COLS = 128;  // columns per thread block
constexpr int BCG_ROWS = 256;  // rows per thread block

__global__ void bcg_init_kernel(int n, int W, int c0, bool project, double* __restrict__ X, double* __restrict__ R,
                                double* __restrict__ P, double* __restrict__ rr0) {
  const int c = blockIdx.x * BCG_COLS + (threadIdx.x % BCG_COLS);
  const int rsub = threadIdx.x / BCG_COLS;
  if (c >= W) return;
  const int r0 = blockIdx.y * BCG_ROWS;
  const int r1 = min(n, r0 + BCG_ROWS);
  const double off = project ? 1.0 / n : 0.0;
  double dot = 0.0;
  for (int i = r0 + rsub; i < r1; i += blockDim.x / BCG_COLS) {
    const double b = (i == c0 + c ? 1.0 : 0.0) - off;
    const size_t o = (size_t)i * W + c;
    X[o] = 0.0;
    R[o] = b;
    P[o] = b;
    dot += b * b;
  }
  atomicAdd(&rr0[c], dot);
}

// AP = A P, pAp += P.AP
__global__ void bcg_spmm_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, int n, int W, const double* __restrict__ P,
                                double* __restrict__ AP, double* __restrict__ pAp) {
  const int c = blockIdx.x * BCG_COLS + (threadIdx.x % BCG_COLS);
  const int rsub = threadIdx.x / BCG_COLS;
  if (c >= W) return;
  const int r0 = blockIdx.y * BCG_ROWS;
  const int r1 = min(n, r0 + BCG_ROWS);
  double dot = 0.0;
  for (int i = r0 + rsub; i < r1; i += blockDim.x / BCG_COLS) {
    double acc = 0.0;
    for (int q = ptr[i]; q < ptr[i + 1]; ++q) acc += val[q] * P[(size_t)col[q] * W + c];
    AP[(size_t)i * W + c] = acc;
    dot += P[(size_t)i * W + c] * acc;
  }
  atomicAdd(&pAp[c], dot);
}

// X += a P, R -= a AP, rr_new += R.R with a = rr / pAp.  A column whose residual has
// reached the tolerance is frozen: continuing CG on it once p^T A p has fallen to rounding
// level (or below zero on the singular Laplacian) makes the step explode.
__global__ void bcg_update_kernel(int n, int W, const double* __restrict__ rr, const double* __restrict__ pAp,
                                  const double* __restrict__ bb, double tol2, double* __restrict__ X,
                                  double* __restrict__ R, const double* __restrict__ P,
                                  const double* __restrict__ AP, double* __restrict__ rr_new) {
  const int c = blockIdx.x * BCG_COLS + (threadIdx.x % BCG_COLS);
  const int rsub = threadIdx.x / BCG_COLS;
  if (c >= W) return;
  if (rr[c] <= tol2 * bb[c]) {
    if (blockIdx.y == 0 && rsub == 0) rr_new[c] = rr[c];
    return;
  }
  const double d = pAp[c];
  const double a = d > 0.0 ? rr[c] / d : 0.0;
  const int r0 = blockIdx.y * BCG_ROWS;
  const int r1 = min(n, r0 + BCG_ROWS);
  double dot = 0.0;
  for (int i = r0 + rsub; i < r1; i += blockDim.x / BCG_COLS) {
    const size_t o = (size_t)i * W + c;
    X[o] += a * P[o];
    const double rv = R[o] - a * AP[o];
    R[o] = rv;
    dot += rv * rv;
  }
  atomicAdd(&rr_new[c], dot);
}

// P = R + (rr_new / rr) P (frozen columns keep P); zero pAp and the next accumulator
__global__ void bcg_direction_kernel(int n, int W, const double* __restrict__ rr, const double* __restrict__ rr_new,
                                     const double* __restrict__ bb, double tol2, const double* __restrict__ R,
                                     double* __restrict__ P, double* __restrict__ pAp, double* __restrict__ rr_next) {
  const int c = blockIdx.x * BCG_COLS + (threadIdx.x % BCG_COLS);
  const int rsub = threadIdx.x / BCG_COLS;
  if (c >= W) return;
  if (blockIdx.y == 0 && rsub == 0) {
    pAp[c] = 0.0;
    rr_next[c] = 0.0;
  }
  if (rr_new[c] <= tol2 * bb[c]) return;
  const double b = rr[c] > 0.0 ? rr_new[c] / rr[c] : 0.0;
  const int r0 = blockIdx.y * BCG_ROWS;
  const int r1 = min(n, r0 + BCG_ROWS);
  for (int i = r0 + rsub; i < r1; i += blockDim.x / BCG_COLS) {
    const size_t o = (size_t)i * W + c;
    P[o] = R[o] + b * P[o];
  }
}

__global__ void bcg_colsum_kernel(int n, int W, const double* __restrict__ X, double* __restrict__ sums) {
  const int c = blockIdx.x * BCG_COLS + (threadIdx.x % BCG_COLS);
  const int rsub = threadIdx.x / BCG_COLS;
  if (c >= W) return;
  const int r0 = blockIdx.y * BCG_ROWS;
  const int r1 = min(n, r0 + BCG_ROWS);
  double s = 0.0;
  for (int i = r0 + rsub; i < r1; i += blockDim.x / BCG_COLS) s += X[(size_t)i * W + c];
  atomicAdd(&sums[c], s);
}

// Xhi/Xlo[i, c0 + c] = X[i, c] - mean_c (projected case), split into FP32 hi + lo
__global__ void bcg_store_kernel(int n, int W, int c0, int ld, const double* __restrict__ X,
                                 const double* __restrict__ sums, bool project, float* __restrict__ Xhi,
                                 float* __restrict__ Xlo) {
  const int c = blockIdx.x * BCG_COLS + (threadIdx.x % BCG_COLS);
  const int rsub = threadIdx.x / BCG_COLS;
  if (c >= W) return;
  const double mean = project ? sums[c] / n : 0.0;
  const int r0 = blockIdx.y * BCG_ROWS;
  const int r1 = min(n, r0 + BCG_ROWS);
  for (int i = r0 + rsub; i < r1; i += blockDim.x / BCG_COLS) {
    const double v = X[(size_t)i * W + c] - mean;
    const float h = (float)v;
    Xhi[(size_t)i * ld + c0 + c] = h;
    Xlo[(size_t)i * ld + c0 + c] = (float)(v - (double)h);
  }
}

}  // namespace

cudaError_t dense_inverse_block_cg(const int32_t* ptr, const int32_t* col, const double* val, int n, bool project,
                                   double tol, int max_iter, float* Xhi, float* Xlo, int* iters, cudaStream_t s) {
  const int ld = padded_ld(n);
  // column block width: bound the four n x W work arrays to about 16 GB
  size_t cap = (size_t)16 << 30;
  int W = (int)std::min<size_t>((size_t)n, cap / (4 * sizeof(double) * (size_t)n));
  W = std::max(BCG_COLS, W / BCG_COLS * BCG_COLS);
  W = std::min(W, (n + BCG_COLS - 1) / BCG_COLS * BCG_COLS);
  double *X = nullptr, *R = nullptr, *P = nullptr, *AP = nullptr, *sc = nullptr;
  size_t bytes = (size_t)n * W * sizeof(double);
  cudaError_t err = cudaSuccess;
  auto fail = [&](cudaError_t e) {
    cudaFree(X);
    cudaFree(R);
    cudaFree(P);
    cudaFree(AP);
    cudaFree(sc);
    return e;
  };
  if ((err = cudaMalloc(&X, bytes)) != cudaSuccess) return fail(err);
  if ((err = cudaMalloc(&R, bytes)) != cudaSuccess) return fail(err);
  if ((err = cudaMalloc(&P, bytes)) != cudaSuccess) return fail(err);
  if ((err = cudaMalloc(&AP, bytes)) != cudaSuccess) return fail(err);
  // scalars: rr ring of 3, pAp, bb, sums
  if ((err = cudaMalloc(&sc, sizeof(double) * W * 6)) != cudaSuccess) return fail(err);
  double* ring = sc;              // 3 W
  double* pAp = sc + 3 * (size_t)W;
  double* bb = sc + 4 * (size_t)W;
  double* sums = sc + 5 * (size_t)W;
  std::vector<double> h_rr(W), h_bb(W);
  int worst_iters = 0;
  const int threads = 256;
  for (int c0 = 0; c0 < n; c0 += W) {
    const int w = std::min(W, n - c0);
    dim3 grid((w + BCG_COLS - 1) / BCG_COLS, (n + BCG_ROWS - 1) / BCG_ROWS);
    if ((err = cudaMemsetAsync(sc, 0, sizeof(double) * W * 6, s)) != cudaSuccess) return fail(err);
    bcg_init_kernel<<<grid, threads, 0, s>>>(n, w, c0, project, X, R, P, ring);
    if ((err = cudaMemcpyAsync(bb, ring, sizeof(double) * w, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return fail(err);
    if ((err = cudaMemcpyAsync(h_bb.data(), ring, sizeof(double) * w, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return fail(err);
    int it = 0;
    bool done = false;
    while (!done && it < max_iter) {
      double* rr = ring + (size_t)(it % 3) * W;
      double* rr_new = ring + (size_t)((it + 1) % 3) * W;
      double* rr_next = ring + (size_t)((it + 2) % 3) * W;
      {
        ProfScope prof("factor_bcg_spmm", 16.0 * n * w, 0.0, s);
        bcg_spmm_kernel<<<grid, threads, 0, s>>>(ptr, col, val, n, w, P, AP, pAp);
      }
      {
        ProfScope prof("factor_bcg_update", 48.0 * n * w, 0.0, s);
        bcg_update_kernel<<<grid, threads, 0, s>>>(n, w, rr, pAp, bb, tol * tol, X, R, P, AP, rr_new);
      }
      {
        ProfScope prof("factor_bcg_direction", 24.0 * n * w, 0.0, s);
        bcg_direction_kernel<<<grid, threads, 0, s>>>(n, w, rr, rr_new, bb, tol * tol, R, P, pAp, rr_next);
      }
      ++it;
      if (it % 16 == 0 || it == max_iter) {
        if ((err = cudaMemcpyAsync(h_rr.data(), rr_new, sizeof(double) * w, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
          return fail(err);
        if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return fail(err);
        double worst = 0.0;
        for (int c = 0; c < w; ++c) worst = std::max(worst, std::sqrt(h_rr[c] / std::max(h_bb[c], 1e-300)));
        done = worst <= tol;
      }
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return fail(err);
    worst_iters = std::max(worst_iters, it);
    if (project) {
      if ((err = cudaMemsetAsync(sums, 0, sizeof(double) * W, s)) != cudaSuccess) return fail(err);
      bcg_colsum_kernel<<<grid, threads, 0, s>>>(n, w, X, sums);
    }
    bcg_store_kernel<<<grid, threads, 0, s>>>(n, w, c0, ld, X, sums, project, Xhi, Xlo);
    if ((err = cudaGetLastError()) != cudaSuccess) return fail(err);
  }
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return fail(err);
  *iters = worst_iters;
  return fail(cudaSuccess);
}

}  // namespace rfcmp
