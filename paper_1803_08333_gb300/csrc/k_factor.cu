// Dense (Sigma^T Sigma)^+ by Newton-Schulz refinement on the tensor cores.
//
// With M = Sigma^T Sigma + 1 1^T / n, the identity of Sec. 3.2 gives
// (Sigma^T Sigma)^+ = M^{-1} - 1 1^T / n.  The start X0 ~ M^{-1} is one symmetric multigrid
// V(1,1) cycle applied to the projected identity (a convergent V-cycle B has the eigenvalues of
// M B in (0, 2), so the spectral radius of I - M X0 is below 1), or a loose multigrid-PCG solve;
// then
//     R_k = I - M X_k   (FP64, formed exactly along rows: (X M)_ij = sum_k X_ik M_kj, M sparse),
//     X_{k+1} = X_k + X_k R_k   (dense product, split-BF16 tensor-core GEMM, FP64 update; X_k R_k
//                                is symmetric, so only its upper tiles are computed)
// converges quadratically: the relative error e_k of X_k obeys e_{k+1} <= e_k^2 + c e_k with
// c ~ 2^-16 the accuracy of one split product.  A V-cycle start leaves the smallest eigenvalue a
// of M X0 near 0.02, where plain steps only double it; so after one plain step (which puts the
// spectrum in (0, 1]) the lower end a is estimated by a few power steps on I - M X and the next
// steps are scaled (X <- alpha X (2 I - alpha M X), alpha = 2 / (1 + a)), which roughly
// quadruples a per step until it nears 1; plain quadratic steps finish.  X_k stays exactly
// symmetric (the update mirrors the upper tiles; the residual below is formed along rows, as
// R^T, which needs it); a plain iteration that stops contracting ends early so that the caller
// can fall back to a PCG solve.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rfcmp_internal.h"

namespace rfcmp {

namespace {

// Rt[i][j] = delta_ij - alpha (X M)[i][j] with M = L + 1 1^T / n (L symmetric CSR; without
// rowsum, M = L), written as BF16 hi/lo planes; rowsum[i] = sum_j X[i][j] is precomputed.  Also
// tracks max |Rt|.  The FP64 sums bound this kernel (GB300's FP64 pipe runs at a small
// fraction of the FP32 rate), so everything else stays off that pipe: the maximum is taken on
// the FP32 value and reduced per CTA before its single atomic.  A CTA sweeps part of one row i,
// whose gathers X[i][col] the CTA's L1 keeps.
constexpr int NSR_THREADS = 256;
constexpr int NSR_SPLIT = 8;  // CTAs per row
__global__ void __launch_bounds__(NSR_THREADS)
ns_residual_kernel(const double* __restrict__ X, long long ldx, int n, const int32_t* __restrict__ ptr,
                   const int32_t* __restrict__ col, const double* __restrict__ val,
                   const double* __restrict__ rowsum, double alpha, __nv_bfloat16* __restrict__ hi,
                   __nv_bfloat16* __restrict__ lo, long long ldp, unsigned long long* __restrict__ maxbits) {
  RF_COUNT_LAUNCH();
  const int i = blockIdx.y;
  const double* xr = X + (size_t)i * ldx;
  const double rs = rowsum ? rowsum[i] / n : 0.0;  // the 1 1^T / n term of the projected case
  float mx = 0.f;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double a = rs;
    for (int q = ptr[j]; q < ptr[j + 1]; ++q) a += xr[col[q]] * val[q];  // (X L)_ij, L symmetric
    const double r = (i == j ? 1.0 : 0.0) - alpha * a;
    const float rf = (float)r;
    const __nv_bfloat16 h = __float2bfloat16_rn(rf);
    hi[(size_t)i * ldp + j] = h;
    lo[(size_t)i * ldp + j] = __float2bfloat16_rn(rf - __bfloat162float(h));
    mx = fmaxf(mx, fabsf(rf));
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  __shared__ float wmax[NSR_THREADS / 32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < NSR_THREADS / 32; ++w) m = fmaxf(m, wmax[w]);
    atomicMax(maxbits, (unsigned long long)__double_as_longlong((double)m));
  }
}

__global__ void row_sum_kernel(const double* __restrict__ X, long long ldx, int n, double* __restrict__ out) {
  RF_COUNT_LAUNCH();
  const int i = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) s += X[(size_t)i * ldx + j];
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[i] = t;
  }
}

// out = (X + X^T)/2 - shift, split into FP32 hi + lo planes (row stride ld)
constexpr int TT = 32;
__global__ void symmetrize_store_kernel(const double* __restrict__ X, long long ldx, int n, double shift,
                                        float* __restrict__ hi, float* __restrict__ lo, long long ld) {
  RF_COUNT_LAUNCH();
  __shared__ double tile[TT][TT + 1];
  const int bi = blockIdx.y * TT, bj = blockIdx.x * TT;
  // load the transposed tile X[bj.., bi..]
  for (int r = threadIdx.y; r < TT; r += blockDim.y) {
    const int row = bj + r, c = bi + threadIdx.x;
    tile[r][threadIdx.x] = (row < n && c < n) ? X[(size_t)row * ldx + c] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < TT; r += blockDim.y) {
    const int i = bi + r, j = bj + threadIdx.x;
    if (i < n && j < n) {
      const double v = 0.5 * (X[(size_t)i * ldx + j] + tile[threadIdx.x][r]) - shift;
      const float h = (float)v;
      hi[(size_t)i * ld + j] = h;
      lo[(size_t)i * ld + j] = (float)(v - (double)h);
    }
  }
}

// X <- (X + X^T) / 2 in place: block (bx, by), by <= bx, averages tile (by, bx) with the
// transpose of tile (bx, by) and writes both
__global__ void symmetrize_inplace_kernel(double* __restrict__ X, long long ldx, int n) {
  RF_COUNT_LAUNCH();
  __shared__ double a[TT][TT + 1], b[TT][TT + 1];
  const int bx = blockIdx.x, by = blockIdx.y;
  if (by > bx) return;
  const int r0 = by * TT, c0 = bx * TT;  // tile a = X[r0.., c0..], tile b = X[c0.., r0..]
  for (int r = threadIdx.y; r < TT; r += blockDim.y) {
    const int i = r0 + r, j = c0 + threadIdx.x;
    a[r][threadIdx.x] = (i < n && j < n) ? X[(size_t)i * ldx + j] : 0.0;
    const int i2 = c0 + r, j2 = r0 + threadIdx.x;
    b[r][threadIdx.x] = (i2 < n && j2 < n) ? X[(size_t)i2 * ldx + j2] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < TT; r += blockDim.y) {
    const int i = r0 + r, j = c0 + threadIdx.x;
    const double v = 0.5 * (a[r][threadIdx.x] + b[threadIdx.x][r]);
    if (i < n && j < n) X[(size_t)i * ldx + j] = v;
    const int i2 = c0 + r, j2 = r0 + threadIdx.x;
    const double w = 0.5 * (b[r][threadIdx.x] + a[threadIdx.x][r]);
    if (i2 < n && j2 < n) X[(size_t)i2 * ldx + j2] = w;
  }
}

// X <- alpha (X + D) for a symmetric D of which only the 128 x 128 tiles on or above the diagonal
// were computed: block (bx, by), by <= bx, adds tile (by, bx) of D to X there and its transpose
// to tile (bx, by); a diagonal tile adds (D + D^T) / 2, so X stays exactly symmetric.  !SCALED:
// alpha = 1 (a plain step), one FP64 operation fewer per entry.
template <bool SCALED>
__global__ void ns_update_sym_kernel(double* __restrict__ X, long long ldx, const float* __restrict__ D, long long ldd,
                                     int n, double alpha) {
  RF_COUNT_LAUNCH();
  __shared__ float t[TT][TT + 1];
  const int bx = blockIdx.x, by = blockIdx.y;
  if (by > bx) return;
  const int r0 = by * TT, c0 = bx * TT;
  for (int r = threadIdx.y; r < TT; r += blockDim.y) {
    const int i = r0 + r, j = c0 + threadIdx.x;
    t[r][threadIdx.x] = (i < n && j < n) ? D[(size_t)i * ldd + j] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < TT; r += blockDim.y) {
    const int c = threadIdx.x;
    const int i = r0 + r, j = c0 + c;
    if (i < n && j < n) {
      double* x = X + (size_t)i * ldx + j;
      const double v = *x + (bx == by ? 0.5 * ((double)t[r][c] + (double)t[c][r]) : (double)t[r][c]);
      *x = SCALED ? alpha * v : v;
    }
    const int i2 = c0 + r, j2 = r0 + c;
    if (bx != by && i2 < n && j2 < n) {
      double* x = X + (size_t)i2 * ldx + j2;
      const double v = *x + (double)t[c][r];
      *x = SCALED ? alpha * v : v;
    }
  }
}

// u = X v (dense FP64, one warp per row); sum += sum_i u_i
__global__ void dmatvec_kernel(const double* __restrict__ X, long long ldx, int n, const double* __restrict__ v,
                               double* __restrict__ u, double* __restrict__ sum) {
  RF_COUNT_LAUNCH();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* xr = X + (size_t)warp * ldx;
  double a = 0.0;
  for (int j = lane; j < n; j += 32) a = fma(xr[j], v[j], a);
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
  if (lane == 0) {
    u[warp] = a;
    atomicAdd(sum, a);
  }
}

// w = v - (L u + (sum / n) 1 if project); norm2 += |w|^2
__global__ void resid_vec_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, int n, int project, const double* __restrict__ v,
                                 const double* __restrict__ u, const double* __restrict__ sum,
                                 double* __restrict__ w, double* __restrict__ norm2) {
  RF_COUNT_LAUNCH();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double d = 0.0;
  if (i < n) {
    double a = project ? *sum / n : 0.0;
    for (int q = ptr[i]; q < ptr[i + 1]; ++q) a += val[q] * u[col[q]];
    const double r = v[i] - a;
    w[i] = r;
    d = r * r;
  }
  for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(norm2, d);
}

__global__ void scale_vec_kernel(int n, double c, const double* __restrict__ w, double* __restrict__ v) {
  RF_COUNT_LAUNCH();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = c * w[i];
}

// X = c D^{-1} (D the diagonal of the CSR matrix), the rest of X zero
__global__ void jacobi_start_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, int n, double c, double* __restrict__ X,
                                    long long ldx) {
  RF_COUNT_LAUNCH();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int q = ptr[i]; q < ptr[i + 1]; ++q)
      if (col[q] == i) d = val[q];
    X[(size_t)i * ldx + i] = d > 0.0 ? c / d : 0.0;
  }
}

}  // namespace

cudaError_t jacobi_start(const int32_t* ptr, const int32_t* col, const double* val, int n, double c, double* X,
                         long long ldx, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(X, 0, sizeof(double) * (size_t)n * ldx, s);
  if (err != cudaSuccess) return err;
  jacobi_start_kernel<<<(n + 255) / 256, 256, 0, s>>>(ptr, col, val, n, c, X, ldx);
  return cudaGetLastError();
}

cudaError_t newton_schulz_pseudo_inverse(const int32_t* ptr, const int32_t* col, const double* val, int n,
                                         bool project, double* X, long long ldx, int max_steps, double tol, float* Xhi,
                                         float* Xlo, int* steps_done, double* final_residual, cudaStream_t s) {
  // X holds an approximation of M^{-1} on entry (row-major, stride ldx): M = L + 1 1^T / n with
  // project (the result is M^{-1} - 1 1^T / n = L^+), M = L without
  const long long ldp = ldx;  // plane stride (elements); ldx is a multiple of 64
  std::vector<void*> own;
  auto fail = [&](cudaError_t e) {
    for (void* p : own) dev_free(p);
    return e;
  };
  cudaError_t err;
  __nv_bfloat16 *xh, *xl, *rh, *rl;
  float* D;
  double* rowsum;
  unsigned long long* maxbits;
  int* gerr;
  const size_t plane = (size_t)n * ldp;
  for (__nv_bfloat16** p : {&xh, &xl, &rh, &rl}) {
    if ((err = dev_malloc(p, plane * sizeof(__nv_bfloat16))) != cudaSuccess) return fail(err);
    own.push_back(*p);
  }
  if ((err = dev_malloc(&D, plane * sizeof(float))) != cudaSuccess) return fail(err);
  own.push_back(D);
  if ((err = dev_malloc(&rowsum, n * sizeof(double))) != cudaSuccess) return fail(err);
  own.push_back(rowsum);
  if ((err = dev_malloc(&maxbits, sizeof(unsigned long long))) != cudaSuccess) return fail(err);
  own.push_back(maxbits);
  if ((err = dev_malloc(&gerr, sizeof(int))) != cudaSuccess) return fail(err);
  own.push_back(gerr);
  if ((err = cudaMemsetAsync(gerr, 0, sizeof(int), s)) != cudaSuccess) return fail(err);
  SplitOperand A, B;
  A.hi = xh;
  A.lo = xl;
  A.rows = n;
  A.ld = ldp;
  B.hi = rh;
  B.lo = rl;
  B.rows = n;
  B.ld = ldp;
  // vectors of the spectral-radius estimate: v, u, w (n each) and two scalars
  double* pv;
  if ((err = dev_malloc(&pv, (3 * (size_t)n + 2) * sizeof(double))) != cudaSuccess) return fail(err);
  own.push_back(pv);
  double *pu = pv + n, *pw = pv + 2 * (size_t)n, *psc = pv + 3 * (size_t)n;
  // rho(I - M X) by a few power steps on I - M X (matrix-free: one dense FP64 product with X and
  // one sparse product with M per step).  Any bound a in (0, 1) keeps the scaled steps
  // convergent.
  auto estimate_rho = [&](double& rho) -> cudaError_t {
    std::vector<double> h(n);
    for (int i = 0; i < n; ++i) h[i] = 1.0 + 0.5 * std::sin(0.7 * i) + 0.25 * std::cos(1.3 * i + 0.4);
    double nrm = 0.0;
    for (double x : h) nrm += x * x;
    for (double& x : h) x /= std::sqrt(nrm);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(pv, h.data(), n * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    rho = 0.0;
    for (int it = 0; it < 12; ++it) {
      if ((e = cudaMemsetAsync(psc, 0, 2 * sizeof(double), s)) != cudaSuccess) return e;
      dmatvec_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(X, ldx, n, pv, pu, psc);
      resid_vec_kernel<<<(n + 255) / 256, 256, 0, s>>>(ptr, col, val, n, project ? 1 : 0, pv, pu, psc, pw, psc + 1);
      double nw2 = 0.0;
      if ((e = cudaMemcpyAsync(&nw2, psc + 1, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
      rho = std::sqrt(nw2);
      if (!(rho > 0.0)) break;
      scale_vec_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, 1.0 / rho, pw, pv);
    }
    return cudaGetLastError();
  };
  double res = 1.0, prev = 1.0;
  bool prev_plain = false;
  double alpha = 1.0, a = -1.0;  // scaling of the next step; lower bound on the spectrum of M X
  int k = 0;
  const dim3 sgrid((n + TT - 1) / TT, (n + TT - 1) / TT), sblock(TT, 8);
  // the residual below is formed along rows as I - X M, which is R^T only for symmetric X
  symmetrize_inplace_kernel<<<sgrid, sblock, 0, s>>>(X, ldx, n);
  for (;; ++k) {
    if (project) row_sum_kernel<<<n, 256, 0, s>>>(X, ldx, n, rowsum);
    if ((err = cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), s)) != cudaSuccess) return fail(err);
    {
      ProfScope prof("factor_ns_residual", 16.0 * (double)n * n, 0.0, s);
      dim3 grid(std::min((n + NSR_THREADS - 1) / NSR_THREADS, NSR_SPLIT), n);
      ns_residual_kernel<<<grid, NSR_THREADS, 0, s>>>(X, ldx, n, ptr, col, val, project ? rowsum : nullptr, alpha, rh, rl,
                                              ldp, maxbits);
    }
    unsigned long long hb = 0;
    if ((err = cudaMemcpyAsync(&hb, maxbits, sizeof(hb), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return fail(err);
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return fail(err);
    const bool plain = alpha == 1.0;
    if (plain) {  // the residual of the current iterate: stop and contraction checks
      std::memcpy(&res, &hb, sizeof(res));
      if (!(res > tol)) break;
      if (prev_plain && k >= 2 && !(res < 0.9 * prev)) break;  // not contracting: the caller falls back
      prev = res;
    }
    prev_plain = plain;
    if (k >= max_steps) break;
    if ((err = split_bf16_f64(X, ldx, n, n, xh, xl, ldp, s)) != cudaSuccess) return fail(err);
    // D = X R' with B = R'^T stored row-major, R' = I - alpha M X; X R' is symmetric, so only the
    // tiles on and above the diagonal are computed; then X <- alpha (X + D)
    if ((err = gemm_bf16x3(&A, &B, nullptr, 1, n, n, n, D, ldp, false, gerr, s, 0, true)) != cudaSuccess)
      return fail(err);
    {
      ProfScope prof("factor_ns_update", 12.0 * (double)n * n, 0.0, s);
      if (alpha == 1.0) ns_update_sym_kernel<false><<<sgrid, sblock, 0, s>>>(X, ldx, D, ldp, n, alpha);
      else ns_update_sym_kernel<true><<<sgrid, sblock, 0, s>>>(X, ldx, D, ldp, n, alpha);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return fail(err);
    // scaling of the next step (scaled Newton-Schulz): with the spectrum of M X in [a, 1], the
    // step X <- alpha X (2 I - alpha M X), alpha = 2 / (1 + a), maps it into [a', 1] with
    // a' = alpha a (2 - alpha a), which grows about four-fold per step while a is small
    if (k == 0) {  // after one plain step the spectrum lies in (0, 1]: estimate its lower end
      double rho = 1.0;
      if ((err = estimate_rho(rho)) != cudaSuccess) return fail(err);
      // the power steps approach rho from below, so 1 - rho can overstate the true lower end;
      // an overstated bound ends the scaled steps too early, an understated one only costs a
      // fraction of a step (the bound roughly quadruples per step), so take half of it
      a = 0.5 * (1.0 - rho);
    } else if (!plain) {
      a = alpha * a * (2.0 - alpha * a);
    }
    alpha = (a > 1e-6 && a < 0.95) ? 2.0 / (1.0 + a) : 1.0;
  }
  int herr = 0;
  if ((err = cudaMemcpyAsync(&herr, gerr, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return fail(err);
  {
    dim3 grid((n + TT - 1) / TT, (n + TT - 1) / TT), block(TT, 8);
    symmetrize_store_kernel<<<grid, block, 0, s>>>(X, ldx, n, project ? 1.0 / n : 0.0, Xhi, Xlo, ldx);
  }
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return fail(err);
  if (herr) return fail(cudaErrorLaunchTimeout);
  *steps_done = k;
  *final_residual = res;
  return fail(cudaSuccess);
}

RF_LAUNCH_READER(launches_factor)

}  // namespace rfcmp
