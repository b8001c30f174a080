// Device-resident CG with iterative refinement (Sec. 4: CG on the Hermitian positive definite
// RF-CMP system; mixed precision with accurate residual sweeps).
//
// Every per-column scalar, the convergence test, the active-column mask and the refinement
// decision live on the device.  The vector work of one CG iteration is three kernels:
//   cg_pap       <p, A p> per column                          -> alpha = rho / <p, A p>
//   cg_update    d += alpha p, r -= alpha A p, <r, r>         -> beta, rho, convergence, live count
//   cg_direction p = r + beta p
// and one refinement step is r = b - A i with its column norms and the decision for the next
// sweep (refine_residual).  Reductions are fixed-order: each block writes one partial per
// column, and the last block of the column (a ticket counter) sums the partials in block order,
// so a column's result does not depend on scheduling or on the other columns of the batch.
//
// The loop itself can run as nested WHILE conditional nodes of one CUDA graph: cg_update sets
// the inner condition, refine_residual the outer one.  Each body first sets its own condition
// to 0 (cg_pap for the inner loop, cg_start for the outer loop) and only the last block of the
// deciding kernel sets it to 1, bounded by the pass counters (at most max_passes inner passes,
// at most max_sweeps outer passes): if a decision kernel did not run, the loop ends.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "rfcmp_internal.h"

namespace rfcmp {

namespace {

constexpr int KT = 256;  // threads per block of the column kernels

__device__ __forceinline__ double2 warp_sum2(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// block-wide sum in a fixed order (lanes by xor tree, warps in index order); result in thread 0
__device__ double2 block_sum2(double2 v) {
  __shared__ double2 red[KT / 32];
  v = warp_sum2(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int w = 0; w < KT / 32; ++w) {
      t.x += red[w].x;
      t.y += red[w].y;
    }
  __syncthreads();
  return t;
}

// Writes this block's partial of column r and returns true in the column's last block, whose
// thread 0 then holds the fixed-order sum of all partials in *sum.
__device__ bool column_reduce(const KrylovView& K, int r, double2 partial, double2* sum) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    K.part[(size_t)r * gridDim.x + blockIdx.x] = partial;
    __threadfence();
    const unsigned t = atomicAdd(&K.ticket[r], 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  if (threadIdx.x == 0) {
    __threadfence();
    double2 s = make_double2(0.0, 0.0);
    for (unsigned b = 0; b < gridDim.x; ++b) {
      const double2 p = __ldcg(&K.part[(size_t)r * gridDim.x + b]);
      s.x += p.x;
      s.y += p.y;
    }
    *sum = s;
    K.ticket[r] = 0;
  }
  return true;
}

// One column finished its per-column step: returns true in the block that finished the last
// column (all per-column results of this launch are then visible to it).
__device__ bool all_columns_done(const KrylovView& K) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&K.ctl->gticket, 1u);
    last = (t == (unsigned)K.nr - 1);
    if (last) K.ctl->gticket = 0;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

__device__ __forceinline__ void set_cond(const KrylovView& K, cudaGraphConditionalHandle h, unsigned v) {
  if (K.graph) cudaGraphSetConditional(h, v);
}

// Refinement decision over all columns (one block, all threads): residuals, convergence, the
// active mask and the inner tolerance of the next sweep; sets the loop conditions.
__device__ void decide(const KrylovView& K) {
  KrylovCtl* c = K.ctl;
  __shared__ int s_live[KT / 32];
  __shared__ double s_worst[KT / 32];
  __shared__ int s_rem[KT / 32];
  int live = 0, rem = 0;
  double worst = 0.0;
  for (int r = threadIdx.x; r < K.nr; r += blockDim.x) {
    const double bb = __ldcg(&K.bb[r]), rr = __ldcg(&K.rr[r]);
    const double res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    const int conv = res <= c->tol;
    const int it = __ldcg(&K.iters[r]);
    const bool in = K.member == nullptr || __ldcg(&K.member[r]) != 0;
    // a column iterates while it is in the solve, above tol, and within its iteration and sweep
    // budgets (its own sweep count: in a batch session columns join at different sweeps)
    const int act = in && !conv && it < c->max_iter && __ldcg(&K.sweeps[r]) < c->max_sweeps;
    K.res[r] = res;
    K.conv[r] = conv;
    K.active[r] = act;
    K.rho[r] = rr;
    K.r0[r] = rr;
    if (act) {
      live++;
      worst = fmax(worst, res);
      rem = max(rem, c->max_iter - it);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    live += __shfl_xor_sync(0xffffffffu, live, o);
    rem = max(rem, __shfl_xor_sync(0xffffffffu, rem, o));
    worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  }
  if ((threadIdx.x & 31) == 0) {
    s_live[threadIdx.x >> 5] = live;
    s_rem[threadIdx.x >> 5] = rem;
    s_worst[threadIdx.x >> 5] = worst;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    live = rem = 0;
    worst = 0.0;
    for (int w = 0; w < KT / 32; ++w) {
      live += s_live[w];
      rem = max(rem, s_rem[w]);
      worst = fmax(worst, s_worst[w]);
    }
    const bool go = live > 0;
    double rel = 0.5 * c->tol;
    if (c->mixed) rel = fmin(fmax(c->inner_tol, 0.5 * c->tol / fmax(worst, 1e-300)), 0.5);
    c->tol2 = rel * rel;
    c->live = live;
    c->passes = 0;
    c->max_passes = rem;
    c->go = go ? 1 : 0;
    set_cond(K, K.h_outer, go ? 1u : 0u);
    set_cond(K, K.h_inner, go ? 1u : 0u);
  }
}

// ---------------------------------------------------------------- kernels
__global__ void __launch_bounds__(KT) solve_params_kernel(KrylovView K, double tol, double inner_tol, int max_iter,
                                                         int max_sweeps, int mixed) {
  RF_COUNT_LAUNCH();
  KrylovCtl* c = K.ctl;
  if (threadIdx.x == 0) {
    c->tol = tol;
    c->inner_tol = inner_tol;
    c->max_iter = max_iter;
    c->max_sweeps = max_sweeps;
    c->mixed = mixed;
    c->sweep = 0;
    c->passes = 0;
    c->max_passes = 0;
    c->live = 0;
    c->go = 0;
    c->gticket = 0;
  }
  for (int r = threadIdx.x; r < K.nr; r += blockDim.x) {
    K.iters[r] = 0;
    K.sweeps[r] = 0;
    K.ticket[r] = 0;
  }
}

// r = b - t (t = A i), or r = b and i = 0 (init); rr = ||r||^2 per column; then the decision.
// init also stores bb = ||b||^2.
__global__ void __launch_bounds__(KT) refine_residual_kernel(KrylovView K, const double2* __restrict__ b,
                                                            const double2* __restrict__ t, double2* __restrict__ rv,
                                                            double2* __restrict__ iv, int init) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.y;
  const size_t off = (size_t)r * K.n;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 v = b[off + i];
    if (init) {
      iv[off + i] = make_double2(0.0, 0.0);
    } else {
      const double2 a = t[off + i];
      v.x -= a.x;
      v.y -= a.y;
    }
    rv[off + i] = v;
    acc = fma(v.x, v.x, fma(v.y, v.y, acc));
  }
  double2 sum;
  const double2 p = block_sum2(make_double2(acc, 0.0));
  if (!column_reduce(K, r, p, &sum)) return;
  if (threadIdx.x == 0) {
    K.rr[r] = sum.x;
    if (init)
      K.bb[r] = sum.x;
    else if (K.member == nullptr || K.member[r])
      K.sweeps[r] += 1;
  }
  if (!all_columns_done(K)) return;
  if (threadIdx.x == 0 && !init) K.ctl->sweep += 1;
  __syncthreads();
  decide(K);
}

// start of a sweep's inner CG: d = 0, r_in = r, p = r; the outer condition reads "stop" until
// the sweep's decision sets it again
__global__ void __launch_bounds__(KT) cg_start_kernel(KrylovView K, const double2* __restrict__ rv,
                                                     double2* __restrict__ d, double2* __restrict__ rin,
                                                     double2* __restrict__ p) {
  RF_COUNT_LAUNCH();
  if ((blockIdx.x | blockIdx.y | threadIdx.x) == 0) set_cond(K, K.h_outer, 0u);
  const int r = blockIdx.y;
  const size_t off = (size_t)r * K.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = rv[off + i];
    d[off + i] = make_double2(0.0, 0.0);
    rin[off + i] = v;
    p[off + i] = v;
  }
}

// alpha = rho / <p, A p> for the active columns; the inner condition reads "stop" until
// cg_update sets it again
__global__ void __launch_bounds__(KT) cg_pap_kernel(KrylovView K, const double2* __restrict__ p,
                                                   const double2* __restrict__ Ap) {
  RF_COUNT_LAUNCH();
  if ((blockIdx.x | blockIdx.y | threadIdx.x) == 0) set_cond(K, K.h_inner, 0u);
  const int r = blockIdx.y;
  if (!__ldcg(&K.active[r])) return;
  const size_t off = (size_t)r * K.n;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = p[off + i], v = Ap[off + i];
    acc = fma(u.x, v.x, fma(u.y, v.y, acc));  // Re(p^H A p); A is Hermitian
  }
  double2 sum;
  const double2 part = block_sum2(make_double2(acc, 0.0));
  if (!column_reduce(K, r, part, &sum)) return;
  if (threadIdx.x == 0) K.alpha[r] = sum.x == 0.0 ? 0.0 : K.rho[r] / sum.x;
}

// d += alpha p, r_in -= alpha A p, rho' = ||r_in||^2, beta = rho'/rho; a column stops when
// rho' <= tol2 * rho_0, is not finite, or has spent max_iter iterations
__global__ void __launch_bounds__(KT) cg_update_kernel(KrylovView K, const double2* __restrict__ p,
                                                      const double2* __restrict__ Ap, double2* __restrict__ d,
                                                      double2* __restrict__ rin) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.y;
  if (!__ldcg(&K.active[r])) {
    if (blockIdx.x == 0) {
      if (!all_columns_done(K)) return;
    } else {
      return;
    }
  } else {
    const size_t off = (size_t)r * K.n;
    const double a = K.alpha[r];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += (int64_t)gridDim.x * blockDim.x) {
      const double2 u = p[off + i], v = Ap[off + i];
      double2 x = d[off + i], w = rin[off + i];
      x.x = fma(a, u.x, x.x);
      x.y = fma(a, u.y, x.y);
      w.x = fma(-a, v.x, w.x);
      w.y = fma(-a, v.y, w.y);
      d[off + i] = x;
      rin[off + i] = w;
      acc = fma(w.x, w.x, fma(w.y, w.y, acc));
    }
    double2 sum;
    const double2 part = block_sum2(make_double2(acc, 0.0));
    if (!column_reduce(K, r, part, &sum)) return;
    if (threadIdx.x == 0) {
      const double rn = sum.x, ro = K.rho[r];
      K.beta[r] = ro == 0.0 ? 0.0 : rn / ro;
      K.rho[r] = rn;
      const int it = K.iters[r] + 1;
      K.iters[r] = it;
      if (!(rn > K.ctl->tol2 * K.r0[r]) || !isfinite(rn) || it >= K.ctl->max_iter) K.active[r] = 0;
    }
    if (!all_columns_done(K)) return;
  }
  // last column done: live count and the inner condition
  __shared__ int s_live[KT / 32];
  int live = 0;
  for (int c = threadIdx.x; c < K.nr; c += blockDim.x) live += __ldcg(&K.active[c]) != 0;
  for (int o = 16; o > 0; o >>= 1) live += __shfl_xor_sync(0xffffffffu, live, o);
  if ((threadIdx.x & 31) == 0) s_live[threadIdx.x >> 5] = live;
  __syncthreads();
  if (threadIdx.x == 0) {
    live = 0;
    for (int w = 0; w < KT / 32; ++w) live += s_live[w];
    KrylovCtl* c = K.ctl;
    c->passes += 1;
    c->live = live;
    set_cond(K, K.h_inner, (live > 0 && c->passes < c->max_passes) ? 1u : 0u);
  }
}

// p = r_in + beta p for the columns still active
__global__ void __launch_bounds__(KT) cg_direction_kernel(KrylovView K, const double2* __restrict__ rin,
                                                         double2* __restrict__ p) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.y;
  if (!__ldcg(&K.active[r])) return;
  const size_t off = (size_t)r * K.n;
  const double bta = K.beta[r];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = rin[off + i];
    double2 v = p[off + i];
    v.x = fma(bta, v.x, u.x);
    v.y = fma(bta, v.y, u.y);
    p[off + i] = v;
  }
}

// i += d (every column; d is zero where a column did not iterate)
__global__ void __launch_bounds__(KT) add_cols_kernel(KrylovView K, const double2* __restrict__ d,
                                                     double2* __restrict__ iv) {
  RF_COUNT_LAUNCH();
  const int r = blockIdx.y;
  const size_t off = (size_t)r * K.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = d[off + i];
    double2 v = iv[off + i];
    v.x += u.x;
    v.y += u.y;
    iv[off + i] = v;
  }
}

__global__ void __launch_bounds__(KT) decide_kernel(KrylovView K) {
  RF_COUNT_LAUNCH();
  decide(K);
}

__global__ void __launch_bounds__(KT) slots_kernel(KrylovView K, const int* __restrict__ slots, int n,
                                                  const double2* __restrict__ dots) {
  RF_COUNT_LAUNCH();
  int* member = const_cast<int*>(K.member);
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int r = slots[q];
    const double v = dots ? dots[q].x : 0.0;
    K.bb[r] = v;
    K.rr[r] = v;
    K.rho[r] = v;
    K.r0[r] = v;
    K.iters[r] = 0;
    K.sweeps[r] = 0;
    K.conv[r] = 0;
    K.active[r] = 0;
    K.res[r] = dots ? 1.0 : 0.0;
    member[r] = dots ? 1 : 0;
  }
}

inline dim3 col_grid(const KrylovView& K) { return dim3(K.G, K.nr); }

}  // namespace

int krylov_blocks_per_column(int64_t n) {
  const int64_t b = (n + 4 * KT - 1) / (4 * KT);
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, KRYLOV_MAX_G));
}

cudaError_t krylov_params(const KrylovView& K, double tol, double inner_tol, int max_iter, int max_sweeps, bool mixed,
                          cudaStream_t s) {
  solve_params_kernel<<<1, KT, 0, s>>>(K, tol, inner_tol, max_iter, max_sweeps, mixed ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t krylov_refine_residual(const KrylovView& K, const double2* b, const double2* t, double2* r, double2* i,
                                   bool init, cudaStream_t s) {
  refine_residual_kernel<<<col_grid(K), KT, 0, s>>>(K, b, t, r, i, init ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t krylov_cg_start(const KrylovView& K, const double2* r, double2* d, double2* rin, double2* p,
                            cudaStream_t s) {
  cg_start_kernel<<<col_grid(K), KT, 0, s>>>(K, r, d, rin, p);
  return cudaGetLastError();
}
cudaError_t krylov_cg_pap(const KrylovView& K, const double2* p, const double2* Ap, cudaStream_t s) {
  cg_pap_kernel<<<col_grid(K), KT, 0, s>>>(K, p, Ap);
  return cudaGetLastError();
}
cudaError_t krylov_cg_update(const KrylovView& K, const double2* p, const double2* Ap, double2* d, double2* rin,
                             cudaStream_t s) {
  cg_update_kernel<<<col_grid(K), KT, 0, s>>>(K, p, Ap, d, rin);
  return cudaGetLastError();
}
cudaError_t krylov_cg_direction(const KrylovView& K, const double2* rin, double2* p, cudaStream_t s) {
  cg_direction_kernel<<<col_grid(K), KT, 0, s>>>(K, rin, p);
  return cudaGetLastError();
}
cudaError_t krylov_decide(const KrylovView& K, cudaStream_t s) {
  decide_kernel<<<1, KT, 0, s>>>(K);
  return cudaGetLastError();
}
cudaError_t krylov_slots(const KrylovView& K, const int* slots, int n, const double2* dots, cudaStream_t s) {
  if (!K.member) return cudaErrorInvalidValue;
  slots_kernel<<<1, KT, 0, s>>>(K, slots, n, dots);
  return cudaGetLastError();
}
cudaError_t krylov_add(const KrylovView& K, const double2* d, double2* i, cudaStream_t s) {
  add_cols_kernel<<<col_grid(K), KT, 0, s>>>(K, d, i);
  return cudaGetLastError();
}

RF_LAUNCH_READER(launches_krylov)

}  // namespace rfcmp
