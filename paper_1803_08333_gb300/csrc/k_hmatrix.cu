// Compressed T_A and V (Sec. 4: the system matrix compressed by an adaptive cross approximation at
// tolerance 1e-4; at extremely low frequency the vector potential compressed apart from the scalar
// one).  Each of T_A (RWG functions) and V (cells) becomes a symmetric hierarchical matrix: a
// cluster tree of its index set, the blocks of the block tree on and above the block diagonal, the
// admissible ones as low-rank crosses U Vt found by ACA with partial pivoting on the GPU, the rest
// dense; a block off the diagonal also stands for its transpose below it, so the compressed
// matrices stay exactly complex symmetric like T_A and V.
//
// Host: cluster trees (median bisection across the longest side of the item centres' extent, items
// carrying support boxes), the admissibility test min(diam a, diam b) <= eta dist(a, b) on
// boxes that do not touch (dist > 0), the block list.  Device: one CTA per admissible block runs the cross approximation on the
// resident dense matrix (rows and columns gathered through the cluster permutation), blocks whose
// crosses reach the rank cap, or would take at least the block's own entries, stay dense, and the factors and dense blocks are packed into one
// buffer per matrix.  The product y = H x gathers x into cluster order, runs one CTA per (block,
// column) with FP64 accumulation and FP64 atomics into y, and scatters back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "rfcmp_internal.h"

namespace rfcmp {

RF_LAUNCH_READER(launches_hmatrix)

// ---------------------------------------------------------------- host partition
namespace {

struct HmNode {
  int start = 0, stop = 0;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int child[2] = {-1, -1};
  double diam() const {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) s += (hi[d] - lo[d]) * (hi[d] - lo[d]);
    return std::sqrt(s);
  }
};

// Recursive bisection: a cluster of more than `leaf` items is sorted (stably) along the axis of
// the largest extent of its item centres and split at the middle position.
int build_tree(const double* cen, const double* slo, const double* shi, int start, int stop, int leaf,
               std::vector<int32_t>& perm, std::vector<HmNode>& nodes) {
  const int id = (int)nodes.size();
  nodes.emplace_back();
  HmNode node;
  node.start = start;
  node.stop = stop;
  for (int d = 0; d < 3; ++d) {
    node.lo[d] = HUGE_VAL;
    node.hi[d] = -HUGE_VAL;
  }
  double clo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, chi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
  for (int p = start; p < stop; ++p) {
    const int i = perm[p];
    for (int d = 0; d < 3; ++d) {
      node.lo[d] = std::min(node.lo[d], slo[3 * i + d]);
      node.hi[d] = std::max(node.hi[d], shi[3 * i + d]);
      clo[d] = std::min(clo[d], cen[3 * i + d]);
      chi[d] = std::max(chi[d], cen[3 * i + d]);
    }
  }
  if (stop - start > leaf) {
    int axis = 0;  // the first axis of the largest extent
    for (int d = 1; d < 3; ++d)
      if (chi[d] - clo[d] > chi[axis] - clo[axis]) axis = d;
    std::stable_sort(perm.begin() + start, perm.begin() + stop,
                     [&](int32_t a, int32_t b) { return cen[3 * a + axis] < cen[3 * b + axis]; });
    const int mid = start + (stop - start) / 2;
    node.child[0] = build_tree(cen, slo, shi, start, mid, leaf, perm, nodes);
    node.child[1] = build_tree(cen, slo, shi, mid, stop, leaf, perm, nodes);
  }
  nodes[id] = node;
  return id;
}

double box_distance(const HmNode& a, const HmNode& b) {
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double g = std::max(0.0, std::max(a.lo[d] - b.hi[d], b.lo[d] - a.hi[d]));
    s += g * g;
  }
  return std::sqrt(s);
}

struct HmBlockHost {
  int r0, r1, c0, c1;
  int admissible;
};

// Leaves of the block tree on and above the block diagonal (r0 <= c0), ordered by (r0, c0).  A pair
// that is not admissible splits into the children of whichever clusters have children; two leaves
// that are not admissible form a dense block.
std::vector<HmBlockHost> block_list(const std::vector<HmNode>& nodes, double eta) {
  std::vector<HmBlockHost> out;
  if (nodes.empty() || nodes[0].stop == 0) return out;
  std::vector<std::pair<int, int>> stack{{0, 0}};
  while (!stack.empty()) {
    const auto [ia, ib] = stack.back();
    stack.pop_back();
    const HmNode &a = nodes[ia], &b = nodes[ib];
    if (a.start > b.start) continue;  // below the diagonal: the transpose of a mirrored block
    const double dist = box_distance(a, b);
    if (dist > 0.0 && std::min(a.diam(), b.diam()) <= eta * dist) {  // boxes that touch: never
      out.push_back({a.start, a.stop, b.start, b.stop, 1});
    } else if (a.child[0] < 0 && b.child[0] < 0) {
      out.push_back({a.start, a.stop, b.start, b.stop, 0});
    } else {
      const int as[2] = {a.child[0] < 0 ? ia : a.child[0], a.child[1]};
      const int bs[2] = {b.child[0] < 0 ? ib : b.child[0], b.child[1]};
      const int na = a.child[0] < 0 ? 1 : 2, nb = b.child[0] < 0 ? 1 : 2;
      for (int x = 0; x < na; ++x)
        for (int y = 0; y < nb; ++y) stack.push_back({as[x], bs[y]});
    }
  }
  std::sort(out.begin(), out.end(), [](const HmBlockHost& p, const HmBlockHost& q) {
    return p.r0 != q.r0 ? p.r0 < q.r0 : p.c0 < q.c0;
  });
  return out;
}

int check_partition_args(int64_t n, int32_t leaf, double eta) {
  if (n < 0 || n > (int64_t)INT32_MAX) return set_error(RFCMP_ERR_INVALID_ARG, "item count out of range");
  if (leaf < 1 || leaf > 65536) return set_error(RFCMP_ERR_INVALID_ARG, "leaf must be in [1, 65536]");
  if (!(eta >= 0.0) || !std::isfinite(eta)) return set_error(RFCMP_ERR_INVALID_ARG, "eta must be finite and >= 0");
  return RFCMP_OK;
}

void partition(const double* cen, const double* slo, const double* shi, int n, int leaf, double eta,
               std::vector<int32_t>& perm, std::vector<HmBlockHost>& blocks) {
  perm.resize(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  std::vector<HmNode> nodes;
  if (n > 0) build_tree(cen, slo, shi, 0, n, leaf, perm, nodes);
  blocks = block_list(nodes, eta);
}

}  // namespace
}  // namespace rfcmp

// ---------------------------------------------------------------- device
namespace rfcmp {
namespace {

constexpr int HM_THREADS = 256;
constexpr int HM_MAX_RANK = 256;              // largest rank cap a caller may ask for
constexpr int HM_MAX_ITER = HM_MAX_RANK + 16;  // crosses plus rows skipped for a zero residual
constexpr unsigned FULL = 0xffffffffu;

// one block of the compressed form: rows [r0, r1) and columns [c0, c1) in cluster order; rank < 0
// for a dense block (m x n row-major at off), else U (rank x m, one cross per row of U) at off and
// Vt (rank x n) at off + rank m
struct HmBlockDev {
  int32_t r0, r1, c0, c1;
  int32_t rank, pad;
  long long off;
};

__device__ __forceinline__ void argmax_merge(float& v, int& i, float v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

// largest v over the CTA (ties: smallest i); every thread receives it
__device__ void block_argmax(float v, int i, float* sv, int* si, float& bv, int& bi) {
  for (int o = 16; o > 0; o >>= 1) argmax_merge(v, i, __shfl_down_sync(FULL, v, o), __shfl_down_sync(FULL, i, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sv[w] = v;
    si[w] = i;
  }
  __syncthreads();
  if (w == 0) {
    v = l < HM_THREADS / 32 ? sv[l] : -1.f;
    i = l < HM_THREADS / 32 ? si[l] : INT_MAX;
    for (int o = 16; o > 0; o >>= 1) argmax_merge(v, i, __shfl_down_sync(FULL, v, o), __shfl_down_sync(FULL, i, o));
    if (l == 0) {
      sv[HM_THREADS / 32] = v;
      si[HM_THREADS / 32] = i;
    }
  }
  __syncthreads();
  bv = sv[HM_THREADS / 32];
  bi = si[HM_THREADS / 32];
  __syncthreads();
}

// sums of four values over the CTA; every thread receives them
__device__ void block_sum4(double (&a)[4], double (*sd)[HM_THREADS / 32 + 1]) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(FULL, a[k], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) sd[k][w] = a[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double x = l < HM_THREADS / 32 ? sd[k][l] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(FULL, x, o);
      if (l == 0) sd[k][HM_THREADS / 32] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = sd[k][HM_THREADS / 32];
  __syncthreads();
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ bool row_used(const int* used, int nused, int p) {
  for (int k = 0; k < nused; ++k)
    if (used[k] == p) return true;
  return false;
}

// ACA with partial pivoting of one admissible block per CTA, on the dense matrix A (row stride
// ld) through the cluster permutation.  The crosses go to the block's slot: U (cap x m) at
// slot[b], Vt (cap x n) after it.  rank_out[b] = crosses kept, status_out[b] = 0 when the
// stopping rule ||u|| ||v|| <= eps ||S||_F held (or every row was used), 1 when the rank cap or
// the iteration cap ended the loop first.  All loops are bounded by the caps and the block's size.
__global__ void __launch_bounds__(HM_THREADS)
    hm_aca_kernel(const float2* __restrict__ A, long long ld, const int32_t* __restrict__ perm,
                  const HmBlockDev* __restrict__ blk, const long long* __restrict__ slot, int cap, int iter_cap,
                  float eps, float2* __restrict__ slots, int32_t* __restrict__ rank_out,
                  int32_t* __restrict__ status_out) {
  RF_COUNT_LAUNCH();
  __shared__ float sv[HM_THREADS / 32 + 1];
  __shared__ int si[HM_THREADS / 32 + 1];
  __shared__ double sd[4][HM_THREADS / 32 + 1];
  __shared__ int used[HM_MAX_ITER];
  __shared__ int s_next;
  const HmBlockDev B = blk[blockIdx.x];
  const int m = B.r1 - B.r0, n = B.c1 - B.c0, tid = threadIdx.x;
  const int32_t* rp = perm + B.r0;
  const int32_t* cp = perm + B.c0;
  float2* U = slots + slot[blockIdx.x];
  float2* Vt = U + (size_t)cap * m;
  int rank = 0, nused = 0, status = 1, i = 0;
  double norm2 = 0.0;  // ||S_rank||_F^2, the same in every thread
  for (int it = 0; it < iter_cap && rank < cap; ++it) {
    if (tid == 0) used[nused] = i;
    ++nused;
    // residual row i into the next cross's Vt row, and its largest entry
    float bv = -1.f;
    int bj = INT_MAX;
    const float2* Arow = A + (size_t)rp[i] * ld;
    for (int j = tid; j < n; j += HM_THREADS) {
      float2 r = Arow[cp[j]];
      for (int l = 0; l < rank; ++l) {
        const float2 p = cmulf(U[(size_t)l * m + i], Vt[(size_t)l * n + j]);
        r.x -= p.x;
        r.y -= p.y;
      }
      Vt[(size_t)rank * n + j] = r;
      argmax_merge(bv, bj, r.x * r.x + r.y * r.y, j);
    }
    int js;
    block_argmax(bv, bj, sv, si, bv, js);
    if (!(bv >= FLT_MIN)) {
      // the residual vanishes on this row (to below the normal range, where 1 / pivot would
      // overflow): the next row not yet used
      if (tid == 0) {
        int c = -1;
        for (int p = 0; p < m && c < 0; ++p)
          if (!row_used(used, nused, p)) c = p;
        s_next = c;
      }
      __syncthreads();
      i = s_next;
      __syncthreads();
      if (i < 0) {
        status = 0;  // every row reproduced
        break;
      }
      continue;
    }
    const float2 piv = Vt[(size_t)rank * n + js];
    __syncthreads();  // every thread holds the pivot before its entry is rescaled
    const float dd = piv.x * piv.x + piv.y * piv.y;
    const float2 ip = make_float2(piv.x / dd, -piv.y / dd);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};  // |u|^2, |v|^2
    for (int j = tid; j < n; j += HM_THREADS) {
      const float2 v = cmulf(Vt[(size_t)rank * n + j], ip);
      Vt[(size_t)rank * n + j] = v;
      acc[1] += (double)v.x * v.x + (double)v.y * v.y;
    }
    // residual column js into the next cross's U row, and the next pivot row
    float bu = -1.f;
    int bp = INT_MAX;
    for (int p = tid; p < m; p += HM_THREADS) {
      float2 u = A[(size_t)rp[p] * ld + cp[js]];
      for (int l = 0; l < rank; ++l) {
        const float2 q = cmulf(Vt[(size_t)l * n + js], U[(size_t)l * m + p]);
        u.x -= q.x;
        u.y -= q.y;
      }
      U[(size_t)rank * m + p] = u;
      acc[0] += (double)u.x * u.x + (double)u.y * u.y;
      if (!row_used(used, nused, p)) argmax_merge(bu, bp, u.x * u.x + u.y * u.y, p);
    }
    block_sum4(acc, sd);
    const double uu = acc[0], vv = acc[1];
    __syncthreads();  // the new cross is complete in global memory
    // ||S + u v^T||^2 = ||S||^2 + 2 Re sum_l (u_l^H u)(v_l^H v) + ||u||^2 ||v||^2
    double cross = 0.0;
    for (int l = 0; l < rank; ++l) {
      double c[4] = {0.0, 0.0, 0.0, 0.0};
      for (int p = tid; p < m; p += HM_THREADS) {
        const float2 a = U[(size_t)l * m + p], b = U[(size_t)rank * m + p];
        c[0] += (double)a.x * b.x + (double)a.y * b.y;  // conj(a) b
        c[1] += (double)a.x * b.y - (double)a.y * b.x;
      }
      for (int j = tid; j < n; j += HM_THREADS) {
        const float2 a = Vt[(size_t)l * n + j], b = Vt[(size_t)rank * n + j];
        c[2] += (double)a.x * b.x + (double)a.y * b.y;
        c[3] += (double)a.x * b.y - (double)a.y * b.x;
      }
      block_sum4(c, sd);
      cross += c[0] * c[2] - c[1] * c[3];
    }
    norm2 += 2.0 * cross + uu * vv;
    ++rank;
    if (sqrt(uu * vv) <= (double)eps * sqrt(fmax(norm2, 0.0))) {
      status = 0;
      break;
    }
    int np;
    block_argmax(bu, bp, sv, si, bu, np);
    if (bu < 0.f) {
      status = 0;  // every row used
      break;
    }
    i = np;
  }
  if (tid == 0) {
    rank_out[blockIdx.x] = rank;
    status_out[blockIdx.x] = status;
  }
}

// Packs the final blocks into one buffer: a dense block gathered from A (m x n row-major), a
// low-rank block copied from its slot (the first rank rows of U and of Vt).
__global__ void __launch_bounds__(HM_THREADS)
    hm_pack_kernel(const float2* __restrict__ A, long long ld, const int32_t* __restrict__ perm,
                   const HmBlockDev* __restrict__ blk, const long long* __restrict__ slot, int cap,
                   const float2* __restrict__ slots, float2* __restrict__ out) {
  RF_COUNT_LAUNCH();
  const HmBlockDev B = blk[blockIdx.x];
  const int m = B.r1 - B.r0, n = B.c1 - B.c0;
  float2* dst = out + B.off;
  if (B.rank < 0) {
    const long long total = (long long)m * n;
    for (long long e = threadIdx.x; e < total; e += HM_THREADS) {
      const int i = (int)(e / n), j = (int)(e % n);
      dst[e] = A[(size_t)perm[B.r0 + i] * ld + perm[B.c0 + j]];
    }
  } else {
    const float2* U = slots + slot[blockIdx.x];
    const float2* Vt = U + (size_t)cap * m;
    const long long nu = (long long)B.rank * m, nv = (long long)B.rank * n;
    for (long long e = threadIdx.x; e < nu; e += HM_THREADS) dst[e] = U[e];
    for (long long e = threadIdx.x; e < nv; e += HM_THREADS) dst[nu + e] = Vt[e];
  }
}

// xp (n x nrhs, cluster order) = x gathered through perm
__global__ void hm_gather_kernel(const double2* __restrict__ x, const int32_t* __restrict__ perm, int n, int nrhs,
                                 double2* __restrict__ xp) {
  RF_COUNT_LAUNCH();
  const long long total = (long long)n * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / n;
    const int p = (int)(e - c * n);
    xp[e] = x[c * n + perm[p]];
  }
}

// y (original order) = yp scattered through perm
__global__ void hm_scatter_kernel(const double2* __restrict__ yp, const int32_t* __restrict__ perm, int n, int nrhs,
                                  double2* __restrict__ y) {
  RF_COUNT_LAUNCH();
  const long long total = (long long)n * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / n;
    const int p = (int)(e - c * n);
    y[c * n + perm[p]] = yp[e];
  }
}

__device__ __forceinline__ void atomic_add_c(double2* p, double re, double im) {
  atomicAdd(&p->x, re);
  atomicAdd(&p->y, im);
}

__device__ __forceinline__ void warp_sum2(double& a, double& b) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(FULL, a, o);
    b += __shfl_down_sync(FULL, b, o);
  }
}

// yp += H xp for one block and one column (grid: blocks x columns), FP64 accumulation.  A block
// off the block diagonal adds its transpose too: y[c0..c1) += B^T x[r0..r1).
__global__ void __launch_bounds__(HM_THREADS)
    hm_apply_kernel(const HmBlockDev* __restrict__ blk, const float2* __restrict__ H, const double2* __restrict__ xp,
                    double2* __restrict__ yp, int n) {
  RF_COUNT_LAUNCH();
  __shared__ double2 t[HM_MAX_RANK];
  const HmBlockDev B = blk[blockIdx.x];
  const int m = B.r1 - B.r0, nn = B.c1 - B.c0, tid = threadIdx.x;
  const double2* xc = xp + (size_t)blockIdx.y * n;
  double2* yc = yp + (size_t)blockIdx.y * n;
  const bool mirror = B.r0 != B.c0;
  const float2* M = H + B.off;
  if (B.rank < 0) {
    for (int i = tid; i < m; i += HM_THREADS) {
      double a = 0.0, b = 0.0;
      const float2* row = M + (size_t)i * nn;
      for (int j = 0; j < nn; ++j) {
        const float2 d = row[j];
        const double2 v = xc[B.c0 + j];
        a += (double)d.x * v.x - (double)d.y * v.y;
        b += (double)d.x * v.y + (double)d.y * v.x;
      }
      atomic_add_c(yc + B.r0 + i, a, b);
    }
    if (mirror) {
      for (int j = tid; j < nn; j += HM_THREADS) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < m; ++i) {
          const float2 d = M[(size_t)i * nn + j];
          const double2 v = xc[B.r0 + i];
          a += (double)d.x * v.x - (double)d.y * v.y;
          b += (double)d.x * v.y + (double)d.y * v.x;
        }
        atomic_add_c(yc + B.c0 + j, a, b);
      }
    }
    return;
  }
  const int r = B.rank, w = tid >> 5, lane = tid & 31;
  const float2* U = M;
  const float2* Vt = M + (size_t)r * m;
  // t = Vt x[c0..c1), one warp per cross
  for (int l = w; l < r; l += HM_THREADS / 32) {
    double a = 0.0, b = 0.0;
    for (int j = lane; j < nn; j += 32) {
      const float2 v = Vt[(size_t)l * nn + j];
      const double2 x = xc[B.c0 + j];
      a += (double)v.x * x.x - (double)v.y * x.y;
      b += (double)v.x * x.y + (double)v.y * x.x;
    }
    warp_sum2(a, b);
    if (lane == 0) t[l] = make_double2(a, b);
  }
  __syncthreads();
  for (int i = tid; i < m; i += HM_THREADS) {
    double a = 0.0, b = 0.0;
    for (int l = 0; l < r; ++l) {
      const float2 u = U[(size_t)l * m + i];
      a += (double)u.x * t[l].x - (double)u.y * t[l].y;
      b += (double)u.x * t[l].y + (double)u.y * t[l].x;
    }
    atomic_add_c(yc + B.r0 + i, a, b);
  }
  if (mirror) {
    __syncthreads();  // t is rewritten
    // t = U x[r0..r1) (the transpose: (U Vt)^T x = Vt^T (U^T x))
    for (int l = w; l < r; l += HM_THREADS / 32) {
      double a = 0.0, b = 0.0;
      for (int i = lane; i < m; i += 32) {
        const float2 u = U[(size_t)l * m + i];
        const double2 x = xc[B.r0 + i];
        a += (double)u.x * x.x - (double)u.y * x.y;
        b += (double)u.x * x.y + (double)u.y * x.x;
      }
      warp_sum2(a, b);
      if (lane == 0) t[l] = make_double2(a, b);
    }
    __syncthreads();
    for (int j = tid; j < nn; j += HM_THREADS) {
      double a = 0.0, b = 0.0;
      for (int l = 0; l < r; ++l) {
        const float2 v = Vt[(size_t)l * nn + j];
        a += (double)v.x * t[l].x - (double)v.y * t[l].y;
        b += (double)v.x * t[l].y + (double)v.y * t[l].x;
      }
      atomic_add_c(yc + B.c0 + j, a, b);
    }
  }
}

}  // namespace

// one compressed matrix (T_A or V)
struct HmPart {
  int n = 0;
  int nblocks = 0;
  int32_t* perm = nullptr;       // cluster order -> original index (device)
  HmBlockDev* blocks = nullptr;  // (device)
  float2* data = nullptr;        // dense blocks and crosses (device)
  long long elems = 0;
  int64_t n_lowrank = 0, n_dense = 0, n_capped = 0, n_small = 0;
  int max_rank = 0;
  uint64_t bytes = 0;
};

#define HM_CUDA(call)                                                                                \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return set_error(RFCMP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Frees the temporaries of one build on every path out of it.
struct HmTemps {
  std::vector<void*> p;
  ~HmTemps() {
    for (void* q : p) dev_free(q);
  }
  template <class T>
  cudaError_t alloc(T** q, size_t bytes) {
    cudaError_t e = dev_malloc(q, bytes);
    if (e == cudaSuccess) p.push_back(*q);
    return e;
  }
};

// Compresses the dense n x n matrix A (row stride ld, both triangles stored) whose items have the
// given centres and support boxes.  owned receives the part's device buffers; budget_left bounds
// the bytes it may hold at the peak of the build.
int build_part(const float2* A, int ld, int n, const std::vector<double>& cen, const std::vector<double>& lo,
               const std::vector<double>& hi, const rfcmp_hm_opts& o, uint64_t budget_left, HmPart& out,
               std::vector<void*>& owned) {
  out.n = n;
  std::vector<int32_t> perm;
  std::vector<HmBlockHost> blocks;
  partition(cen.data(), lo.data(), hi.data(), n, o.leaf, o.eta, perm, blocks);
  const int cap = o.max_rank;
  std::vector<HmBlockDev> cand;
  std::vector<long long> slot;
  long long slot_elems = 0, dense_elems = 0;
  for (const HmBlockHost& b : blocks) {
    const long long m = b.r1 - b.r0, nn = b.c1 - b.c0;
    if (b.admissible) {
      cand.push_back({b.r0, b.r1, b.c0, b.c1, 0, 0, 0});
      slot.push_back(slot_elems);
      slot_elems += (long long)cap * (m + nn);
    } else {
      dense_elems += m * nn;
    }
  }
  // the peak holds the slots and, at worst, every block dense
  long long worst = dense_elems;
  for (const HmBlockDev& c : cand) worst += (long long)(c.r1 - c.r0) * (c.c1 - c.c0);
  const uint64_t peak = 8ull * (uint64_t)(slot_elems + worst) + 64ull * blocks.size() + 4ull * n;
  if (budget_left != UINT64_MAX && peak > budget_left)
    return set_error(RFCMP_ERR_OUT_OF_BUDGET, "compression needs up to " + std::to_string(peak) + " bytes, budget has " +
                                                  std::to_string(budget_left));
  HmTemps tmp;
  HM_CUDA(dev_malloc(&out.perm, std::max<size_t>(4 * (size_t)n, 4)));
  owned.push_back(out.perm);
  if (n > 0) HM_CUDA(cudaMemcpy(out.perm, perm.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
  std::vector<int32_t> rank(cand.size(), 0), status(cand.size(), 1);
  float2* slots = nullptr;
  long long* slot_d = nullptr;
  if (!cand.empty()) {
    HmBlockDev* cand_d = nullptr;
    int32_t *rank_d = nullptr, *status_d = nullptr;
    HM_CUDA(tmp.alloc(&cand_d, cand.size() * sizeof(HmBlockDev)));
    HM_CUDA(tmp.alloc(&slot_d, slot.size() * sizeof(long long)));
    HM_CUDA(tmp.alloc(&slots, 8 * (size_t)slot_elems));
    HM_CUDA(tmp.alloc(&rank_d, 4 * cand.size()));
    HM_CUDA(tmp.alloc(&status_d, 4 * cand.size()));
    HM_CUDA(cudaMemcpy(cand_d, cand.data(), cand.size() * sizeof(HmBlockDev), cudaMemcpyHostToDevice));
    HM_CUDA(cudaMemcpy(slot_d, slot.data(), slot.size() * sizeof(long long), cudaMemcpyHostToDevice));
    const int iter_cap = std::min(cap + 16, HM_MAX_ITER);
    {
      ProfScope prof("hm_aca", 8.0 * (double)slot_elems, 0.0, 0);
      hm_aca_kernel<<<(unsigned)cand.size(), HM_THREADS>>>(A, ld, out.perm, cand_d, slot_d, cap, iter_cap,
                                                          (float)o.eps, slots, rank_d, status_d);
    }
    HM_CUDA(cudaGetLastError());
    HM_CUDA(cudaMemcpy(rank.data(), rank_d, 4 * cand.size(), cudaMemcpyDeviceToHost));
    HM_CUDA(cudaMemcpy(status.data(), status_d, 4 * cand.size(), cudaMemcpyDeviceToHost));
  }
  // final blocks: the admissible ones whose crosses met the stopping rule in low rank, the rest dense
  std::vector<HmBlockDev> fin;
  std::vector<long long> fin_slot;
  long long off = 0;
  size_t ci = 0;
  for (const HmBlockHost& b : blocks) {
    const long long m = b.r1 - b.r0, nn = b.c1 - b.c0;
    HmBlockDev d{b.r0, b.r1, b.c0, b.c1, -1, 0, off};
    long long s = 0;
    if (b.admissible) {
      const size_t c = ci++;
      if (status[c] != 0 || rank[c] < 0 || rank[c] > cap) {
        ++out.n_capped;
      } else if ((long long)rank[c] * (m + nn) >= m * nn) {
        ++out.n_small;  // the crosses would take at least the block's own entries
      } else {
        d.rank = rank[c];
        s = slot[c];
        ++out.n_lowrank;
        out.max_rank = std::max(out.max_rank, rank[c]);
      }
    }
    if (d.rank < 0) ++out.n_dense;
    off += d.rank < 0 ? m * nn : (long long)d.rank * (m + nn);
    fin.push_back(d);
    fin_slot.push_back(s);
  }
  out.elems = off;
  out.nblocks = (int)fin.size();
  HM_CUDA(dev_malloc(&out.data, std::max<size_t>(8 * (size_t)off, 8)));
  owned.push_back(out.data);
  HM_CUDA(dev_malloc(&out.blocks, std::max<size_t>(fin.size() * sizeof(HmBlockDev), 8)));
  owned.push_back(out.blocks);
  if (!fin.empty()) {
    long long* fslot_d = nullptr;
    HM_CUDA(tmp.alloc(&fslot_d, fin_slot.size() * sizeof(long long)));
    HM_CUDA(cudaMemcpy(out.blocks, fin.data(), fin.size() * sizeof(HmBlockDev), cudaMemcpyHostToDevice));
    HM_CUDA(cudaMemcpy(fslot_d, fin_slot.data(), fin_slot.size() * sizeof(long long), cudaMemcpyHostToDevice));
    hm_pack_kernel<<<(unsigned)fin.size(), HM_THREADS>>>(A, ld, out.perm, out.blocks, fslot_d, cap, slots, out.data);
    HM_CUDA(cudaGetLastError());
  }
  HM_CUDA(cudaStreamSynchronize(0));
  out.bytes = 8ull * (uint64_t)off + sizeof(HmBlockDev) * fin.size() + 4ull * n;
  return RFCMP_OK;
}

}  // namespace rfcmp

// ============================================================================ C ABI
struct rfcmp_hm {
  int device = 0;
  rfcmp::HmPart part[2];  // RFCMP_HM_T_A, RFCMP_HM_V
  std::vector<void*> owned;
  std::atomic<uint64_t>* ctx_bytes = nullptr;
  std::atomic<int>* ctx_live = nullptr;
  uint64_t bytes = 0;
  rfcmp_hm_opts opts{};
  std::mutex mu;                          // guards nb_streams
  std::vector<cudaStream_t> nb_streams;   // non-blocking streams products were queued on
  ~rfcmp_hm() {
    for (void* p : owned) rfcmp::dev_free(p);
  }
};

using namespace rfcmp;

namespace {

// supports of the cells (centroid; box of the three vertices) and of the RWG functions (edge
// midpoint; box of the vertices of both cells)
void supports(const Topology& top, const double* verts, std::vector<double>& ccen, std::vector<double>& clo,
              std::vector<double>& chi, std::vector<double>& ecen, std::vector<double>& elo, std::vector<double>& ehi) {
  const int64_t nc = top.nc, ne = top.ne;
  ccen.assign(3 * nc, 0.0);
  clo.assign(3 * nc, 0.0);
  chi.assign(3 * nc, 0.0);
  for (int64_t c = 0; c < nc; ++c) {
    const double* p0 = verts + 3 * (int64_t)top.tris[3 * c];
    const double* p1 = verts + 3 * (int64_t)top.tris[3 * c + 1];
    const double* p2 = verts + 3 * (int64_t)top.tris[3 * c + 2];
    for (int d = 0; d < 3; ++d) {
      ccen[3 * c + d] = (p0[d] + p1[d] + p2[d]) / 3.0;
      clo[3 * c + d] = std::min(std::min(p0[d], p1[d]), p2[d]);
      chi[3 * c + d] = std::max(std::max(p0[d], p1[d]), p2[d]);
    }
  }
  ecen.assign(3 * ne, 0.0);
  elo.assign(3 * ne, 0.0);
  ehi.assign(3 * ne, 0.0);
  for (int64_t e = 0; e < ne; ++e) {
    const double* a = verts + 3 * (int64_t)top.edge_verts[2 * e];
    const double* b = verts + 3 * (int64_t)top.edge_verts[2 * e + 1];
    const int64_t cp = top.edge_cells[2 * e], cm = top.edge_cells[2 * e + 1];
    for (int d = 0; d < 3; ++d) {
      ecen[3 * e + d] = 0.5 * (a[d] + b[d]);
      elo[3 * e + d] = std::min(clo[3 * cp + d], clo[3 * cm + d]);
      ehi[3 * e + d] = std::max(chi[3 * cp + d], chi[3 * cm + d]);
    }
  }
}

int check_opts(const rfcmp_hm_opts& o) {
  for (int i = 0; i < 6; ++i)
    if (o.reserved[i] != 0) return set_error(RFCMP_ERR_INVALID_ARG, "opts.reserved must be zero");
  if (!(o.eps > 0.0 && o.eps < 1.0)) return set_error(RFCMP_ERR_INVALID_ARG, "eps must be in (0, 1)");
  if (!(o.eta > 0.0) || !std::isfinite(o.eta)) return set_error(RFCMP_ERR_INVALID_ARG, "eta must be positive");
  if (o.leaf < 8 || o.leaf > 1024) return set_error(RFCMP_ERR_INVALID_ARG, "leaf must be in [8, 1024]");
  if (o.max_rank < 1 || o.max_rank > HM_MAX_RANK) return set_error(RFCMP_ERR_INVALID_ARG, "max_rank must be in [1, 256]");
  return RFCMP_OK;
}

}  // namespace

extern "C" {

void rfcmp_hm_opts_default(rfcmp_hm_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eps = 1e-4;
  o->eta = 1.0;
  o->leaf = 32;
  o->max_rank = 64;
}

int rfcmp_hm_partition(const double* centres, const double* sup_lo, const double* sup_hi, int64_t n, int32_t leaf,
                       double eta, int32_t* perm, int32_t* blocks, int64_t capacity, int64_t* n_blocks) {
  if (!n_blocks || !perm || (n > 0 && (!centres || !sup_lo || !sup_hi)))
    return set_error(RFCMP_ERR_INVALID_ARG, "NULL argument");
  int rc = check_partition_args(n, leaf, eta);
  if (rc != RFCMP_OK) return rc;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(centres[i]) || !std::isfinite(sup_lo[i]) || !std::isfinite(sup_hi[i]))
      return set_error(RFCMP_ERR_INVALID_ARG, "non-finite coordinate");
  std::vector<int32_t> p;
  std::vector<HmBlockHost> b;
  partition(centres, sup_lo, sup_hi, (int)n, leaf, eta, p, b);
  *n_blocks = (int64_t)b.size();
  if (n > 0) std::memcpy(perm, p.data(), 4 * (size_t)n);
  if (!blocks) return RFCMP_OK;
  if (capacity < (int64_t)b.size()) return set_error(RFCMP_ERR_INVALID_ARG, "blocks capacity too small");
  for (size_t i = 0; i < b.size(); ++i) {
    blocks[5 * i] = b[i].r0;
    blocks[5 * i + 1] = b[i].r1;
    blocks[5 * i + 2] = b[i].c0;
    blocks[5 * i + 3] = b[i].c1;
    blocks[5 * i + 4] = b[i].admissible;
  }
  return RFCMP_OK;
}

int rfcmp_hm_create(rfcmp_op* op, const rfcmp_hm_opts* opts_in, rfcmp_hm** out) {
  if (!op || !out) return set_error(RFCMP_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  rfcmp_hm_opts o;
  rfcmp_hm_opts_default(&o);
  if (opts_in) o = *opts_in;
  int rc = check_opts(o);
  if (rc != RFCMP_OK) return rc;
  OpDenseView v;
  if (!op_dense_view(op, &v)) return set_error(RFCMP_ERR_INVALID_ARG, "op has no resident T_A and V");
  HM_CUDA(cudaSetDevice(v.device));
  auto hm = std::make_unique<rfcmp_hm>();
  hm->device = v.device;
  hm->opts = o;
  std::vector<double> ccen, clo, chi, ecen, elo, ehi;
  supports(*v.top, v.verts, ccen, clo, chi, ecen, elo, ehi);
  const float2* mats[2] = {v.TA, v.V};
  const int lds[2] = {v.ldN, v.ldC}, ns[2] = {v.n, v.nc};
  for (int w = 0; w < 2; ++w) {
    uint64_t left = UINT64_MAX;
    if (v.budget) {
      const uint64_t used = v.ctx_bytes->load() + hm->bytes;
      left = v.budget > used ? v.budget - used : 0;
    }
    rc = build_part(mats[w], lds[w], ns[w], w == 0 ? ecen : ccen, w == 0 ? elo : clo, w == 0 ? ehi : chi, o, left,
                    hm->part[w], hm->owned);
    if (rc != RFCMP_OK) return rc;
    hm->bytes += hm->part[w].bytes;
  }
  hm->ctx_bytes = v.ctx_bytes;
  hm->ctx_live = v.ctx_live;
  *hm->ctx_bytes += hm->bytes;
  ++*hm->ctx_live;
  *out = hm.release();
  return RFCMP_OK;
}

int rfcmp_hm_apply(rfcmp_hm* hm, int which, const rfcmp_c128* x, rfcmp_c128* y, int64_t nrhs, void* stream) {
  if (!hm || !x || !y || nrhs < 1 || nrhs > 65535 || (which != RFCMP_HM_T_A && which != RFCMP_HM_V))
    return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  if ((const void*)x == (const void*)y) return set_error(RFCMP_ERR_INVALID_ARG, "x and y must not alias");
  const HmPart& P = hm->part[which];
  HM_CUDA(cudaSetDevice(hm->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (st) {
    unsigned int flags = 0;
    HM_CUDA(cudaStreamGetFlags(st, &flags));
    if (flags & cudaStreamNonBlocking) {
      std::lock_guard<std::mutex> lk(hm->mu);
      if (std::find(hm->nb_streams.begin(), hm->nb_streams.end(), st) == hm->nb_streams.end())
        hm->nb_streams.push_back(st);
    }
  }
  const long long total = (long long)P.n * nrhs;
  if (total == 0) return RFCMP_OK;
  double2 *xp = nullptr, *yp = nullptr;
  HM_CUDA(cudaMallocAsync(&xp, 16 * (size_t)total, st));
  cudaError_t e = cudaMallocAsync(&yp, 16 * (size_t)total, st);
  if (e == cudaSuccess) {
    const int grid = (int)std::min<long long>((total + HM_THREADS - 1) / HM_THREADS, 152 * 8);
    hm_gather_kernel<<<grid, HM_THREADS, 0, st>>>(reinterpret_cast<const double2*>(x), P.perm, P.n, (int)nrhs, xp);
    e = cudaMemsetAsync(yp, 0, 16 * (size_t)total, st);
    if (e == cudaSuccess && P.nblocks > 0) {
      ProfScope prof("hm_apply", 8.0 * (double)P.elems + 32.0 * (double)total, 0.0, st);
      hm_apply_kernel<<<dim3((unsigned)P.nblocks, (unsigned)nrhs), HM_THREADS, 0, st>>>(P.blocks, P.data, xp, yp, P.n);
    }
    if (e == cudaSuccess)
      hm_scatter_kernel<<<grid, HM_THREADS, 0, st>>>(yp, P.perm, P.n, (int)nrhs, reinterpret_cast<double2*>(y));
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFreeAsync(yp, st);
  }
  cudaFreeAsync(xp, st);
  if (e != cudaSuccess) return set_error(RFCMP_ERR_CUDA, std::string("rfcmp_hm_apply: ") + cudaGetErrorString(e));
  return RFCMP_OK;
}

int rfcmp_hm_info_get(const rfcmp_hm* hm, rfcmp_hm_info* out) {
  if (!hm || !out) return set_error(RFCMP_ERR_INVALID_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  for (int w = 0; w < 2; ++w) {
    const HmPart& P = hm->part[w];
    out->n[w] = P.n;
    out->lowrank_blocks[w] = P.n_lowrank;
    out->dense_blocks[w] = P.n_dense;
    out->capped_blocks[w] = P.n_capped;
    out->small_blocks[w] = P.n_small;
    out->bytes[w] = P.bytes;
    out->max_rank[w] = P.max_rank;
  }
  return RFCMP_OK;
}

int rfcmp_hm_destroy(rfcmp_hm* hm) {
  if (!hm) return RFCMP_OK;
  cudaSetDevice(hm->device);
  // frees are queued on the legacy stream: make it wait for the streams products ran on
  if (!hm->nb_streams.empty()) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
      for (cudaStream_t s : hm->nb_streams)
        if (cudaEventRecord(ev, s) == cudaSuccess) cudaStreamWaitEvent(0, ev, 0);
      cudaEventDestroy(ev);
    } else {
      for (cudaStream_t s : hm->nb_streams) cudaStreamSynchronize(s);
    }
  }
  if (hm->ctx_bytes) *hm->ctx_bytes -= hm->bytes;
  if (hm->ctx_live) --*hm->ctx_live;
  delete hm;
  return RFCMP_OK;
}

}  // extern "C"
