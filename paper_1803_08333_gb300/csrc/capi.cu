// C ABI of librfcmp (include/rfcmp.h): context, operator lifecycle, the
// RF-CMP application (Sec. 3 Eq. NewFormulation, numerical variant of Sec. 4),
// power-iteration scaling (Sec. 4) and the CG solve with float-float
// residual refinement.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "rfcmp_internal.h"

using namespace rfcmp;

// ---------------------------------------------------------------- errors
namespace {
thread_local std::string g_last_error;
}  // namespace

namespace rfcmp {
int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
}  // namespace rfcmp

namespace {

#define RF_CUDA(call)                                                                                  \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess)                                                                             \
      return set_error(RFCMP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

#define RF_TRY(call)            \
  do {                          \
    int rc_ = (call);           \
    if (rc_ != RFCMP_OK) return rc_; \
  } while (0)

// Radon's 7-point degree-5 rule in barycentric coordinates (weights sum to 1)
struct Rule7 {
  double bary[7][3];
  double w[7];
  Rule7() {
    const double s15 = std::sqrt(15.0);
    const double a = (6.0 - s15) / 21.0, b = (6.0 + s15) / 21.0;
    const double wa = (155.0 - s15) / 1200.0, wb = (155.0 + s15) / 1200.0;
    const double pts[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {a, a, 1 - 2 * a}, {a, 1 - 2 * a, a}, {1 - 2 * a, a, a},
                              {b, b, 1 - 2 * b},          {b, 1 - 2 * b, b}, {1 - 2 * b, b, b}};
    const double ws[7] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
    for (int q = 0; q < 7; ++q) {
      for (int i = 0; i < 3; ++i) bary[q][i] = pts[q][i];
      w[q] = ws[q];
    }
  }
};

template <class T>
int dalloc(T** p, size_t count, std::vector<void*>& owned) {
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = dev_malloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return set_error(RFCMP_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  owned.push_back(q);
  *p = static_cast<T*>(q);
  return RFCMP_OK;
}

template <class T>
int upload(T** p, const std::vector<T>& h, std::vector<void*>& owned) {
  RF_TRY(dalloc(p, h.size(), owned));
  if (!h.empty()) RF_CUDA(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return RFCMP_OK;
}

double2 c2(double re, double im) { return make_double2(re, im); }

}  // namespace

// ---------------------------------------------------------------- profiling
namespace {
struct ProfFamily {
  std::string name;
  int64_t launches = 0;
  double bytes = 0.0, flops = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  double ms = 0.0;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfFamily> g_prof;
std::vector<cudaEvent_t> g_event_pool;
uint64_t g_prof_generation = 0;  // bumped when rfcmp_profile_enable clears the families

// Launches captured into a CUDA graph (the solve loop) cannot carry CUDA events: a conditional
// body holds kernel, memset and memcpy nodes only, and one capture runs many times.  A captured
// scope is bracketed by two one-thread kernels instead, which read the device's global
// nanosecond timer before and after the launch and add the difference, one launch and the
// launch's algorithmic bytes and FLOPs to the family's device accumulators.
constexpr int PROF_DEV_FAMILIES = 64;
constexpr int PROF_DEV_SCOPES = 4096;
struct DevProfFamily {
  unsigned long long ns, launches;
  double bytes, flops;
};
__device__ DevProfFamily g_prof_dev[PROF_DEV_FAMILIES];
__device__ unsigned long long g_prof_t0[PROF_DEV_SCOPES];
int g_next_scope = 0;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__global__ void prof_begin_kernel(int scope) { g_prof_t0[scope] = global_ns(); }
__global__ void prof_end_kernel(int scope, int fam, double bytes, double flops) {
  const unsigned long long t = global_ns();
  DevProfFamily& f = g_prof_dev[fam];
  atomicAdd(&f.ns, t - g_prof_t0[scope]);
  atomicAdd(&f.launches, 1ULL);
  atomicAdd(&f.bytes, bytes);
  atomicAdd(&f.flops, flops);
}

void prof_dev_clear() {
  static const DevProfFamily zero[PROF_DEV_FAMILIES] = {};
  if (cudaMemcpyToSymbol(g_prof_dev, zero, sizeof(zero)) != cudaSuccess) (void)cudaGetLastError();
}

cudaEvent_t pool_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Pending pairs hold only scopes whose end event has been recorded (the destructor pushes them),
// so resolving never waits on an event that is not on a stream.  A failed elapsed-time query
// (an event of a stream that was destroyed, say) drops that pair and clears the runtime's
// last error, so it cannot surface later as the failure of an unrelated launch check.
void prof_resolve_family_locked(ProfFamily& f) {
  for (auto& pr : f.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(pr.second) == cudaSuccess && cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess)
      f.ms += ms;
    else
      (void)cudaGetLastError();
    g_event_pool.push_back(pr.first);
    g_event_pool.push_back(pr.second);
  }
  f.pending.clear();
}

void prof_resolve_locked() {
  for (auto& f : g_prof) prof_resolve_family_locked(f);
}

constexpr size_t PROF_MAX_PENDING = 4096;
}  // namespace

namespace {
std::atomic<int> g_solve_graphs{-1};  // -1: not yet read from the environment

bool solve_graphs_enabled() {
  int v = g_solve_graphs.load();
  if (v < 0) {
    const char* e = std::getenv("RFCMP_SOLVE_GRAPHS");
    v = (e && e[0] == '0') ? 0 : 1;
    g_solve_graphs.store(v);
  }
  return v != 0;
}

}  // namespace

uint64_t prof_capture_key() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_prof_on.load() ? (g_prof_generation << 1) | 1u : 0u;
}

namespace rfcmp {
ProfScope::ProfScope(const char* family, double bytes, double flops, cudaStream_t s) : s_(s) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  int idx = -1;
  for (size_t i = 0; i < g_prof.size(); ++i)
    if (g_prof[i].name == family) idx = (int)i;
  if (idx < 0) {
    g_prof.push_back(ProfFamily());
    g_prof.back().name = family;
    idx = (int)g_prof.size() - 1;
  }
  if (cap == cudaStreamCaptureStatusActive) {
    if (idx >= PROF_DEV_FAMILIES) return;
    scope_ = g_next_scope;
    g_next_scope = (g_next_scope + 1) % PROF_DEV_SCOPES;
    prof_begin_kernel<<<1, 1, 0, s>>>(scope_);
    if (cudaGetLastError() != cudaSuccess) return;
    captured_ = true;
    bytes_ = bytes;
    flops_ = flops;
    slot_ = idx;
    gen_ = g_prof_generation;
    return;
  }
  ProfFamily& f = g_prof[idx];
  f.launches++;
  f.bytes += bytes;
  f.flops += flops;
  a_ = pool_event();
  b_ = pool_event();
  if (!a_ || !b_ || cudaEventRecord(a_, s) != cudaSuccess) {
    (void)cudaGetLastError();
    if (a_) g_event_pool.push_back(a_);
    if (b_) g_event_pool.push_back(b_);
    a_ = b_ = nullptr;
    return;
  }
  slot_ = idx;
  gen_ = g_prof_generation;
}
ProfScope::~ProfScope() {
  if (slot_ < 0) return;
  if (captured_) {
    prof_end_kernel<<<1, 1, 0, s_>>>(scope_, slot_, bytes_, flops_);
    (void)cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  // rfcmp_profile_enable may have cleared the families since the constructor ran
  if (gen_ != g_prof_generation || slot_ >= (int)g_prof.size() || cudaEventRecord(b_, s_) != cudaSuccess) {
    (void)cudaGetLastError();
    g_event_pool.push_back(a_);
    g_event_pool.push_back(b_);
    return;
  }
  ProfFamily& f = g_prof[slot_];
  f.pending.push_back({a_, b_});
  if (f.pending.size() >= PROF_MAX_PENDING) prof_resolve_family_locked(f);
}
}  // namespace rfcmp

// ---------------------------------------------------------------- factor cache
// (Sigma^T Sigma)^+ of meshes with at least this many cells is refined by Newton-Schulz steps on
// the tensor cores from a multigrid-PCG start accurate to NS_START_TOL.
constexpr int NS_MIN_CELLS = 256;
// Products with at least this many right-hand sides in the FP32 inner iterations run on the tensor
// cores (split-BF16 GEMM) instead of the HBM-bound GEMV: one pass over the BF16 planes (as many
// bytes as the complex64 matrix) serves every column, so from about 4 columns on it beats the
// GEMV's pass per 4 columns (measured on GB300 from 2k to 31k unknowns).
constexpr int MRHS_MIN = 4;
// Float-float accurate products (right-hand side, refinement residuals, accurate applications)
// with at least this many columns run as exact-digit tensor-core products instead of the
// float-float GEMV, which spends some 40 FP32 instructions per complex multiply-add (measured on
// GB300: the exact-digit product wins from 4 columns at 2k unknowns, from 2 at 17k and above).
constexpr int EXACT_MIN = 4;
constexpr double NS_START_TOL = 1e-2;
constexpr int NS_MAX_STEPS = 24;
// Newton-Schulz stops at max |I - M X| <= max(factor_tol, NS_TARGET): the FP64 residual of tens
// of thousands of cells floors near 1e-13 on closed surfaces (measured 1.2e-13 at 27380 cells)
// and near 1e-12 on an open plate of 20000 cells.  A refinement that stalls within NS_ACCEPT of
// the target has reached that floor and is kept.
constexpr double NS_TARGET = 1e-12;
constexpr double NS_ACCEPT = 10.0;

struct DenseFactor {
  int n = 0;
  int ns_steps = 0;
  double ns_residual = 0.0;
  RealPlanes planes;  // BF16 hi/lo of the FP32 hi plane, built on the first multi-RHS product
  ExactOperand digits;  // exact-digit planes of hi + lo, built on the first accurate multi-RHS product
  std::mutex planes_mu;
  float* hi = nullptr;
  float* lo = nullptr;
  size_t bytes = 0;
  int iterations = 0;
  double ms = 0.0;
  ~DenseFactor() {
    if (hi) dev_free(hi);
    if (lo) dev_free(lo);
    if (planes.h) dev_free(planes.h);
    if (planes.l) dev_free(planes.l);
    if (digits.d) dev_free(digits.d);
    if (digits.e) dev_free(digits.e);
  }
};

// Topology and device geometry of one mesh, shared by every operator on it (a frequency sweep
// or several requests on one mesh build them once).
struct MeshEntry {
  Topology top;
  std::vector<double> verts;
  DeviceGeometry g;
  std::vector<void*> owned;
  ~MeshEntry() {
    for (void* p : owned) dev_free(p);
  }
};

struct rfcmp_ctx {
  int device = 0;
  uint64_t budget = 0;
  std::atomic<uint64_t> bytes{0};
  std::mutex mu;
  std::map<uint64_t, std::shared_ptr<DenseFactor>> lplus_cache;  // key: connectivity hash
  std::map<uint64_t, std::shared_ptr<DenseFactor>> gll_cache;    // key: connectivity + coordinates hash
  std::map<uint64_t, std::shared_ptr<DenseFactor>> gtp_cache;    // key: connectivity hash (G_l~p^{-1})
  std::map<uint64_t, std::shared_ptr<MeshEntry>> mesh_cache;      // key: connectivity + coordinates
  std::mutex build_mu;  // one factor build at a time, so concurrent ops on one mesh share it
  std::atomic<int> live_ops{0};
  rfcmp_plan plan{};    // plan of operators created from now on
};

struct Workspace {
  int cols = 0;
  std::vector<void*> owned;
  // edge space (N)
  double2 *v = nullptr, *u = nullptr, *y = nullptr, *up = nullptr, *tmpN = nullptr;
  // cell space (N_C)
  double2 *s = nullptr, *z = nullptr, *w = nullptr, *zu = nullptr, *q0 = nullptr, *q = nullptr, *Lq = nullptr,
          *vp = nullptr, *g1 = nullptr, *g2 = nullptr;
  // vertex space (N_V)
  double2 *t = nullptr, *tg = nullptr;
  double* mean = nullptr;  // 4 x cols
  GemvScratch gs;
  MrhsScratch ms;
  ~Workspace() {
    for (void* p : owned) dev_free(p);
  }
};

struct SolveBuffers {
  int cols = 0;
  std::vector<void*> owned;
  double2 *b = nullptr, *i = nullptr, *r = nullptr, *d = nullptr, *rin = nullptr, *p = nullptr, *Ap = nullptr,
          *tmp = nullptr, *eh = nullptr, *jh = nullptr;
  double2* dots = nullptr;  // cols
  double *rho = nullptr, *alpha = nullptr, *beta = nullptr;
  int* active = nullptr;
  // device-resident CG state (k_krylov.cu)
  KrylovCtl* ctl = nullptr;
  double *bb = nullptr, *rr = nullptr, *r0 = nullptr, *res = nullptr;
  int *conv = nullptr, *iters = nullptr, *sweeps = nullptr;
  double2* part = nullptr;
  unsigned int* ticket = nullptr;
  int* member = nullptr;  // batch sessions only: 1 for the columns of running requests
  ~SolveBuffers() {
    for (void* p : owned) dev_free(p);
  }
};

// The solve loop of one op as an executable CUDA graph (refinement sweeps and CG iterations as
// nested WHILE nodes), with what it was captured for: a different shape, buffer set, plan or
// profiling state means a new capture.
struct SolveGraph {
  cudaGraphExec_t exec = nullptr;
  int nr = 0, mode = 0, max_sweeps = 0;
  const void* ws = nullptr;
  const void* sb = nullptr;
  int ws_cols = 0, sb_cols = 0;
  const void* lazy[10] = {};
  rfcmp_plan plan{};
  uint64_t prof_key = 0;
  ~SolveGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

struct rfcmp_op {
  rfcmp_ctx* ctx = nullptr;
  Topology top;
  std::vector<double> verts;
  DeviceGeometry g;
  std::vector<void*> owned;  // geometry + matrices
  float2* TA = nullptr;
  float2* V = nullptr;
  int ldN = 0, ldC = 0;
  std::shared_ptr<DenseFactor> lplus, gll;
  std::shared_ptr<DenseFactor> gtp;  // G_l~p^{-1} (outer = RFCMP_OUTER_GSIGMA only)
  int outer = RFCMP_OUTER_SIGMA;
  std::shared_ptr<MeshEntry> mesh;  // owns the device geometry in g
  double k = 0.0, alpha = 1.0, beta = 1.0, gamma = 1.0;
  uint64_t bytes = 0;
  rfcmp_op_info info{};
  std::unique_ptr<Workspace> ws;
  std::unique_ptr<SolveBuffers> sb;
  double2* power_vecs = nullptr;  // N x 3: Ritz vectors of the X, Z and Y norm iterations
  double2* lanczos = nullptr;     // Lanczos basis of the norm iterations (lanczos_slots x N x 2)
  int lanczos_slots = 0;
  CplxPlanes ta_planes, v_planes;  // BF16 planes of T_A and V, built on the first multi-RHS product
  ExactOperand ta_digits, v_digits;  // exact-digit planes of T_A and V, built on the first accurate one
  std::vector<void*> lazy;           // the planes and digits above, released by rfcmp_op_trim
  uint64_t lazy_bytes = 0;
  rfcmp_plan plan{};               // launch shapes (zero fields: built-in choices)
  std::vector<cudaStream_t> nb_streams;  // non-blocking streams this op's work was queued on
  cudaEvent_t order_ev = nullptr;        // orders streams against the legacy stream (no timing)
  std::unique_ptr<SolveGraph> solve_graph;  // the captured solve loop (rebuilt when stale)
  cudaStream_t capture[3] = {};    // streams the solve loop is captured on (never run work)
  bool graphs_failed = false;      // a capture failed once: this op solves eagerly
  ~rfcmp_op() {
    if (order_ev) cudaEventDestroy(order_ev);
    solve_graph.reset();
    for (cudaStream_t c : capture)
      if (c) cudaStreamDestroy(c);
    for (void* p : owned) dev_free(p);
    for (void* p : lazy) dev_free(p);
    if (lanczos) dev_free(lanczos);
  }
};

namespace {

uint64_t mix(uint64_t h, uint64_t v) {
  uint64_t z = h ^ (v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2));
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// columns from which inner-iteration products take the tensor cores
int plan_mrhs(const rfcmp_op* op) { return op->plan.mrhs_min > 0 ? op->plan.mrhs_min : MRHS_MIN; }
// columns from which float-float accurate products take the exact-digit tensor-core GEMM
int plan_exact(const rfcmp_op* op) { return op->plan.exact_min > 0 ? op->plan.exact_min : EXACT_MIN; }

void plan_to_scratch(rfcmp_op* op) {
  op->ws->gs.chunk = op->plan.gemv_chunk;
  op->ws->gs.ctas_per_sm = op->plan.gemv_ctas_per_sm;
  op->ws->ms.bn = op->plan.gemm_bn;
}

// Device memory is allocated and freed in the order of the legacy default stream, which the
// blocking streams are ordered with.  A non-blocking caller stream is not, so an entry point
// that queues work on one makes it wait for the legacy stream (the allocations made so far), and
// the op remembers it so that its memory is freed only after that stream's work.
int order_stream(rfcmp_op* op, cudaStream_t st) {
  if (!st) return RFCMP_OK;
  unsigned int flags = 0;
  RF_CUDA(cudaStreamGetFlags(st, &flags));
  if (!(flags & cudaStreamNonBlocking)) return RFCMP_OK;
  if (std::find(op->nb_streams.begin(), op->nb_streams.end(), st) == op->nb_streams.end())
    op->nb_streams.push_back(st);
  if (!op->order_ev) RF_CUDA(cudaEventCreateWithFlags(&op->order_ev, cudaEventDisableTiming));
  RF_CUDA(cudaEventRecord(op->order_ev, 0));
  RF_CUDA(cudaStreamWaitEvent(st, op->order_ev, 0));
  return RFCMP_OK;
}

// The legacy stream (where frees are queued) waits for the non-blocking streams op was used on.
int drain_streams(rfcmp_op* op) {
  for (cudaStream_t s : op->nb_streams) {
    if (!op->order_ev) RF_CUDA(cudaEventCreateWithFlags(&op->order_ev, cudaEventDisableTiming));
    RF_CUDA(cudaEventRecord(op->order_ev, s));
    RF_CUDA(cudaStreamWaitEvent(0, op->order_ev, 0));
  }
  return RFCMP_OK;
}

int ensure_workspace(rfcmp_op* op, int cols) {
  if (op->ws && op->ws->cols >= cols && (cols < plan_mrhs(op) || (op->ws->ms.xb && op->ws->ms.cap_cols >= cols)) &&
      (cols < plan_exact(op) || (op->ws->ms.xd && op->ws->ms.cap_cols >= cols))) {
    plan_to_scratch(op);
    return RFCMP_OK;
  }
  RF_TRY(drain_streams(op));  // the old workspace, if any, is freed below
  auto ws = std::make_unique<Workspace>();
  ws->cols = cols;
  const size_t N = op->top.ne, C = op->top.nc, NV = op->top.nv;
  for (double2** p : {&ws->v, &ws->u, &ws->y, &ws->up, &ws->tmpN}) RF_TRY(dalloc(p, N * cols, ws->owned));
  for (double2** p : {&ws->s, &ws->z, &ws->w, &ws->zu, &ws->q0, &ws->q, &ws->Lq, &ws->vp})
    RF_TRY(dalloc(p, C * cols, ws->owned));
  if (op->gtp)
    for (double2** p : {&ws->g1, &ws->g2}) RF_TRY(dalloc(p, C * cols, ws->owned));
  for (double2** p : {&ws->t, &ws->tg}) RF_TRY(dalloc(p, NV * cols, ws->owned));
  RF_TRY(dalloc(&ws->mean, 4 * (size_t)cols, ws->owned));  // pgp_apply uses 4 per column
  {
    const int capn = (int)std::max<int64_t>(N, std::max<int64_t>(C, NV));
    ws->gs.cap_n = capn;
    ws->gs.cap_ld = padded_ld(capn);
    ws->gs.cap_cols = 4;
    RF_TRY(dalloc(&ws->gs.xh, (size_t)ws->gs.cap_ld * 4, ws->owned));
    RF_TRY(dalloc(&ws->gs.xl, (size_t)ws->gs.cap_ld * 4, ws->owned));
    // one error flag for every bounded device-side wait (streaming GEMV, tensor-core products)
    RF_TRY(dalloc(&ws->ms.err, 1, ws->owned));
    RF_CUDA(cudaMemset(ws->ms.err, 0, sizeof(int)));
    ws->gs.err = ws->ms.err;
    ws->gs.symmetric = true;  // T_A, V, (Sigma^T Sigma)^+ and G_ll^{-1} are all symmetric
    const bool bf = cols >= plan_mrhs(op), ex = cols >= plan_exact(op);
    if (bf || ex) {
      ws->ms.cap_cols = cols;
      ws->ms.cap_n = capn;
      ws->ms.cap_ld = padded_ld(capn);
    }
    if (bf) {
      RF_TRY(dalloc(&ws->ms.xb, (size_t)4 * cols * ws->ms.cap_ld, ws->owned));
      RF_TRY(dalloc(&ws->ms.D, (size_t)4 * cols * capn, ws->owned));
    }
    if (ex) {
      RF_TRY(dalloc(&ws->ms.xd, (size_t)EXACT_DIGITS * 2 * cols * ws->ms.cap_ld, ws->owned));
      RF_TRY(dalloc(&ws->ms.xe, (size_t)2 * cols, ws->owned));
      RF_TRY(dalloc(&ws->ms.D64, (size_t)4 * cols * capn, ws->owned));
    }
  }
  op->ws = std::move(ws);
  plan_to_scratch(op);
  return RFCMP_OK;
}

int alloc_solve_buffers(rfcmp_op* op, int cols, std::unique_ptr<SolveBuffers>& out);

int ensure_solve_buffers(rfcmp_op* op, int cols) {
  if (op->sb && op->sb->cols >= cols) return RFCMP_OK;
  RF_TRY(drain_streams(op));
  return alloc_solve_buffers(op, cols, op->sb);
}

int alloc_solve_buffers(rfcmp_op* op, int cols, std::unique_ptr<SolveBuffers>& out) {
  auto sb = std::make_unique<SolveBuffers>();
  sb->cols = cols;
  const size_t N = op->top.ne;
  for (double2** p : {&sb->b, &sb->i, &sb->r, &sb->d, &sb->rin, &sb->p, &sb->Ap, &sb->tmp})
    RF_TRY(dalloc(p, N * cols, sb->owned));
  RF_TRY(dalloc(&sb->dots, cols, sb->owned));
  RF_TRY(dalloc(&sb->rho, cols, sb->owned));
  RF_TRY(dalloc(&sb->alpha, cols, sb->owned));
  RF_TRY(dalloc(&sb->beta, cols, sb->owned));
  RF_TRY(dalloc(&sb->active, cols, sb->owned));
  RF_TRY(dalloc(&sb->ctl, 1, sb->owned));
  for (double** p : {&sb->bb, &sb->rr, &sb->r0, &sb->res}) RF_TRY(dalloc(p, cols, sb->owned));
  for (int** p : {&sb->conv, &sb->iters, &sb->sweeps}) RF_TRY(dalloc(p, cols, sb->owned));
  RF_TRY(dalloc(&sb->part, (size_t)cols * KRYLOV_MAX_G, sb->owned));
  RF_TRY(dalloc(&sb->ticket, cols, sb->owned));
  RF_CUDA(cudaMemset(sb->ticket, 0, sizeof(unsigned int) * cols));
  RF_CUDA(cudaMemset(sb->ctl, 0, sizeof(KrylovCtl)));
  out = std::move(sb);
  return RFCMP_OK;
}

int ensure_planes(rfcmp_op* op, cudaStream_t st);

#define RF_K(call)                                                                                      \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return set_error(RFCMP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int make_cplx_planes(rfcmp_op* op, const float2* M, int n, int ld, CplxPlanes& P, cudaStream_t st) {
  if (P.rh) return RFCMP_OK;
  CplxPlanes q;
  q.n = n;
  q.ldp = ld;
  const size_t pl = (size_t)n * ld;
  // Re and Im rows stacked in one hi and one lo buffer: the product reads them as one 2n-row operand
  RF_TRY(dalloc(&q.rh, 2 * pl, op->lazy));
  RF_TRY(dalloc(&q.rl, 2 * pl, op->lazy));
  q.ih = q.rh + pl;
  q.il = q.rl + pl;
  RF_K(split_c64_planes(M, n, ld, q, st));
  op->bytes += 4 * pl * sizeof(__nv_bfloat16);
  op->lazy_bytes += 4 * pl * sizeof(__nv_bfloat16);
  op->ctx->bytes += 4 * pl * sizeof(__nv_bfloat16);
  P = q;
  return RFCMP_OK;
}

int make_real_planes(rfcmp_op* op, DenseFactor& f, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(f.planes_mu);
  if (f.planes.h) return RFCMP_OK;
  RealPlanes q;
  q.n = f.n;
  q.ldp = padded_ld(f.n);
  const size_t pl = (size_t)f.n * q.ldp;
  RF_CUDA(dev_malloc(&q.h, pl * sizeof(__nv_bfloat16)));
  RF_CUDA(dev_malloc(&q.l, pl * sizeof(__nv_bfloat16)));
  RF_CUDA(cudaMemsetAsync(q.h, 0, pl * sizeof(__nv_bfloat16), st));
  RF_CUDA(cudaMemsetAsync(q.l, 0, pl * sizeof(__nv_bfloat16), st));
  RF_K(split_bf16_f32(f.hi, q.ldp, f.n, f.n, q.h, q.l, q.ldp, st));
  f.bytes += 2 * pl * sizeof(__nv_bfloat16);
  op->ctx->bytes += 2 * pl * sizeof(__nv_bfloat16);
  f.planes = q;
  return RFCMP_OK;
}

int ensure_planes(rfcmp_op* op, cudaStream_t st) {
  RF_TRY(make_cplx_planes(op, op->TA, (int)op->top.ne, op->ldN, op->ta_planes, st));
  RF_TRY(make_cplx_planes(op, op->V, (int)op->top.nc, op->ldC, op->v_planes, st));
  RF_TRY(make_real_planes(op, *op->lplus, st));
  RF_TRY(make_real_planes(op, *op->gll, st));
  if (op->gtp) RF_TRY(make_real_planes(op, *op->gtp, st));
  return RFCMP_OK;
}

// Reads the error flag of the bounded device-side waits (tensor-core products, streaming GEMV).
int check_tensor_core_waits(rfcmp_op* op, cudaStream_t st) {
  if (!op->ws || !op->ws->ms.err) return RFCMP_OK;
  int h_err = 0;
  RF_CUDA(cudaMemcpyAsync(&h_err, op->ws->ms.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaStreamSynchronize(st));
  if (h_err) {
    RF_CUDA(cudaMemsetAsync(op->ws->ms.err, 0, sizeof(int), st));
    return set_error(RFCMP_ERR_DEVICE_TIMEOUT,
                     "a bounded device-side wait gave up (code " + std::to_string(h_err) + ")");
  }
  return RFCMP_OK;
}

int alloc_digits(ExactOperand& q, int rows, long long ldp, std::vector<void*>* owned) {
  q.rows = rows;
  q.ldp = ldp;
  q.plane_stride = (long long)rows * ldp;
  if (owned) {
    RF_TRY(dalloc(&q.d, (size_t)EXACT_DIGITS * q.plane_stride, *owned));
    RF_TRY(dalloc(&q.e, (size_t)rows, *owned));
  } else {
    RF_CUDA(dev_malloc(&q.d, (size_t)EXACT_DIGITS * q.plane_stride * sizeof(__nv_bfloat16)));
    RF_CUDA(dev_malloc(&q.e, (size_t)rows * sizeof(int)));
  }
  return RFCMP_OK;
}

int make_cplx_digits(rfcmp_op* op, const float2* M, int n, int ld, ExactOperand& P, cudaStream_t st) {
  if (P.d) return RFCMP_OK;
  ExactOperand q;
  RF_TRY(alloc_digits(q, 2 * n, ld, &op->lazy));
  RF_K(exact_digits_c64(M, n, ld, q, st));
  const uint64_t b = (uint64_t)EXACT_DIGITS * q.plane_stride * sizeof(__nv_bfloat16) + 2ull * n * sizeof(int);
  op->bytes += b;
  op->lazy_bytes += b;
  op->ctx->bytes += b;
  P = q;
  return RFCMP_OK;
}

int make_real_digits(rfcmp_op* op, DenseFactor& f, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(f.planes_mu);
  if (f.digits.d) return RFCMP_OK;
  ExactOperand q;
  RF_TRY(alloc_digits(q, f.n, padded_ld(f.n), nullptr));
  RF_K(exact_digits_f32pair(f.hi, f.lo, f.n, q.ldp, q, st));
  const uint64_t b = (uint64_t)EXACT_DIGITS * q.plane_stride * sizeof(__nv_bfloat16) + (uint64_t)f.n * sizeof(int);
  f.bytes += b;
  op->ctx->bytes += b;
  f.digits = q;
  return RFCMP_OK;
}

int ensure_digits(rfcmp_op* op, cudaStream_t st) {
  RF_TRY(make_cplx_digits(op, op->TA, (int)op->top.ne, op->ldN, op->ta_digits, st));
  RF_TRY(make_cplx_digits(op, op->V, (int)op->top.nc, op->ldC, op->v_digits, st));
  RF_TRY(make_real_digits(op, *op->lplus, st));
  RF_TRY(make_real_digits(op, *op->gll, st));
  if (op->gtp) RF_TRY(make_real_digits(op, *op->gtp, st));
  return RFCMP_OK;
}

// y = scale * op(M) x (+ y) for M = T_A or V: GEMV, or the tensor-core product for wide FP32 blocks
// (split-BF16 in the inner iterations, exact digits where float-float accuracy is asked)
int prod_c(rfcmp_op* op, bool ta, const double2* x, double2* y, int nr, bool conj, double2 scale, bool acc,
           GemvMode m, cudaStream_t st, bool fed = false) {
  if (m == GEMV_FF && nr >= plan_exact(op)) {
    RF_TRY(ensure_digits(op, st));
    RF_K(exact_cplx_gemm(ta ? op->ta_digits : op->v_digits, ta ? (int)op->top.ne : (int)op->top.nc, x, y, nr, conj,
                         scale, acc, op->ws->ms, st));
    return RFCMP_OK;
  }
  if (m == GEMV_F32 && nr >= plan_mrhs(op)) {
    RF_TRY(ensure_planes(op, st));
    RF_K(cplx_gemm(ta ? op->ta_planes : op->v_planes, x, y, nr, conj, scale, acc, op->ws->ms, st));
    return RFCMP_OK;
  }
  RF_K(gemv_c64(ta ? op->TA : op->V, ta ? (int)op->top.ne : (int)op->top.nc, x, y, nr, conj, scale, acc, m,
                op->ws->gs, st, fed));
  return RFCMP_OK;
}

// y = scale * F x (+ y) for a dense real factor
int prod_r(rfcmp_op* op, DenseFactor& f, const double2* x, double2* y, int nr, double scale, bool acc, GemvMode m,
           cudaStream_t st, bool fed = false) {
  if (m == GEMV_FF && nr >= plan_exact(op)) {
    RF_TRY(ensure_digits(op, st));
    RF_K(exact_real_gemm(f.digits, f.n, x, y, nr, scale, acc, op->ws->ms, st));
    return RFCMP_OK;
  }
  if (m == GEMV_F32 && nr >= plan_mrhs(op)) {
    RF_TRY(ensure_planes(op, st));
    RF_K(real_gemm(f.planes, x, y, nr, scale, acc, op->ws->ms, st));
    return RFCMP_OK;
  }
  RF_K(gemv_r32(f.hi, f.lo, f.n, x, y, nr, scale, acc, m, op->ws->gs, st, fed));
  return RFCMP_OK;
}

// Whether prod_c / prod_r of nr columns in mode m take the GEMV (1, 2 or 4 columns below the
// tensor-core widths), so that the sparse kernel producing their x can write its split
// (GemvFeed) and the GEMV skip its own.
bool gemv_feedable(const rfcmp_op* op, int nr, GemvMode m) {
  if (nr != 1 && nr != 2 && nr != 4) return false;
  return m == GEMV_FF ? nr < plan_exact(op) : nr < plan_mrhs(op);
}

// the feed of a length-n vector whose GEMV writes y (and a second GEMV of it y2); none if !on
GemvFeed make_feed(rfcmp_op* op, bool on, int n, GemvMode m, double2* y, double2* y2 = nullptr) {
  GemvFeed f;
  if (!on) return f;
  f.xh = op->ws->gs.xh;
  f.xl = m == GEMV_FF ? op->ws->gs.xl : nullptr;
  f.ld = padded_ld(n);
  f.y = y;
  f.y2 = y2;
  return f;
}

// ---- building blocks of the application, nrhs columns, column-major ----
// z = (Sigma^T Sigma)^+ Sigma^T x  (N_C) using s as scratch for Sigma^T x
int star_coeff(rfcmp_op* op, const double2* x, double2* s, double2* z, int nr, GemvMode m, cudaStream_t st) {
  RF_K(sigma_t(op->g, x, s, nr, st));
  RF_TRY(prod_r(op, *op->lplus, s, z, nr, 1.0, false, m, st));
  return RFCMP_OK;
}

// out = A x (Sec. 3 Eq. NewFormulation, numerical variant of Sec. 4) in the
// low-frequency-stable order: analytically vanishing products are not formed.
int apply_A_gsigma(rfcmp_op* op, const double2* x, double2* out, int nr, GemvMode m, cudaStream_t st);

int apply_A(rfcmp_op* op, const double2* x, double2* out, int nr, GemvMode m, cudaStream_t st) {
  if (op->outer == RFCMP_OUTER_GSIGMA) return apply_A_gsigma(op, x, out, nr, m, st);
  RF_TRY(ensure_workspace(op, nr));
  Workspace& W = *op->ws;
  const DeviceGeometry& g = op->g;
  const double k = op->k, a = op->alpha, b = op->beta, gm = op->gamma;
  const int N = (int)op->top.ne, C = (int)op->top.nc, NV = (int)op->top.nv;
  // every sparse kernel below writes the split of its output for the GEMV that reads it next
  const bool fd = gemv_feedable(op, nr, m);
  // s = Sigma^T x, z = L^+ s ; w = V Sigma^T x / (k b) (the same split of s)
  RF_K(sigma_t(g, x, W.s, nr, st, make_feed(op, fd, C, m, W.z, W.w)));
  RF_TRY(prod_r(op, *op->lplus, W.s, W.z, nr, 1.0, false, m, st, fd));
  RF_TRY(prod_c(op, false, W.s, W.w, nr, false, c2(1.0 / (k * b), 0.0), false, m, st, fd));
  // v = (ik/a) x - (ik/a + k/b) Sigma z      = i k x_L / a - k x_S / b ; u = T_A v
  {
    EdgeCombo c;
    c.x = x;
    c.a = c2(0.0, k / a);
    c.zs = W.z;
    c.b = c2(-k / b, -k / a);
    RF_K(edge_combo(g, c, W.v, nr, st, make_feed(op, fd, N, m, W.u)));
  }
  RF_TRY(prod_c(op, true, W.v, W.u, nr, false, c2(1.0, 0.0), false, m, st, fd));
  // zu = L^+ Sigma^T u ; tg = G_ll^{-1} Lambda^T u
  RF_K(sigma_t(g, W.u, W.s, nr, st, make_feed(op, fd, C, m, W.zu)));
  RF_TRY(prod_r(op, *op->lplus, W.s, W.zu, nr, 1.0, false, m, st, fd));
  RF_K(lambda_t(g, W.u, W.t, nr, st, make_feed(op, fd, NV, m, W.tg)));
  RF_TRY(prod_r(op, *op->gll, W.t, W.tg, nr, 1.0, false, m, st, fd));
  // q = L^+ G_pp^{-1} (zu + w - mean(w)) / b^2
  RF_K(star_middle(g, W.zu, W.w, 1.0, W.q0, nr, W.mean, st, make_feed(op, fd, C, m, W.q)));
  RF_TRY(prod_r(op, *op->lplus, W.q0, W.q, nr, 1.0 / (b * b), false, m, st, fd));
  // y = Lambda tg / a^2 + (u - Sigma zu) / gamma + Sigma q
  {
    EdgeCombo c;
    c.zl = W.tg;
    c.c = c2(1.0 / (a * a), 0.0);
    c.x = W.u;
    c.a = c2(1.0 / gm, 0.0);
    c.zs = W.zu;
    c.b = c2(-1.0 / gm, 0.0);
    c.zs2 = W.q;
    c.d = c2(1.0, 0.0);
    RF_K(edge_combo(g, c, W.y, nr, st, make_feed(op, fd, N, m, W.up)));
  }
  // up = conj(T_A) y ; vp = conj(V) (Sigma^T Sigma) q / (k b)
  RF_TRY(prod_c(op, true, W.y, W.up, nr, true, c2(1.0, 0.0), false, m, st, fd));
  RF_K(lap_apply(g, W.q, W.Lq, nr, st, make_feed(op, fd, C, m, W.vp)));
  RF_TRY(prod_c(op, false, W.Lq, W.vp, nr, true, c2(1.0 / (k * b), 0.0), false, m, st, fd));
  // zp = L^+ Sigma^T up
  RF_K(sigma_t(g, W.up, W.s, nr, st, make_feed(op, fd, C, m, W.z)));
  RF_TRY(prod_r(op, *op->lplus, W.s, W.z, nr, 1.0, false, m, st, fd));
  // out = -(ik/a) up + (ik/a - k/b) Sigma zp + Sigma vp
  {
    EdgeCombo c;
    c.x = W.up;
    c.a = c2(0.0, -k / a);
    c.zs = W.z;
    c.b = c2(-k / b, k / a);
    c.zs2 = W.vp;
    c.d = c2(1.0, 0.0);
    RF_K(edge_combo(g, c, out, nr, st));
  }
  return RFCMP_OK;
}

// y = P_m T P_o x from u (= T_A v) and w (= V ... / (k b)), the middle of both forms of A:
//   y = Lambda G_ll^{-1} Lambda^T u / a^2 + (u - Sigma zu) / gamma + Sigma q,
//   zu = L^+ Sigma^T u,  q = L^+ G_pp^{-1} (zu + w - mean(w)) / b^2  (W.zu, W.q, W.y)
int apply_middle(rfcmp_op* op, GemvMode m, int nr, cudaStream_t st) {
  Workspace& W = *op->ws;
  const DeviceGeometry& g = op->g;
  const double a = op->alpha, b = op->beta, gm = op->gamma;
  RF_TRY(star_coeff(op, W.u, W.s, W.zu, nr, m, st));
  RF_K(lambda_t(g, W.u, W.t, nr, st));
  RF_TRY(prod_r(op, *op->gll, W.t, W.tg, nr, 1.0, false, m, st));
  RF_K(star_middle(g, W.zu, W.w, 1.0, W.q0, nr, W.mean, st));
  RF_TRY(prod_r(op, *op->lplus, W.q0, W.q, nr, 1.0 / (b * b), false, m, st));
  EdgeCombo c;
  c.zl = W.tg;
  c.c = c2(1.0 / (a * a), 0.0);
  c.x = W.u;
  c.a = c2(1.0 / gm, 0.0);
  c.zs = W.zu;
  c.b = c2(-1.0 / gm, 0.0);
  c.zs2 = W.q;
  c.d = c2(1.0, 0.0);
  RF_K(edge_combo(g, c, W.y, nr, st));
  return RFCMP_OK;
}

// out = A x with P_o = P_LH / a + i P_gS / b, P_gS = Sigma L^+ G^{-1} Sigma^T (Sec. 3, Eq. Pgs;
// G = G_l~p, L = Sigma^T Sigma), in the low-frequency-stable order.  With s = Sigma^T x,
// z = L^+ s (x_L = x - Sigma z), t = G^{-1} s, z' = L^+ t:
//   T P_o x = u + Sigma w,  u = T_A ((ik/a) x_L - (k/b) Sigma z'),  w = V Pi t / (k b),
// (Sigma^T x_L = 0, Sigma^T Sigma L^+ = Pi = I - 1 1^T / N_C); y = P_m T P_o x as in apply_A;
//   A x = -(ik/a) P_LH u' + Sigma G^{-1} (-(k/b) zp + Pi vp),
// u' = conj(T_A) y, zp = L^+ Sigma^T u', vp = conj(V) L q / (k b), from P_gS^H = Sigma G^{-1} L^+
// Sigma^T and Sigma^T y = L q.
int apply_A_gsigma(rfcmp_op* op, const double2* x, double2* out, int nr, GemvMode m, cudaStream_t st) {
  RF_TRY(ensure_workspace(op, nr));
  Workspace& W = *op->ws;
  const DeviceGeometry& g = op->g;
  const double k = op->k, a = op->alpha, b = op->beta;
  RF_K(sigma_t(g, x, W.s, nr, st));
  RF_TRY(prod_r(op, *op->lplus, W.s, W.z, nr, 1.0, false, m, st));
  RF_TRY(prod_r(op, *op->gtp, W.s, W.g1, nr, 1.0, false, m, st));
  RF_TRY(prod_r(op, *op->lplus, W.g1, W.g2, nr, 1.0, false, m, st));
  {  // v = (ik/a) x - (ik/a) Sigma z - (k/b) Sigma z'
    EdgeCombo c;
    c.x = x;
    c.a = c2(0.0, k / a);
    c.zs = W.z;
    c.b = c2(0.0, -k / a);
    c.zs2 = W.g2;
    c.d = c2(-k / b, 0.0);
    RF_K(edge_combo(g, c, W.v, nr, st));
  }
  RF_TRY(prod_c(op, true, W.v, W.u, nr, false, c2(1.0, 0.0), false, m, st));
  RF_K(cell_combo(g, nullptr, c2(0, 0), W.g1, c2(1.0, 0.0), W.q0, nr, W.mean, st));  // Pi t
  RF_TRY(prod_c(op, false, W.q0, W.w, nr, false, c2(1.0 / (k * b), 0.0), false, m, st));
  RF_TRY(apply_middle(op, m, nr, st));
  RF_TRY(prod_c(op, true, W.y, W.up, nr, true, c2(1.0, 0.0), false, m, st));
  RF_K(lap_apply(g, W.q, W.Lq, nr, st));
  RF_TRY(prod_c(op, false, W.Lq, W.vp, nr, true, c2(1.0 / (k * b), 0.0), false, m, st));
  RF_TRY(star_coeff(op, W.up, W.s, W.z, nr, m, st));  // zp
  RF_K(cell_combo(g, W.z, c2(-k / b, 0.0), W.vp, c2(1.0, 0.0), W.g1, nr, W.mean, st));
  RF_TRY(prod_r(op, *op->gtp, W.g1, W.g2, nr, 1.0, false, m, st));
  EdgeCombo c;  // out = -(ik/a) up + (ik/a) Sigma zp + Sigma G^{-1}(...)
  c.x = W.up;
  c.a = c2(0.0, -k / a);
  c.zs = W.z;
  c.b = c2(0.0, k / a);
  c.zs2 = W.g2;
  c.d = c2(1.0, 0.0);
  RF_K(edge_combo(g, c, out, nr, st));
  return RFCMP_OK;
}

// b = -P_o^H T^H P_m e in the same order
int apply_rhs(rfcmp_op* op, const double2* e, double2* out, int nr, GemvMode m, cudaStream_t st) {
  RF_TRY(ensure_workspace(op, nr));
  Workspace& W = *op->ws;
  const DeviceGeometry& g = op->g;
  const double k = op->k, a = op->alpha, b = op->beta, gm = op->gamma;
  const int N = (int)op->top.ne, C = (int)op->top.nc, NV = (int)op->top.nv;
  RF_TRY(star_coeff(op, e, W.s, W.zu, nr, m, st));  // ze
  RF_K(star_middle(g, W.zu, nullptr, 1.0, W.q0, nr, W.mean, st));
  RF_TRY(prod_r(op, *op->lplus, W.q0, W.q, nr, 1.0 / (b * b), false, m, st));
  RF_K(lambda_t(g, e, W.t, nr, st));
  RF_TRY(prod_r(op, *op->gll, W.t, W.tg, nr, 1.0, false, m, st));
  {
    EdgeCombo c;
    c.zl = W.tg;
    c.c = c2(1.0 / (a * a), 0.0);
    c.x = e;
    c.a = c2(1.0 / gm, 0.0);
    c.zs = W.zu;
    c.b = c2(-1.0 / gm, 0.0);
    c.zs2 = W.q;
    c.d = c2(1.0, 0.0);
    RF_K(edge_combo(g, c, W.y, nr, st));
  }
  RF_TRY(prod_c(op, true, W.y, W.up, nr, true, c2(1.0, 0.0), false, m, st));
  RF_K(lap_apply(g, W.q, W.Lq, nr, st));
  RF_TRY(prod_c(op, false, W.Lq, W.vp, nr, true, c2(1.0, 0.0), false, m, st));
  {  // th = -ik up + (i/k) Sigma vp
    EdgeCombo c;
    c.x = W.up;
    c.a = c2(0.0, -k);
    c.zs = W.vp;
    c.b = c2(0.0, 1.0 / k);
    RF_K(edge_combo(g, c, W.tmpN, nr, st));
  }
  RF_TRY(star_coeff(op, W.tmpN, W.s, W.z, nr, m, st));
  if (op->outer == RFCMP_OUTER_GSIGMA) {  // out = -th / a + Sigma zt / a + (i/b) Sigma G^{-1} zt
    RF_TRY(prod_r(op, *op->gtp, W.z, W.g1, nr, 1.0, false, m, st));
    EdgeCombo c;
    c.x = W.tmpN;
    c.a = c2(-1.0 / a, 0.0);
    c.zs = W.z;
    c.b = c2(1.0 / a, 0.0);
    c.zs2 = W.g1;
    c.d = c2(0.0, 1.0 / b);
    RF_K(edge_combo(g, c, out, nr, st));
    return RFCMP_OK;
  }
  {  // out = -th / a + Sigma zt (1/a + i/b)
    EdgeCombo c;
    c.x = W.tmpN;
    c.a = c2(-1.0 / a, 0.0);
    c.zs = W.z;
    c.b = c2(1.0 / a, 1.0 / b);
    RF_K(edge_combo(g, c, out, nr, st));
  }
  return RFCMP_OK;
}

// P_o x (adj: P_o^H x) = x / a + Sigma z (-1/a +- i/b)
int apply_Po(rfcmp_op* op, const double2* x, double2* out, int nr, bool adj, GemvMode m, cudaStream_t st) {
  RF_TRY(ensure_workspace(op, nr));
  Workspace& W = *op->ws;
  RF_TRY(star_coeff(op, x, W.s, W.z, nr, m, st));
  if (op->outer == RFCMP_OUTER_GSIGMA) {
    // P_o x = x_L / a + (i/b) Sigma L^+ G^{-1} Sigma^T x;  P_o^H x = x_L / a - (i/b) Sigma G^{-1} L^+ Sigma^T x
    if (adj) {
      RF_TRY(prod_r(op, *op->gtp, W.z, W.g2, nr, 1.0, false, m, st));
    } else {
      RF_TRY(prod_r(op, *op->gtp, W.s, W.g1, nr, 1.0, false, m, st));
      RF_TRY(prod_r(op, *op->lplus, W.g1, W.g2, nr, 1.0, false, m, st));
    }
    EdgeCombo c;
    c.x = x;
    c.a = c2(1.0 / op->alpha, 0.0);
    c.zs = W.z;
    c.b = c2(-1.0 / op->alpha, 0.0);
    c.zs2 = W.g2;
    c.d = c2(0.0, adj ? -1.0 / op->beta : 1.0 / op->beta);
    RF_K(edge_combo(op->g, c, out, nr, st));
    return RFCMP_OK;
  }
  EdgeCombo c;
  c.x = x;
  c.a = c2(1.0 / op->alpha, 0.0);
  c.zs = W.z;
  c.b = c2(-1.0 / op->alpha, adj ? -1.0 / op->beta : 1.0 / op->beta);
  RF_K(edge_combo(op->g, c, out, nr, st));
  return RFCMP_OK;
}

// ---- power iteration operators (unscaled by k, frequency-scaled reading of Sec. 4) ----
// Columns 0 and 1 of x (N x 2) go through
//   X = P_LH T_A^H Lambda G_ll^{-1} Lambda^T T_A P_LH   (column 0, for alpha) and
//   Z = P_LH T_A^H P_LH T_A P_LH                         (column 1, for gamma),
// sharing each pass over T_A.
int op_XZ(rfcmp_op* op, const double2* x, double2* out, cudaStream_t st) {
  Workspace& W = *op->ws;
  const int N = (int)op->top.ne, NV = (int)op->top.nv;
  const GemvMode m = GEMV_F32;
  RF_TRY(star_coeff(op, x, W.s, W.z, 2, m, st));
  EdgeCombo c;
  c.x = x;
  c.a = c2(1, 0);
  c.zs = W.z;
  c.b = c2(-1, 0);
  RF_K(edge_combo(op->g, c, W.v, 2, st));
  RF_K(gemv_c64(op->TA, N, W.v, W.u, 2, false, c2(1, 0), false, m, op->ws->gs, st));
  // column 0: Lambda G_ll^{-1} Lambda^T u0
  RF_K(lambda_t(op->g, W.u, W.t, 1, st));
  RF_K(gemv_r32(op->gll->hi, op->gll->lo, NV, W.t, W.tg, 1, 1.0, false, m, op->ws->gs, st));
  EdgeCombo l;
  l.zl = W.tg;
  l.c = c2(1, 0);
  RF_K(edge_combo(op->g, l, W.y, 1, st));
  // column 1: P_LH u1
  RF_TRY(star_coeff(op, W.u + N, W.s, W.z, 1, m, st));
  EdgeCombo p1;
  p1.x = W.u + N;
  p1.a = c2(1, 0);
  p1.zs = W.z;
  p1.b = c2(-1, 0);
  RF_K(edge_combo(op->g, p1, W.y + N, 1, st));
  RF_K(gemv_c64(op->TA, N, W.y, W.up, 2, true, c2(1, 0), false, m, op->ws->gs, st));
  RF_TRY(star_coeff(op, W.up, W.s, W.z, 2, m, st));
  EdgeCombo o;
  o.x = W.up;
  o.a = c2(1, 0);
  o.zs = W.z;
  o.b = c2(-1, 0);
  RF_K(edge_combo(op->g, o, out, 2, st));
  return RFCMP_OK;
}

// Y x = P_S T_Phi^H M_S T_Phi P_S x = Sigma conj(V) Pi G_pp^{-1} Pi V Sigma^T x,  Pi = I - 1 1^T / N_C
// (Sigma^T P_S = Sigma^T, (Sigma^T Sigma)(Sigma^T Sigma)^+ = Pi, P_S Sigma = Sigma)
int op_Y(rfcmp_op* op, const double2* x, double2* out, cudaStream_t st) {
  Workspace& W = *op->ws;
  const int C = (int)op->top.nc;
  const GemvMode m = GEMV_F32;
  RF_K(sigma_t(op->g, x, W.s, 1, st));
  RF_K(gemv_c64(op->V, C, W.s, W.w, 1, false, c2(1, 0), false, m, op->ws->gs, st));
  RF_K(pgp_apply(op->g, W.w, W.q0, 1, W.mean, st));
  RF_K(gemv_c64(op->V, C, W.q0, W.vp, 1, true, c2(1, 0), false, m, op->ws->gs, st));
  EdgeCombo c;
  c.zs = W.vp;
  c.b = c2(1, 0);
  RF_K(edge_combo(op->g, c, out, 1, st));
  return RFCMP_OK;
}

// deterministic start vector: splitmix64(seed * 2^32 + i) top 53 bits / 2^53 - 1/2 (real)
void splitmix_start(std::vector<double2>& h, int64_t n, uint64_t seed) {
  h.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t z = seed * (1ull << 32) + (uint64_t)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    h[i] = make_double2((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5, 0.0);
  }
}

// Largest eigenvalues of `cols` HPSD operators applied together (column c of the block goes
// through operator c), by normalised power steps from splitmix64 start vectors (seeds[c]);
// Rayleigh-quotient estimates.  Each column stops once its estimate changes by at most rtol
// (relative) between steps (after at least 2 steps; rtol = 0: always `steps`).
// Largest eigenpair of a small symmetric matrix (row-major m x m) by cyclic Jacobi rotations.
double small_sym_max_eig(std::vector<double> A, int m, std::vector<double>& vec) {
  std::vector<double> V((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) off += A[(size_t)p * m + q] * A[(size_t)p * m + q];
    if (off < 1e-30) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[(size_t)p * m + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double th = 0.5 * (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / apq;
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
          A[(size_t)k * m + p] = c * akp - sn * akq;
          A[(size_t)k * m + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
          A[(size_t)p * m + k] = c * apk - sn * aqk;
          A[(size_t)q * m + k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
          V[(size_t)k * m + p] = c * vkp - sn * vkq;
          V[(size_t)k * m + q] = sn * vkp + c * vkq;
        }
      }
  }
  int best = 0;
  for (int i = 1; i < m; ++i)
    if (A[(size_t)i * m + i] > A[(size_t)best * m + best]) best = i;
  vec.resize(m);
  for (int k = 0; k < m; ++k) vec[k] = V[(size_t)k * m + best];
  return A[(size_t)best * m + best];
}

// Largest eigenvalue of the Hermitian positive semi-definite operators X, Z (two columns at once)
// and Y of the scaling (Sec. 4, second display), i.e. their spectral norms, by a Lanczos
// iteration per column: the Ritz value of the tridiagonal T_j grows monotonically to the largest
// eigenvalue and converges far faster than the power iteration's Rayleigh quotient from the same
// start.  Stops a column once its Ritz value moves by at most rtol (relative) between two steps,
// after at least 2 and at most `steps` steps (rtol = 0: always `steps`).  The start is the
// splitmix64 vector of each seed or `start`; `keep` receives each column's Ritz vector (the warm
// start of the next wavenumber of a sweep).
template <class Op>
int power_norms(rfcmp_op* op, Op apply, int cols, const uint64_t* seeds, int steps, double rtol, double* lam,
                const double2* start, double2* keep, cudaStream_t st) {
  const int64_t N = op->top.ne;
  RF_TRY(ensure_solve_buffers(op, cols));
  RF_TRY(ensure_workspace(op, cols));
  SolveBuffers& B = *op->sb;
  const size_t slot = (size_t)N * cols;
  if (op->lanczos_slots < steps + 1) {
    if (op->lanczos) dev_free(op->lanczos);
    op->lanczos = nullptr;
    op->lanczos_slots = 0;
    RF_CUDA(dev_malloc(&op->lanczos, sizeof(double2) * slot * 2 * (steps + 1)));  // room for 2 columns
    op->lanczos_slots = steps + 1;
  }
  double2* Vb = op->lanczos;
  auto Vs = [&](int j) { return Vb + (size_t)j * slot; };
  if (start) {
    RF_CUDA(cudaMemcpyAsync(Vs(0), start, sizeof(double2) * slot, cudaMemcpyDeviceToDevice, st));
  } else {
    std::vector<double2> h;
    for (int c = 0; c < cols; ++c) {
      splitmix_start(h, N, seeds[c]);
      RF_CUDA(cudaMemcpyAsync(Vs(0) + c * N, h.data(), sizeof(double2) * N, cudaMemcpyHostToDevice, st));
    }
  }
  std::vector<double2> d(cols);
  std::vector<double> coef(cols);
  std::vector<std::vector<double>> al(cols), be(cols);  // T_j: diagonal al, off-diagonal be[1..]
  std::vector<double> theta(cols, 0.0);
  std::vector<int> done(cols, 0), size(cols, 0);
  RF_K(vec_dot(Vs(0), Vs(0), N, cols, B.dots, st));
  RF_CUDA(cudaMemcpyAsync(d.data(), B.dots, sizeof(double2) * cols, cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaStreamSynchronize(st));
  for (int c = 0; c < cols; ++c) coef[c] = d[c].x > 0.0 ? 1.0 / std::sqrt(d[c].x) : 0.0;
  RF_CUDA(cudaMemcpyAsync(B.alpha, coef.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st));
  RF_K(vec_copy_scale_cols(Vs(0), B.alpha, Vs(0), N, cols, st));
  int j = 0;
  for (; j < steps; ++j) {
    double2* W = B.Ap;
    RF_TRY(apply(op, Vs(j), W, st));
    RF_K(vec_dot(Vs(j), W, N, cols, B.dots, st));  // alpha_j = v_j^H A v_j (real)
    RF_CUDA(cudaMemcpyAsync(d.data(), B.dots, sizeof(double2) * cols, cudaMemcpyDeviceToHost, st));
    RF_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < cols; ++c) coef[c] = d[c].x;
    for (int c = 0; c < cols; ++c)
      if (!done[c]) al[c].push_back(d[c].x);
    RF_CUDA(cudaMemcpyAsync(B.alpha, coef.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st));
    RF_K(vec_axpy_cols(B.alpha, true, Vs(j), W, N, cols, nullptr, st));  // w -= alpha_j v_j
    if (j > 0) {
      for (int c = 0; c < cols; ++c) coef[c] = be[c].size() > (size_t)j ? be[c][j] : 0.0;
      RF_CUDA(cudaMemcpyAsync(B.beta, coef.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st));
      RF_K(vec_axpy_cols(B.beta, true, Vs(j - 1), W, N, cols, nullptr, st));  // w -= beta_j v_{j-1}
    }
    RF_K(vec_dot(W, W, N, cols, B.dots, st));
    RF_CUDA(cudaMemcpyAsync(d.data(), B.dots, sizeof(double2) * cols, cudaMemcpyDeviceToHost, st));
    RF_CUDA(cudaStreamSynchronize(st));
    bool all = true;
    for (int c = 0; c < cols; ++c) {
      if (done[c]) continue;
      const int m = (int)al[c].size();
      std::vector<double> T((size_t)m * m, 0.0), s;
      for (int i = 0; i < m; ++i) {
        T[(size_t)i * m + i] = al[c][i];
        if (i > 0) T[(size_t)i * m + i - 1] = T[(size_t)(i - 1) * m + i] = be[c][i];
      }
      const double prev = theta[c];
      theta[c] = small_sym_max_eig(T, m, s);
      size[c] = m;
      const double bnext = d[c].x > 0.0 ? std::sqrt(d[c].x) : 0.0;
      if (be[c].empty()) be[c].push_back(0.0);  // be[0] unused
      be[c].push_back(bnext);
      if ((rtol > 0.0 && j >= 1 && std::fabs(theta[c] - prev) <= rtol * std::fabs(theta[c])) ||
          !(bnext > 1e-14 * std::fabs(theta[c])))
        done[c] = 1;
      all &= done[c] != 0;
    }
    if (all || j + 1 == steps) {
      ++j;
      break;
    }
    for (int c = 0; c < cols; ++c) coef[c] = !done[c] && be[c].back() > 0.0 ? 1.0 / be[c].back() : 0.0;
    RF_CUDA(cudaMemcpyAsync(B.alpha, coef.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st));
    RF_K(vec_copy_scale_cols(W, B.alpha, Vs(j + 1), N, cols, st));  // v_{j+1} = w / beta_{j+1}
  }
  for (int c = 0; c < cols; ++c) lam[c] = theta[c];
  if (keep) {
    // Ritz vectors: keep[:, c] = sum_i s_i v_i with s the top eigenvector of column c's T
    RF_CUDA(cudaMemsetAsync(keep, 0, sizeof(double2) * slot, st));
    std::vector<std::vector<double>> S(cols);
    for (int c = 0; c < cols; ++c) {
      const int m = size[c];
      std::vector<double> T((size_t)m * m, 0.0);
      for (int i = 0; i < m; ++i) {
        T[(size_t)i * m + i] = al[c][i];
        if (i > 0) T[(size_t)i * m + i - 1] = T[(size_t)(i - 1) * m + i] = be[c][i];
      }
      small_sym_max_eig(T, m, S[c]);
    }
    int mmax = 0;
    for (int c = 0; c < cols; ++c) mmax = std::max(mmax, size[c]);
    for (int i = 0; i < mmax; ++i) {
      for (int c = 0; c < cols; ++c) coef[c] = i < size[c] ? S[c][i] : 0.0;
      RF_CUDA(cudaMemcpyAsync(B.alpha, coef.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st));
      RF_K(vec_axpy_cols(B.alpha, false, Vs(i), keep, N, cols, nullptr, st));
    }
  }
  return RFCMP_OK;
}

int compute_scaling(rfcmp_op* op, const rfcmp_op_opts& o, cudaStream_t st) {
  const double k = op->k;
  if (o.scaling == RFCMP_SCALE_K) {
    op->alpha = std::sqrt(k);
    op->beta = 1.0 / std::sqrt(k);
    op->gamma = k;
    return RFCMP_OK;
  }
  if (o.scaling == RFCMP_SCALE_FIXED) {
    op->alpha = o.alpha;
    op->beta = o.beta;
    op->gamma = o.gamma;
    return RFCMP_OK;
  }
  double lxz[2] = {0, 0}, ly = 0;
  const uint64_t sxz[2] = {1, 3}, sy = 2;
  const int64_t N = op->top.ne;
  if (!op->power_vecs) {
    RF_CUDA(dev_malloc(&op->power_vecs, sizeof(double2) * N * 3));
    op->owned.push_back(op->power_vecs);
  }
  const rfcmp_op* from = o.scaling_start;
  const bool warm = from && from->power_vecs && from->top.ne == N && from->top.hash == op->top.hash;
  RF_TRY(power_norms(op, op_XZ, 2, sxz, o.power_steps, o.power_rtol, lxz, warm ? from->power_vecs : nullptr,
                     op->power_vecs, st));
  RF_TRY(power_norms(op, op_Y, 1, &sy, o.power_steps, o.power_rtol, &ly, warm ? from->power_vecs + 2 * N : nullptr,
                     op->power_vecs + 2 * N, st));
  const double nx = lxz[0], nz = lxz[1], ny = ly;
  // alpha^4 = k^2 ||X||, beta^4 = ||Y|| / k^2, gamma = k^2 ||Z|| / alpha^2 (frequency-scaled reading)
  op->alpha = std::pow(k * k * nx, 0.25);
  op->beta = std::pow(ny / (k * k), 0.25);
  op->gamma = k * k / (op->alpha * op->alpha) * nz;
  if (!(op->alpha > 0) || !(op->beta > 0) || !(op->gamma > 0) || !std::isfinite(op->alpha) ||
      !std::isfinite(op->beta) || !std::isfinite(op->gamma))
    return set_error(RFCMP_ERR_CUDA, "power iteration produced a non-positive or non-finite scaling");
  return RFCMP_OK;
}

// ---- geometry upload ----
int upload_geometry(const Topology& T, const std::vector<double>& verts, DeviceGeometry& g, std::vector<void*>& own) {
  const int64_t nc = T.nc, nv = T.nv;
  const double* X = verts.data();
  static const Rule7 R;
  std::vector<double> area(nc), cen(3 * nc), qp(21 * nc);
  std::vector<float> cen_hi(3 * nc), cen_lo(3 * nc), rho(21 * nc), wq(7 * nc), aloc(9 * nc), inv_area(nc);
  for (int64_t c = 0; c < nc; ++c) {
    const double* P[3] = {X + 3 * T.tris[3 * c], X + 3 * T.tris[3 * c + 1], X + 3 * T.tris[3 * c + 2]};
    double u[3], v[3];
    for (int a = 0; a < 3; ++a) {
      u[a] = P[1][a] - P[0][a];
      v[a] = P[2][a] - P[0][a];
    }
    const double cr0 = u[1] * v[2] - u[2] * v[1], cr1 = u[2] * v[0] - u[0] * v[2], cr2 = u[0] * v[1] - u[1] * v[0];
    area[c] = 0.5 * std::sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
    if (!(area[c] > 0.0)) return set_error(RFCMP_ERR_MESH_NOT_MANIFOLD, "cell " + std::to_string(c) + " has zero area");
    for (int a = 0; a < 3; ++a) cen[3 * c + a] = (P[0][a] + P[1][a] + P[2][a]) / 3.0;
    for (int q = 0; q < 7; ++q)
      for (int a = 0; a < 3; ++a)
        qp[21 * c + 3 * q + a] = R.bary[q][0] * P[0][a] + R.bary[q][1] * P[1][a] + R.bary[q][2] * P[2][a];
    for (int a = 0; a < 3; ++a) {
      cen_hi[3 * c + a] = (float)cen[3 * c + a];
      cen_lo[3 * c + a] = (float)(cen[3 * c + a] - (double)cen_hi[3 * c + a]);
    }
    for (int q = 0; q < 7; ++q) {
      for (int a = 0; a < 3; ++a) rho[21 * c + 3 * q + a] = (float)(qp[21 * c + 3 * q + a] - cen[3 * c + a]);
      wq[7 * c + q] = (float)(R.w[q] * area[c]);
    }
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) aloc[9 * c + 3 * i + a] = (float)(P[i][a] - cen[3 * c + a]);
    inv_area[c] = (float)(1.0 / area[c]);
    double rc = 0.0;
    for (int q = 0; q < 7; ++q) {
      double r2 = 0.0;
      for (int a = 0; a < 3; ++a) r2 += (qp[21 * c + 3 * q + a] - cen[3 * c + a]) * (qp[21 * c + 3 * q + a] - cen[3 * c + a]);
      rc = std::max(rc, std::sqrt(r2));
    }
    g.rq_max = std::max(g.rq_max, (float)(rc * 1.001));  // margin over the kernel's FP32 radii
    g.rq_mean += (float)(rc / (double)nc);
  }
  g.nc = (int32_t)nc;
  g.ne = (int32_t)T.ne;
  g.nv = (int32_t)nv;
  g.ldN = padded_ld((int)T.ne);
  g.ldC = padded_ld((int)nc);
  RF_TRY(upload(&g.cen_hi, cen_hi, own));
  RF_TRY(upload(&g.cen_lo, cen_lo, own));
  RF_TRY(upload(&g.rho, rho, own));
  RF_TRY(upload(&g.wq, wq, own));
  RF_TRY(upload(&g.aloc, aloc, own));
  RF_TRY(upload(&g.inv_area, inv_area, own));
  RF_TRY(upload(&g.verts, verts, own));
  RF_TRY(upload(&g.cen64, cen, own));
  RF_TRY(upload(&g.area64, area, own));
  RF_TRY(upload(&g.qp64, qp, own));
  RF_TRY(upload(&g.tris, T.tris, own));
  RF_TRY(upload(&g.cell_edges, T.cell_edges, own));
  RF_TRY(upload(&g.cell_sign, T.cell_sign, own));
  RF_TRY(upload(&g.edge_cells, T.edge_cells, own));
  RF_TRY(upload(&g.edge_loops, T.edge_loops, own));
  RF_TRY(upload(&g.edge_free, T.edge_free, own));
  RF_TRY(upload(&g.vtx_ptr, T.vtx_ptr, own));
  RF_TRY(upload(&g.vtx_edge, T.vtx_edge, own));
  RF_TRY(upload(&g.vtx_sign, T.vtx_sign, own));
  RF_TRY(upload(&g.lap_ptr, T.lap_ptr, own));
  RF_TRY(upload(&g.lap_col, T.lap_col, own));
  RF_TRY(upload(&g.lap_val, T.lap_val, own));
  RF_TRY(upload(&g.near_pairs, T.near_pairs, own));
  g.n_near = (int32_t)(T.near_pairs.size() / 2);
  return RFCMP_OK;
}

// dense inverse of a sparse SPD matrix (CSR on the host), FP32 hi + lo planes
int build_factor(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col, const std::vector<double>& val,
                 int n, bool project, bool multigrid, double tol, std::shared_ptr<DenseFactor>& out,
                 double jacobi_c = 0.8) {
  auto f = std::make_shared<DenseFactor>();
  f->n = n;
  const size_t ld = (size_t)padded_ld(n);
  f->bytes = 2 * ld * (size_t)n * sizeof(float);
  RF_CUDA(dev_malloc(&f->hi, ld * n * sizeof(float)));
  RF_CUDA(dev_malloc(&f->lo, ld * n * sizeof(float)));
  RF_CUDA(cudaMemset(f->hi, 0, ld * n * sizeof(float)));
  RF_CUDA(cudaMemset(f->lo, 0, ld * n * sizeof(float)));
  std::vector<void*> tmp;
  int32_t *dptr = nullptr, *dcol = nullptr;
  double* dval = nullptr;
  int rc = upload(&dptr, ptr, tmp);
  if (rc == RFCMP_OK) rc = upload(&dcol, col, tmp);
  if (rc == RFCMP_OK) rc = upload(&dval, val, tmp);
  if (rc != RFCMP_OK) {
    for (void* p : tmp) dev_free(p);
    return rc;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, 0);
  AmgHierarchy H;
  if (multigrid) {
    std::string err;
    int rc2 = build_amg(ptr, col, val, n, 64, H, err);
    if (rc2 != RFCMP_OK) {
      for (void* p : tmp) dev_free(p);
      return set_error(rc2, err);
    }
  }
  int iters = 0;
  cudaError_t err;
  if (multigrid && project && n >= NS_MIN_CELLS) {
    // Newton-Schulz steps on the tensor cores from one V-cycle; if they do not reach the target
    // (a V-cycle too weak to contract), from a multigrid-PCG solve to NS_START_TOL instead
    const double target = std::max(tol, NS_TARGET), accept = NS_ACCEPT * target;
    double* Xd = nullptr;
    err = dev_malloc(&Xd, sizeof(double) * (size_t)n * padded_ld(n));
    int steps = 0;
    double res = 1.0;
    for (int attempt = 0; attempt < 2 && err == cudaSuccess && !(res <= accept); ++attempt) {
      int it = 0;
      err = dense_inverse_block_cg(dptr, dcol, dval, n, project, &H, NS_START_TOL, attempt == 0 ? 0 : 20000, f->hi,
                                   f->lo, &it, 0, Xd);
      iters += it;
      int st = 0;
      if (err == cudaSuccess)
        err = newton_schulz_pseudo_inverse(dptr, dcol, dval, n, true, Xd, padded_ld(n), NS_MAX_STEPS, target, f->hi,
                                           f->lo, &st, &res, 0);
      steps += st;
    }
    if (Xd) dev_free(Xd);
    f->ns_steps = steps;
    f->ns_residual = res;
    if (err == cudaSuccess && !(res <= accept)) {
      for (void* p : tmp) dev_free(p);
      char msg[128];
      std::snprintf(msg, sizeof(msg), "(Sigma^T Sigma)^+ refinement stalled at residual %.3e after %d steps", res,
                    steps);
      return set_error(RFCMP_ERR_NOT_CONVERGED, msg);
    }
  } else if (!project && !multigrid && n >= NS_MIN_CELLS) {
    // G_ll^{-1}: the P1 mass matrix has the eigenvalues of D^{-1} G_ll in [1/2, 2] (element by
    // element), so X0 = 0.8 D^{-1} leaves I - G_ll X0 a spectral radius of at most 0.6 and
    // Newton-Schulz reaches rounding level in about six steps.  G_l~p^{-1}: G_l~p is strictly
    // diagonally dominant with the off-diagonal row sums below 0.8 of the diagonal, so
    // X0 = D^{-1} (jacobi_c = 1) leaves a spectral radius below 0.8.  Block CG is the fallback
    const double target = std::max(tol, NS_TARGET), accept = NS_ACCEPT * target;
    double* Xd = nullptr;
    err = dev_malloc(&Xd, sizeof(double) * (size_t)n * padded_ld(n));
    int steps = 0;
    double res = 1.0;
    if (err == cudaSuccess) err = jacobi_start(dptr, dcol, dval, n, jacobi_c, Xd, padded_ld(n), 0);
    if (err == cudaSuccess)
      err = newton_schulz_pseudo_inverse(dptr, dcol, dval, n, false, Xd, padded_ld(n), NS_MAX_STEPS, target, f->hi,
                                         f->lo, &steps, &res, 0);
    if (Xd) dev_free(Xd);
    f->ns_steps = steps;
    f->ns_residual = res;
    if (err == cudaSuccess && !(res <= accept))
      err = dense_inverse_block_cg(dptr, dcol, dval, n, project, nullptr, tol, 20000, f->hi, f->lo, &iters, 0);
  } else {
    err = dense_inverse_block_cg(dptr, dcol, dval, n, project, multigrid ? &H : nullptr, tol, 20000, f->hi, f->lo,
                                 &iters, 0);
  }
  cudaEventRecord(e1, 0);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (void* p : tmp) dev_free(p);
  if (err != cudaSuccess) return set_error(RFCMP_ERR_CUDA, std::string("dense inverse: ") + cudaGetErrorString(err));
  f->iterations = iters;
  f->ms = ms;
  out = f;
  return RFCMP_OK;
}

int check_device(int device) {
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0)
    return set_error(RFCMP_ERR_NO_DEVICE, "no CUDA device visible");
  if (device < 0 || device >= count) return set_error(RFCMP_ERR_INVALID_ARG, "device ordinal out of range");
  cudaDeviceProp p;
  RF_CUDA(cudaGetDeviceProperties(&p, device));
  if (p.major != 10 || p.minor != 3)
    return set_error(RFCMP_ERR_NO_DEVICE, std::string("device is sm_") + std::to_string(p.major) +
                                              std::to_string(p.minor) + ", this library is built for sm_103a");
  return RFCMP_OK;
}

}  // namespace

namespace rfcmp {
bool op_ta_view(const rfcmp_op* op, OpTaView* out) {
  if (!op || !out || !op->TA) return false;
  out->TA = op->TA;
  out->n = (int)op->top.ne;
  out->device = op->ctx->device;
  return true;
}

bool op_dense_view(rfcmp_op* op, OpDenseView* out) {
  if (!op || !out || !op->TA || !op->V) return false;
  out->TA = op->TA;
  out->V = op->V;
  out->n = (int)op->top.ne;
  out->nc = (int)op->top.nc;
  out->ldN = op->ldN;
  out->ldC = op->ldC;
  out->device = op->ctx->device;
  out->top = &op->top;
  out->verts = op->verts.data();
  out->ctx_bytes = &op->ctx->bytes;
  out->ctx_live = &op->ctx->live_ops;
  out->budget = op->ctx->budget;
  return true;
}
}  // namespace rfcmp

// ============================================================================ C ABI
extern "C" {

int rfcmp_launch_count(uint64_t* out) {
  if (!out) return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  *out = launches_assembly() + launches_exact() + launches_factor() + launches_gemm() + launches_gemv_stream() +
         launches_linalg() + launches_krylov() + launches_hmatrix();
  return RFCMP_OK;
}

int rfcmp_pool_stats(uint64_t* used, uint64_t* used_high, uint64_t* reserved, uint64_t* reserved_high) {
  int dev = 0;
  cudaMemPool_t pool;
  RF_CUDA(cudaGetDevice(&dev));
  RF_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t v = 0;
  if (used) RF_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, used));
  if (used_high) RF_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, used_high));
  if (reserved) RF_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, reserved));
  if (reserved_high) RF_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemHigh, reserved_high));
  (void)v;
  return RFCMP_OK;
}

int rfcmp_pool_trim(void) {
  dev_pool_trim();
  RF_CUDA(cudaGetLastError());
  return RFCMP_OK;
}

int rfcmp_pool_reset_high(void) {
  int dev = 0;
  cudaMemPool_t pool;
  RF_CUDA(cudaGetDevice(&dev));
  RF_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t zero = 0;
  RF_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
  RF_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReservedMemHigh, &zero));
  return RFCMP_OK;
}

int rfcmp_set_solve_graphs(int enable) {
  const int prev = solve_graphs_enabled() ? 1 : 0;
  g_solve_graphs.store(enable ? 1 : 0);
  return prev;
}

const char* rfcmp_strerror(int st) {
  switch (st) {
    case RFCMP_OK: return "ok";
    case RFCMP_ERR_INVALID_ARG: return "invalid argument";
    case RFCMP_ERR_MESH_NOT_MANIFOLD: return "mesh is not a closed 2-manifold";
    case RFCMP_ERR_MESH_ORIENTATION: return "mesh is not consistently oriented";
    case RFCMP_ERR_OUT_OF_BUDGET: return "HBM budget exceeded";
    case RFCMP_ERR_CUDA: return "CUDA error";
    case RFCMP_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case RFCMP_ERR_NOT_CONVERGED: return "solve did not converge";
    case RFCMP_ERR_NO_DEVICE: return "no usable sm_103 device";
    default: return "unknown status";
  }
}

const char* rfcmp_last_error(void) { return g_last_error.c_str(); }

int rfcmp_profile_enable(int enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_resolve_locked();
  g_prof.clear();
  ++g_prof_generation;
  prof_dev_clear();
  g_prof_on.store(enable != 0);
  return RFCMP_OK;
}

int rfcmp_profile_read(rfcmp_profile_entry* out, int max_entries, int* n_entries) {
  if (!n_entries || (max_entries > 0 && !out)) return set_error(RFCMP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_resolve_locked();
  // launches captured into graphs: the device accumulators (after the device has drained)
  static DevProfFamily dev[PROF_DEV_FAMILIES];
  std::memset(dev, 0, sizeof(dev));
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpyFromSymbol(dev, g_prof_dev, sizeof(dev)) != cudaSuccess) {
    (void)cudaGetLastError();
    std::memset(dev, 0, sizeof(dev));
  }
  *n_entries = (int)g_prof.size();
  for (int i = 0; i < max_entries && i < (int)g_prof.size(); ++i) {
    std::memset(&out[i], 0, sizeof(out[i]));
    std::strncpy(out[i].name, g_prof[i].name.c_str(), sizeof(out[i].name) - 1);
    const DevProfFamily d = i < PROF_DEV_FAMILIES ? dev[i] : DevProfFamily{};
    out[i].launches = g_prof[i].launches + (int64_t)d.launches;
    out[i].total_ms = g_prof[i].ms + 1e-6 * (double)d.ns;
    out[i].bytes = g_prof[i].bytes + d.bytes;
    out[i].flops = g_prof[i].flops + d.flops;
  }
  return RFCMP_OK;
}

void rfcmp_op_opts_default(rfcmp_op_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->scaling = RFCMP_SCALE_POWER;
  o->power_steps = 30;
  o->alpha = o->beta = o->gamma = 1.0;
  o->factor_tol = 1e-13;
  o->power_rtol = 1e-3;
  o->scaling_start = nullptr;
}

void rfcmp_solve_opts_default(rfcmp_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-6;
  o->max_iter = 2000;
  o->max_refine = 24;
  o->inner_tol = 1e-4;
  o->precision = RFCMP_PREC_MIXED;
}

int rfcmp_ctx_create(int device, uint64_t budget, rfcmp_ctx** out) {
  if (!out) return set_error(RFCMP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  RF_TRY(check_device(device));
  RF_CUDA(cudaSetDevice(device));
  RF_CUDA(dev_free(0));
  auto* c = new rfcmp_ctx();
  c->device = device;
  c->budget = budget;
  *out = c;
  return RFCMP_OK;
}

int rfcmp_ctx_destroy(rfcmp_ctx* ctx) {
  if (!ctx) return RFCMP_OK;
  if (ctx->live_ops.load() != 0) return set_error(RFCMP_ERR_INVALID_ARG, "context still has live ops");
  cudaSetDevice(ctx->device);
  delete ctx;
  dev_pool_trim();  // hand the memory the context's buffers left in the pool back to the driver
  return RFCMP_OK;
}

int rfcmp_ctx_clear_cache(rfcmp_ctx* ctx) {
  if (!ctx) return set_error(RFCMP_ERR_INVALID_ARG, "ctx is NULL");
  std::lock_guard<std::mutex> lk(ctx->mu);
  for (auto& kv : ctx->lplus_cache)
    if (kv.second.use_count() == 1) ctx->bytes -= kv.second->bytes;
  for (auto& kv : ctx->gll_cache)
    if (kv.second.use_count() == 1) ctx->bytes -= kv.second->bytes;
  for (auto& kv : ctx->gtp_cache)
    if (kv.second.use_count() == 1) ctx->bytes -= kv.second->bytes;
  ctx->lplus_cache.clear();
  ctx->gll_cache.clear();
  ctx->gtp_cache.clear();
  ctx->mesh_cache.clear();
  return RFCMP_OK;
}

uint64_t rfcmp_ctx_bytes_in_use(const rfcmp_ctx* ctx) { return ctx ? ctx->bytes.load() : 0; }

int rfcmp_op_create(rfcmp_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t nc, double k,
                    const rfcmp_op_opts* opts_in, rfcmp_op** out) {
  if (!ctx || !verts || !tris || !out) return set_error(RFCMP_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (!(k > 0.0) || !std::isfinite(k)) return set_error(RFCMP_ERR_INVALID_ARG, "k must be positive and finite");
  rfcmp_op_opts o;
  rfcmp_op_opts_default(&o);
  if (opts_in) o = *opts_in;
  for (int i = 0; i < 7; ++i)
    if (o.reserved[i] != 0) return set_error(RFCMP_ERR_INVALID_ARG, "opts.reserved must be zero");
  if (o.outer != RFCMP_OUTER_SIGMA && o.outer != RFCMP_OUTER_GSIGMA)
    return set_error(RFCMP_ERR_INVALID_ARG, "opts.outer must be RFCMP_OUTER_SIGMA or RFCMP_OUTER_GSIGMA");
  if (o.scaling < 0 || o.scaling > 2 || o.power_steps < 1 || !(o.factor_tol > 0.0) || !(o.power_rtol >= 0.0))
    return set_error(RFCMP_ERR_INVALID_ARG, "invalid op options");
  if (o.scaling == RFCMP_SCALE_FIXED && !(o.alpha > 0 && o.beta > 0 && o.gamma > 0))
    return set_error(RFCMP_ERR_INVALID_ARG, "fixed scaling needs positive alpha, beta, gamma");
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(verts[i])) return set_error(RFCMP_ERR_INVALID_ARG, "non-finite vertex coordinate");
  {
    // the far-pair kernel reduces k R by multiples of pi/2 whose leading part (8 bits) times the
    // multiple stays exact below 2^16 multiples, k R < 1.029e5; R is at most the diagonal of the
    // vertices' bounding box
    double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
    for (int64_t i = 0; i < nv; ++i)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], verts[3 * i + a]);
        hi[a] = std::max(hi[a], verts[3 * i + a]);
      }
    double d2 = 0.0;
    for (int a = 0; a < 3 && nv > 0; ++a) d2 += (hi[a] - lo[a]) * (hi[a] - lo[a]);
    if (k * std::sqrt(d2) > RFCMP_MAX_K_EXTENT) {
      char msg[160];
      snprintf(msg, sizeof msg, "k times the mesh extent (%.4g) exceeds %.4g, the phase range of the FP32 assembly",
               k * std::sqrt(d2), (double)RFCMP_MAX_K_EXTENT);
      return set_error(RFCMP_ERR_INVALID_ARG, msg);
    }
  }
  RF_CUDA(cudaSetDevice(ctx->device));
  auto op = std::make_unique<rfcmp_op>();
  op->ctx = ctx;
  op->k = k;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    op->plan = ctx->plan;
  }
  std::string err;
  int rc = RFCMP_OK;
  // topology and device geometry: from the context's mesh cache when the same mesh (connectivity
  // and coordinates, compared exactly) was seen before
  uint64_t mesh_key = mix((uint64_t)nc, (uint64_t)nv);
  for (int64_t i = 0; i < 3 * nc; ++i) mesh_key = mix(mesh_key, (uint64_t)(uint32_t)tris[i]);
  for (int64_t i = 0; i < 3 * nv; ++i) {
    uint64_t b;
    std::memcpy(&b, &verts[i], 8);
    mesh_key = mix(mesh_key, b);
  }
  std::shared_ptr<MeshEntry> me;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->mesh_cache.find(mesh_key);
    if (it != ctx->mesh_cache.end() && it->second->top.nc == nc && it->second->top.nv_mesh == nv &&
        std::equal(tris, tris + 3 * nc, it->second->top.tris.begin()) &&
        std::equal(verts, verts + 3 * nv, it->second->verts.begin()))
      me = it->second;
  }
  if (!me) {
    auto fresh = std::make_shared<MeshEntry>();
    rc = build_topology(tris, nc, nv, fresh->top, err);
    if (rc != RFCMP_OK) return set_error(rc, err);
    if (fresh->top.ne >= (1ll << 31) / 1 || (double)fresh->top.ne * fresh->top.ne > 9e18)
      return set_error(RFCMP_ERR_INVALID_ARG, "mesh too large");
    fresh->verts.assign(verts, verts + 3 * nv);
    RF_TRY(upload_geometry(fresh->top, fresh->verts, fresh->g, fresh->owned));
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->mesh_cache.size() >= 16)  // keep the cache small: drop entries no operator holds
      for (auto it = ctx->mesh_cache.begin(); it != ctx->mesh_cache.end();)
        it = it->second.use_count() == 1 ? ctx->mesh_cache.erase(it) : std::next(it);
    ctx->mesh_cache[mesh_key] = fresh;
    me = fresh;
  }
  op->mesh = me;
  op->top = me->top;
  op->verts = me->verts;
  op->g = me->g;
  if (op->top.nv == 0)
    return set_error(RFCMP_ERR_MESH_NOT_MANIFOLD, "the open surface has no interior vertex (no loop function)");
  if (o.outer == RFCMP_OUTER_GSIGMA && op->top.boundaries > 0)
    return set_error(RFCMP_ERR_INVALID_ARG,
                     "the theory variant P_gSigma needs a closed surface (its dual functions are defined there)");
  const int N = (int)op->top.ne, C = (int)op->top.nc, NV = (int)op->top.nv;
  op->ldN = padded_ld(N);
  op->ldC = padded_ld(C);
  const uint64_t mat_bytes = (uint64_t)op->ldN * N * 8 + (uint64_t)op->ldC * C * 8;
  // factor cache lookups
  uint64_t geo_hash = op->top.hash;
  for (int64_t i = 0; i < 3 * nv; ++i) {
    uint64_t b;
    std::memcpy(&b, &verts[i], 8);
    geo_hash = mix(geo_hash, b);
  }
  std::shared_ptr<DenseFactor> lp, gl, gt;
  const bool gsigma = o.outer == RFCMP_OUTER_GSIGMA;
  op->outer = o.outer;
  std::unique_lock<std::mutex> build_lock(ctx->build_mu);
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto a = ctx->lplus_cache.find(op->top.hash);
    if (a != ctx->lplus_cache.end()) lp = a->second;
    auto b = ctx->gll_cache.find(geo_hash);
    if (b != ctx->gll_cache.end()) gl = b->second;
    auto c = ctx->gtp_cache.find(op->top.hash);
    if (gsigma && c != ctx->gtp_cache.end()) gt = c->second;
  }
  uint64_t need = mat_bytes;
  if (!lp) need += 2ull * padded_ld(C) * C * 4;
  if (!gl) need += 2ull * padded_ld(NV) * NV * 4;
  if (gsigma && !gt) need += 2ull * padded_ld(C) * C * 4;
  if (ctx->budget && ctx->bytes.load() + need > ctx->budget)
    return set_error(RFCMP_ERR_OUT_OF_BUDGET, "op needs " + std::to_string(need) + " bytes, budget has " +
                                                  std::to_string(ctx->budget - std::min(ctx->budget, ctx->bytes.load())));
  // topology factors
  op->info.ms_factors = 0.0;
  if (!lp) {
    RF_TRY(build_factor(op->top.lap_ptr, op->top.lap_col, op->top.lap_val, C, true, true, o.factor_tol, lp));
    op->info.ms_factors += lp->ms;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->lplus_cache[op->top.hash] = lp;
    ctx->bytes += lp->bytes;
  }
  if (!gl) {
    std::vector<int32_t> mp, mc;
    std::vector<double> mv;
    mass_matrix_csr(op->top, op->verts.data(), mp, mc, mv);
    RF_TRY(build_factor(mp, mc, mv, NV, false, false, o.factor_tol, gl));
    op->info.ms_factors += gl->ms;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->gll_cache[geo_hash] = gl;
    ctx->bytes += gl->bytes;
  }
  if (gsigma && !gt) {
    std::vector<int32_t> gp, gc;
    std::vector<double> gv;
    gtp_matrix_csr(op->top, gp, gc, gv);
    RF_TRY(build_factor(gp, gc, gv, C, false, false, o.factor_tol, gt, 1.0));
    op->info.ms_factors += gt->ms;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->gtp_cache[op->top.hash] = gt;
    ctx->bytes += gt->bytes;
  }
  op->lplus = lp;
  op->gll = gl;
  op->gtp = gt;
  build_lock.unlock();
  // The pool keeps freed memory mapped; after a factor build of tens of GB the work arrays would
  // stay reserved beside matrices of tens of GB more, so a large operator hands them back first.
  if (mat_bytes > (32ull << 30)) dev_pool_trim();
  op->info.factor_iterations_lplus = lp->iterations;
  op->info.factor_iterations_gll = gl->iterations;
  // assembly
  RF_CUDA(dev_malloc(&op->TA, (size_t)op->ldN * N * sizeof(float2)));
  op->owned.push_back(op->TA);
  RF_CUDA(dev_malloc(&op->V, (size_t)op->ldC * C * sizeof(float2)));
  op->owned.push_back(op->V);
  op->bytes = mat_bytes;
  rfcmp_op* raw = op.get();
  cudaEvent_t e0, e1, e2;
  RF_CUDA(cudaEventCreate(&e0));
  RF_CUDA(cudaEventCreate(&e1));
  RF_CUDA(cudaEventCreate(&e2));
  RF_CUDA(cudaEventRecord(e0, 0));
  RF_CUDA(cudaMemsetAsync(op->TA, 0, (size_t)op->ldN * N * sizeof(float2), 0));
  RF_CUDA(cudaMemsetAsync(op->V, 0, (size_t)op->ldC * C * sizeof(float2), 0));
  RF_K(launch_assemble_far(op->g, (float)k, op->TA, op->V, op->plan.far_min_blocks, 0));
  RF_K(launch_assemble_near(op->g, k, op->TA, op->V, 0));
  RF_K(launch_mirror_upper(op->TA, N, op->ldN, 0));
  RF_CUDA(cudaEventRecord(e1, 0));
  rc = compute_scaling(raw, o, 0);
  RF_CUDA(cudaEventRecord(e2, 0));
  RF_CUDA(cudaEventSynchronize(e2));
  float ms_a = 0.f, ms_s = 0.f;
  cudaEventElapsedTime(&ms_a, e0, e1);
  cudaEventElapsedTime(&ms_s, e1, e2);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  if (rc != RFCMP_OK) return rc;
  RF_CUDA(cudaGetLastError());
  ctx->bytes += op->bytes;
  ctx->live_ops++;
  op->info.n_edges = N;
  op->info.n_vertices = NV;
  op->info.n_cells = C;
  op->info.genus = op->top.genus;
  op->info.boundaries = op->top.boundaries;
  op->info.k = k;
  op->info.alpha = op->alpha;
  op->info.beta = op->beta;
  op->info.gamma = op->gamma;
  op->info.ms_assembly = ms_a;
  op->info.ms_scaling = ms_s;
  *out = op.release();
  return RFCMP_OK;
}

int rfcmp_op_info_get(const rfcmp_op* op, rfcmp_op_info* out) {
  if (!op || !out) return set_error(RFCMP_ERR_INVALID_ARG, "NULL argument");
  *out = op->info;
  uint64_t ws = 0;
  if (op->ws) ws += (uint64_t)op->ws->cols * (5 * op->top.ne + 8 * op->top.nc + 2 * op->top.nv) * 16;
  if (op->sb) ws += (uint64_t)op->sb->cols * 8 * op->top.ne * 16;
  out->device_bytes = op->bytes + ws;
  return RFCMP_OK;
}

int rfcmp_op_trim(rfcmp_op* op) {
  if (!op) return set_error(RFCMP_ERR_INVALID_ARG, "NULL op");
  RF_CUDA(cudaSetDevice(op->ctx->device));
  RF_TRY(drain_streams(op));  // frees are queued behind every stream op was used on
  for (void* p : op->lazy) dev_free(p);
  op->lazy.clear();
  op->ta_planes = CplxPlanes();
  op->v_planes = CplxPlanes();
  op->ta_digits = ExactOperand();
  op->v_digits = ExactOperand();
  op->ctx->bytes -= op->lazy_bytes;
  op->bytes -= op->lazy_bytes;
  op->lazy_bytes = 0;
  op->ws.reset();
  op->sb.reset();
  return RFCMP_OK;
}

int rfcmp_op_destroy(rfcmp_op* op) {
  if (!op) return RFCMP_OK;
  rfcmp_ctx* ctx = op->ctx;
  cudaSetDevice(ctx->device);
  drain_streams(op);  // frees are queued behind every stream op was used on
  ctx->bytes -= op->bytes;
  ctx->live_ops--;
  delete op;
  return RFCMP_OK;
}

int rfcmp_op_export(const rfcmp_op* op, int which, void* dst, uint64_t dst_bytes, void* stream) {
  if (!op || !dst) return set_error(RFCMP_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = (int)op->top.ne, C = (int)op->top.nc, NV = (int)op->top.nv;
  if (which == 0 || which == 1) {
    const int n = which == 0 ? N : C;
    const int ld = which == 0 ? op->ldN : op->ldC;
    if (dst_bytes < (uint64_t)n * n * 8) return set_error(RFCMP_ERR_INVALID_ARG, "destination too small");
    const float2* M = which == 0 ? op->TA : op->V;
    RF_CUDA(cudaMemcpy2DAsync(dst, (size_t)n * 8, M, (size_t)ld * 8, (size_t)n * 8, n, cudaMemcpyDeviceToDevice, st));
    return RFCMP_OK;
  }
  if (which == 4 && !op->gtp) return set_error(RFCMP_ERR_INVALID_ARG, "op has no G_l~p factor");
  if (which == 2 || which == 3 || which == 4) {
    const DenseFactor& f = which == 2 ? *op->lplus : (which == 3 ? *op->gll : *op->gtp);
    const int n = which == 3 ? NV : C;
    if (dst_bytes < (uint64_t)n * n * 8) return set_error(RFCMP_ERR_INVALID_ARG, "destination too small");
    // hi and lo planes side by side: first n*n floats hi, then n*n floats lo
    float* d = static_cast<float*>(dst);
    const int ld = padded_ld(n);
    RF_CUDA(cudaMemcpy2DAsync(d, (size_t)n * 4, f.hi, (size_t)ld * 4, (size_t)n * 4, n, cudaMemcpyDeviceToDevice, st));
    RF_CUDA(cudaMemcpy2DAsync(d + (size_t)n * n, (size_t)n * 4, f.lo, (size_t)ld * 4, (size_t)n * 4, n,
                              cudaMemcpyDeviceToDevice, st));
    return RFCMP_OK;
  }
  return set_error(RFCMP_ERR_INVALID_ARG, "unknown matrix id");
}

int rfcmp_op_edges(const rfcmp_op* op, int32_t* edge_verts, int32_t* edge_cells) {
  if (!op || !edge_verts || !edge_cells) return set_error(RFCMP_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(edge_verts, op->top.edge_verts.data(), op->top.edge_verts.size() * 4);
  std::memcpy(edge_cells, op->top.edge_cells.data(), op->top.edge_cells.size() * 4);
  return RFCMP_OK;
}

int rfcmp_rhs_planewave(rfcmp_op* op, const double* khat, const double* pol, int64_t nrhs, rfcmp_c128* e,
                        void* stream) {
  if (!op || !khat || !pol || !e || nrhs <= 0 || nrhs > 65535)
    return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  double* d = nullptr;
  RF_CUDA(cudaMallocAsync(&d, sizeof(double) * 6 * nrhs, st));
  RF_CUDA(cudaMemcpyAsync(d, khat, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, st));
  RF_CUDA(cudaMemcpyAsync(d + 3 * nrhs, pol, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, st));
  RF_K(launch_rhs_planewave(op->g, op->k, d, d + 3 * nrhs, (int)nrhs, reinterpret_cast<double2*>(e), st));
  RF_CUDA(cudaFreeAsync(d, st));
  RF_CUDA(cudaStreamSynchronize(st));
  return RFCMP_OK;
}

int rfcmp_rhs_voltage_gap(rfcmp_op* op, const double* origin, const double* normal, rfcmp_c128 voltage, rfcmp_c128* e,
                          void* stream) {
  if (!op || !origin || !normal || !e) return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  const double nn = normal[0] * normal[0] + normal[1] * normal[1] + normal[2] * normal[2];
  if (!(nn > 0.0) || !std::isfinite(nn) || !std::isfinite(origin[0] + origin[1] + origin[2]))
    return set_error(RFCMP_ERR_INVALID_ARG, "the gap plane needs a finite origin and a nonzero normal");
  cudaStream_t st = (cudaStream_t)stream;
  RF_TRY(order_stream(op, st));
  RF_K(launch_rhs_voltage_gap(op->g, origin, normal, make_double2(voltage.re, voltage.im),
                              reinterpret_cast<double2*>(e), st));
  return RFCMP_OK;
}

int rfcmp_apply(rfcmp_op* op, int which, const rfcmp_c128* xin, rfcmp_c128* yout, int64_t nrhs, void* stream) {
  if (!op || !xin || !yout || nrhs <= 0 || nrhs > 4096) return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  const double2* x = reinterpret_cast<const double2*>(xin);
  double2* y = reinterpret_cast<double2*>(yout);
  const int nr = (int)nrhs;
  const int N = (int)op->top.ne, C = (int)op->top.nc;
  const double k = op->k;
  const GemvMode m = GEMV_FF;
  RF_TRY(ensure_workspace(op, nr));
  if (which == RFCMP_APPLY_A_INNER && nr >= plan_mrhs(op)) RF_TRY(ensure_planes(op, 0));
  if (which != RFCMP_APPLY_A_INNER && nr >= plan_exact(op)) RF_TRY(ensure_digits(op, 0));
  RF_TRY(order_stream(op, st));
  Workspace& W = *op->ws;
  switch (which) {
    case RFCMP_APPLY_T_A:
      RF_TRY(prod_c(op, true, x, y, nr, false, c2(1, 0), false, m, st));
      return nr >= plan_exact(op) ? check_tensor_core_waits(op, st) : RFCMP_OK;
    case RFCMP_APPLY_T_PHI: {
      RF_K(sigma_t(op->g, x, W.s, nr, st));
      RF_TRY(prod_c(op, false, W.s, W.w, nr, false, c2(1, 0), false, m, st));
      EdgeCombo c;
      c.zs = W.w;
      c.b = c2(1, 0);
      RF_K(edge_combo(op->g, c, y, nr, st));
      return nr >= plan_exact(op) ? check_tensor_core_waits(op, st) : RFCMP_OK;
    }
    case RFCMP_APPLY_T:
    case RFCMP_APPLY_T_ADJ: {
      const bool adj = which == RFCMP_APPLY_T_ADJ;
      RF_K(sigma_t(op->g, x, W.s, nr, st));
      RF_TRY(prod_c(op, false, W.s, W.w, nr, adj, c2(1, 0), false, m, st));
      RF_TRY(prod_c(op, true, x, W.u, nr, adj, c2(1, 0), false, m, st));
      // T x = i k T_A x - (i/k) Sigma V Sigma^T x ; T^H x = -i k conj(T_A) x + (i/k) Sigma conj(V) Sigma^T x
      EdgeCombo c;
      c.x = W.u;
      c.a = c2(0.0, adj ? -k : k);
      c.zs = W.w;
      c.b = c2(0.0, adj ? 1.0 / k : -1.0 / k);
      RF_K(edge_combo(op->g, c, y, nr, st));
      return nr >= plan_exact(op) ? check_tensor_core_waits(op, st) : RFCMP_OK;
    }
    case RFCMP_APPLY_A:
      RF_TRY(apply_A(op, x, y, nr, m, st));
      return nr >= plan_exact(op) ? check_tensor_core_waits(op, st) : RFCMP_OK;
    case RFCMP_APPLY_A_INNER:
      RF_TRY(apply_A(op, x, y, nr, GEMV_F32, st));
      return nr >= plan_mrhs(op) ? check_tensor_core_waits(op, st) : RFCMP_OK;
    default:
      return set_error(RFCMP_ERR_INVALID_ARG, "unknown operator id");
  }
}

void rfcmp_plan_default(rfcmp_plan* plan) {
  if (plan) std::memset(plan, 0, sizeof(*plan));
}

namespace {
int check_plan(const rfcmp_plan& p) {
  for (int i = 0; i < 2; ++i)
    if (p.reserved[i] != 0) return set_error(RFCMP_ERR_INVALID_ARG, "plan.reserved must be zero");
  if (p.exact_min < 0 || p.exact_min > 65536) return set_error(RFCMP_ERR_INVALID_ARG, "plan.exact_min out of range");
  if (p.mrhs_min < 0 || p.mrhs_min > 65536) return set_error(RFCMP_ERR_INVALID_ARG, "plan.mrhs_min out of range");
  if (p.gemm_bn != 0 && p.gemm_bn != 32 && p.gemm_bn != 64 && p.gemm_bn != 128)
    return set_error(RFCMP_ERR_INVALID_ARG, "plan.gemm_bn must be 0, 32, 64 or 128");
  if (p.gemv_chunk != 0 && (p.gemv_chunk % 256 != 0 || p.gemv_chunk < 256 || p.gemv_chunk > 8192))
    return set_error(RFCMP_ERR_INVALID_ARG, "plan.gemv_chunk must be a multiple of 256 in [256, 8192]");
  if (p.gemv_ctas_per_sm < 0 || p.gemv_ctas_per_sm > 8)
    return set_error(RFCMP_ERR_INVALID_ARG, "plan.gemv_ctas_per_sm out of range");
  if (p.far_min_blocks < 0 || p.far_min_blocks > 4)
    return set_error(RFCMP_ERR_INVALID_ARG, "plan.far_min_blocks must be 0..4");
  return RFCMP_OK;
}
}  // namespace

int rfcmp_ctx_set_plan(rfcmp_ctx* ctx, const rfcmp_plan* plan) {
  if (!ctx) return set_error(RFCMP_ERR_INVALID_ARG, "NULL context");
  rfcmp_plan p{};
  if (plan) p = *plan;
  RF_TRY(check_plan(p));
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->plan = p;
  return RFCMP_OK;
}

int rfcmp_op_set_plan(rfcmp_op* op, const rfcmp_plan* plan) {
  if (!op) return set_error(RFCMP_ERR_INVALID_ARG, "NULL op");
  rfcmp_plan p{};
  if (plan) p = *plan;
  RF_TRY(check_plan(p));
  op->plan = p;
  if (op->ws) plan_to_scratch(op);
  return RFCMP_OK;
}

int rfcmp_op_get_plan(const rfcmp_op* op, rfcmp_plan* out) {
  if (!op || !out) return set_error(RFCMP_ERR_INVALID_ARG, "NULL argument");
  *out = op->plan;
  return RFCMP_OK;
}

int rfcmp_precondition(rfcmp_op* op, int which, const rfcmp_c128* xin, rfcmp_c128* yout, int64_t nrhs, void* stream) {
  if (!op || !xin || !yout || nrhs <= 0 || nrhs > 4096) return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  const double2* x = reinterpret_cast<const double2*>(xin);
  double2* y = reinterpret_cast<double2*>(yout);
  const int nr = (int)nrhs;
  const GemvMode m = GEMV_FF;
  RF_TRY(ensure_workspace(op, nr));
  if (nr >= plan_exact(op)) RF_TRY(ensure_digits(op, 0));
  RF_TRY(order_stream(op, st));
  Workspace& W = *op->ws;
  const double a = op->alpha, b = op->beta, gm = op->gamma;
  switch (which) {
    case RFCMP_PREC_P_O:
      return apply_Po(op, x, y, nr, false, m, st);
    case RFCMP_PREC_P_O_ADJ:
      return apply_Po(op, x, y, nr, true, m, st);
    case RFCMP_PREC_P_SIGMA:
    case RFCMP_PREC_P_LAMBDAH: {
      RF_TRY(star_coeff(op, x, W.s, W.z, nr, m, st));
      EdgeCombo c;
      c.zs = W.z;
      if (which == RFCMP_PREC_P_SIGMA) {
        c.b = c2(1, 0);
      } else {
        c.x = x;
        c.a = c2(1, 0);
        c.b = c2(-1, 0);
      }
      RF_K(edge_combo(op->g, c, y, nr, st));
      return RFCMP_OK;
    }
    case RFCMP_PREC_P_GSIGMA: {  // Sigma L^+ G^{-1} Sigma^T x
      if (!op->gtp) return set_error(RFCMP_ERR_INVALID_ARG, "op was created without outer = RFCMP_OUTER_GSIGMA");
      RF_K(sigma_t(op->g, x, W.s, nr, st));
      RF_TRY(prod_r(op, *op->gtp, W.s, W.g1, nr, 1.0, false, m, st));
      RF_TRY(prod_r(op, *op->lplus, W.g1, W.g2, nr, 1.0, false, m, st));
      EdgeCombo c;
      c.zs = W.g2;
      c.b = c2(1, 0);
      RF_K(edge_combo(op->g, c, y, nr, st));
      return nr >= plan_exact(op) ? check_tensor_core_waits(op, st) : RFCMP_OK;
    }
    case RFCMP_PREC_P_M: {
      const int C = (int)op->top.nc, NV = (int)op->top.nv;
      RF_TRY(star_coeff(op, x, W.s, W.zu, nr, m, st));
      RF_K(star_middle(op->g, W.zu, nullptr, 1.0, W.q0, nr, W.mean, st));
      RF_TRY(prod_r(op, *op->lplus, W.q0, W.q, nr, 1.0 / (b * b), false, m, st));
      RF_K(lambda_t(op->g, x, W.t, nr, st));
      RF_TRY(prod_r(op, *op->gll, W.t, W.tg, nr, 1.0, false, m, st));
      EdgeCombo c;
      c.zl = W.tg;
      c.c = c2(1.0 / (a * a), 0.0);
      c.x = x;
      c.a = c2(1.0 / gm, 0.0);
      c.zs = W.zu;
      c.b = c2(-1.0 / gm, 0.0);
      c.zs2 = W.q;
      c.d = c2(1.0, 0.0);
      RF_K(edge_combo(op->g, c, y, nr, st));
      return nr >= plan_exact(op) ? check_tensor_core_waits(op, st) : RFCMP_OK;
    }
    default:
      return set_error(RFCMP_ERR_INVALID_ARG, "unknown preconditioner id");
  }
}

}  // extern "C"

// ---------------------------------------------------------------- the solve
namespace {

KrylovView krylov_view(rfcmp_op* op, SolveBuffers& B, int nr) {
  KrylovView K;
  K.ctl = B.ctl;
  K.bb = B.bb;
  K.rr = B.rr;
  K.rho = B.rho;
  K.r0 = B.r0;
  K.alpha = B.alpha;
  K.beta = B.beta;
  K.res = B.res;
  K.active = B.active;
  K.conv = B.conv;
  K.iters = B.iters;
  K.sweeps = B.sweeps;
  K.part = B.part;
  K.ticket = B.ticket;
  K.member = B.member;
  K.n = op->top.ne;
  K.nr = nr;
  K.G = krylov_blocks_per_column(op->top.ne);
  return K;
}

// one CG iteration of the inner solve on the active columns (Sec. 4: CG on A d = r)
int cg_iteration(rfcmp_op* op, SolveBuffers& B, const KrylovView& K, int nr, GemvMode m, cudaStream_t st) {
  RF_TRY(apply_A(op, B.p, B.Ap, nr, m, st));
  RF_K(krylov_cg_pap(K, B.p, B.Ap, st));
  RF_K(krylov_cg_update(K, B.p, B.Ap, B.d, B.rin, st));
  RF_K(krylov_cg_direction(K, B.rin, B.p, st));
  return RFCMP_OK;
}

// the end of a sweep: i += d, r = b - A i (float-float accurate), norms and the next decision
int refine_step(rfcmp_op* op, SolveBuffers& B, const KrylovView& K, int nr, cudaStream_t st) {
  RF_K(krylov_add(K, B.d, B.i, st));
  RF_TRY(apply_A(op, B.i, B.tmp, nr, GEMV_FF, st));
  RF_K(krylov_refine_residual(K, B.b, B.tmp, B.r, B.i, false, st));
  return RFCMP_OK;
}

int read_ctl(const SolveBuffers& B, KrylovCtl& h, cudaStream_t st) {
  RF_CUDA(cudaMemcpyAsync(&h, B.ctl, sizeof(KrylovCtl), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaStreamSynchronize(st));
  return RFCMP_OK;
}

// Eager driver: the same kernels launched one by one, the host reading the control block after
// every decision (used where graphs are switched off or a capture failed).
// One refinement sweep of the eager driver: the inner CG on the active columns (the host reading
// the device's decision after every iteration), then i += d and the accurate residual.
int eager_sweep(rfcmp_op* op, SolveBuffers& B, const KrylovView& K, int nr, GemvMode inner, int max_iter,
                cudaStream_t st) {
  KrylovCtl h{};
  RF_K(krylov_cg_start(K, B.r, B.d, B.rin, B.p, st));
  for (int pass = 0; pass < max_iter; ++pass) {
    RF_TRY(cg_iteration(op, B, K, nr, inner, st));
    RF_TRY(read_ctl(B, h, st));
    if (h.live == 0 || h.passes >= h.max_passes) break;
  }
  return refine_step(op, B, K, nr, st);
}

int solve_loop_eager(rfcmp_op* op, int nr, GemvMode inner, int max_sweeps, int max_iter, cudaStream_t st) {
  SolveBuffers& B = *op->sb;
  KrylovView K = krylov_view(op, B, nr);
  RF_K(krylov_refine_residual(K, B.b, nullptr, B.r, B.i, true, st));
  KrylovCtl h{};
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    RF_TRY(read_ctl(B, h, st));
    if (!h.go) break;
    RF_TRY(eager_sweep(op, B, K, nr, inner, max_iter, st));
  }
  return RFCMP_OK;
}

// Ends a capture left open by an error path.  The graph it captured into is owned elsewhere (the
// top-level graph by the capture function, a conditional body by its node), so nothing is freed.
struct CaptureGuard {
  cudaStream_t s;
  bool open = true;
  explicit CaptureGuard(cudaStream_t st) : s(st) {}
  ~CaptureGuard() {
    if (!open) return;
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(s, &g);
    (void)cudaGetLastError();
  }
};

// Adds a WHILE node on handle h after what stream s has captured so far and returns its body.
int add_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus stat;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  RF_CUDA(cudaStreamGetCaptureInfo(s, &stat, nullptr, &g, &deps, nullptr, &ndeps));
  if (stat != cudaStreamCaptureStatusActive) return set_error(RFCMP_ERR_CUDA, "capture not active");
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  RF_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &p));
  *body = p.conditional.phGraph_out[0];
  RF_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return RFCMP_OK;
}

bool solve_graph_current(const rfcmp_op* op, int nr, GemvMode inner, int max_sweeps) {
  const SolveGraph* G = op->solve_graph.get();
  if (!G || !G->exec) return false;
  const void* lazy[10] = {op->ta_planes.rh,   op->v_planes.rh,     op->ta_digits.d,  op->v_digits.d,
                          op->lplus->planes.h, op->lplus->digits.d, op->gll->planes.h, op->gll->digits.d,
                          op->gtp ? op->gtp->planes.h : nullptr, op->gtp ? op->gtp->digits.d : nullptr};
  return G->nr == nr && G->mode == (int)inner && G->max_sweeps == max_sweeps && G->ws == op->ws.get() &&
         G->sb == op->sb.get() && G->ws_cols == op->ws->cols && G->sb_cols == op->sb->cols &&
         std::memcmp(G->lazy, lazy, sizeof(lazy)) == 0 && std::memcmp(&G->plan, &op->plan, sizeof(rfcmp_plan)) == 0 &&
         G->prof_key == prof_capture_key();
}

// Captures the solve loop of op for nr columns into one executable graph:
//   refine_residual(init)                       sets go
//   WHILE go:  cg_start
//              WHILE live: apply A (inner arithmetic), cg_pap, cg_update, cg_direction
//              i += d, r = b - A i (accurate), refine_residual  (sets go)
int capture_solve_graph(rfcmp_op* op, int nr, GemvMode inner, int max_sweeps) {
  SolveBuffers& B = *op->sb;
  for (cudaStream_t& c : op->capture)
    if (!c) RF_CUDA(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
  op->solve_graph.reset();
  cudaGraph_t g = nullptr;
  RF_CUDA(cudaGraphCreate(&g, 0));
  struct GraphGuard {
    cudaGraph_t g;
    ~GraphGuard() {
      if (g) cudaGraphDestroy(g);
    }
  } gg{g};
  KrylovView K = krylov_view(op, B, nr);
  K.graph = 1;
  RF_CUDA(cudaGraphConditionalHandleCreate(&K.h_outer, g, 0, 0));
  RF_CUDA(cudaGraphConditionalHandleCreate(&K.h_inner, g, 0, 0));
  cudaStream_t s0 = op->capture[0], s1 = op->capture[1], s2 = op->capture[2];
  RF_CUDA(cudaStreamBeginCaptureToGraph(s0, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  CaptureGuard c0(s0);
  RF_K(krylov_refine_residual(K, B.b, nullptr, B.r, B.i, true, s0));
  cudaGraph_t outer = nullptr;
  RF_TRY(add_while(s0, K.h_outer, &outer));
  {
    RF_CUDA(cudaStreamBeginCaptureToGraph(s1, outer, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    CaptureGuard c1(s1);
    RF_K(krylov_cg_start(K, B.r, B.d, B.rin, B.p, s1));
    cudaGraph_t body = nullptr;
    RF_TRY(add_while(s1, K.h_inner, &body));
    {
      RF_CUDA(cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      CaptureGuard c2(s2);
      RF_TRY(cg_iteration(op, B, K, nr, inner, s2));
      c2.open = false;
      RF_CUDA(cudaStreamEndCapture(s2, &body));
    }
    RF_TRY(refine_step(op, B, K, nr, s1));
    c1.open = false;
    RF_CUDA(cudaStreamEndCapture(s1, &outer));
  }
  c0.open = false;
  RF_CUDA(cudaStreamEndCapture(s0, &g));
  auto G = std::make_unique<SolveGraph>();
  RF_CUDA(cudaGraphInstantiate(&G->exec, g, 0));
  G->nr = nr;
  G->mode = (int)inner;
  G->max_sweeps = max_sweeps;
  G->ws = op->ws.get();
  G->sb = op->sb.get();
  G->ws_cols = op->ws->cols;
  G->sb_cols = op->sb->cols;
  const void* lazy[10] = {op->ta_planes.rh,   op->v_planes.rh,     op->ta_digits.d,  op->v_digits.d,
                          op->lplus->planes.h, op->lplus->digits.d, op->gll->planes.h, op->gll->digits.d,
                          op->gtp ? op->gtp->planes.h : nullptr, op->gtp ? op->gtp->digits.d : nullptr};
  std::memcpy(G->lazy, lazy, sizeof(lazy));
  G->plan = op->plan;
  G->prof_key = prof_capture_key();
  op->solve_graph = std::move(G);
  return RFCMP_OK;
}

// The refinement loop (Sec. 4 CG inside FP64-accurate residual sweeps), device-resident: one
// graph launch where graphs are available, else the eager driver.
int solve_loop(rfcmp_op* op, int nr, GemvMode inner, int max_sweeps, int max_iter, cudaStream_t st) {
  if (solve_graphs_enabled() && !op->graphs_failed) {
    if (!solve_graph_current(op, nr, inner, max_sweeps)) {
      const int rc = capture_solve_graph(op, nr, inner, max_sweeps);
      if (rc != RFCMP_OK) {
        op->solve_graph.reset();
        op->graphs_failed = true;
        (void)cudaGetLastError();
      }
    }
    if (op->solve_graph) {
      RF_CUDA(cudaGraphLaunch(op->solve_graph->exec, st));
      return RFCMP_OK;
    }
  }
  return solve_loop_eager(op, nr, inner, max_sweeps, max_iter, st);
}

int solve_impl(rfcmp_op* op, const double2* e, double2* j, int nr, const rfcmp_solve_opts& o,
               rfcmp_solve_report* rep, cudaStream_t st) {
  RF_TRY(ensure_workspace(op, nr));
  RF_TRY(ensure_solve_buffers(op, nr));
  SolveBuffers& B = *op->sb;
  const bool mixed = o.precision == RFCMP_PREC_MIXED;
  const GemvMode inner_mode = mixed ? GEMV_F32 : GEMV_FF;
  const int max_sweeps = mixed ? o.max_refine : 1;
  // operands built on first use must exist before the loop is captured
  if (inner_mode == GEMV_F32 && nr >= plan_mrhs(op)) RF_TRY(ensure_planes(op, 0));
  if (nr >= plan_exact(op)) RF_TRY(ensure_digits(op, 0));
  RF_TRY(order_stream(op, st));
  // b = -P_o^H T^H P_m e (float-float accurate)
  RF_TRY(apply_rhs(op, e, B.b, nr, GEMV_FF, st));
  const KrylovView K = krylov_view(op, B, nr);
  RF_K(krylov_params(K, o.tol, o.inner_tol, o.max_iter, max_sweeps, mixed, st));
  RF_TRY(solve_loop(op, nr, inner_mode, max_sweeps, o.max_iter, st));
  // j = P_o i
  RF_TRY(apply_Po(op, B.i, j, nr, false, GEMV_FF, st));
  // the per-column report and the wait-error flag, read once the stream has drained
  std::vector<int> iters(nr), sweeps(nr), conv(nr);
  std::vector<double> res(nr);
  int h_err = 0;
  RF_CUDA(cudaMemcpyAsync(iters.data(), B.iters, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaMemcpyAsync(sweeps.data(), B.sweeps, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaMemcpyAsync(conv.data(), B.conv, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaMemcpyAsync(res.data(), B.res, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
  if (op->ws->ms.err) RF_CUDA(cudaMemcpyAsync(&h_err, op->ws->ms.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaStreamSynchronize(st));
  if (h_err) {
    RF_CUDA(cudaMemset(op->ws->ms.err, 0, sizeof(int)));
    return set_error(RFCMP_ERR_DEVICE_TIMEOUT, "a bounded device-side wait gave up (code " +
                                                   std::to_string(h_err) + ")");
  }
  bool all = true;
  for (int c = 0; c < nr; ++c) {
    if (rep) {
      rep[c].converged = conv[c];
      rep[c].iterations = iters[c];
      rep[c].refinements = sweeps[c];
      rep[c].reserved = 0;
      rep[c].residual = res[c];
    }
    all &= conv[c] != 0;
  }
  if (!all && o.fail_on_nonconvergence) return set_error(RFCMP_ERR_NOT_CONVERGED, "a column did not reach tol");
  return RFCMP_OK;
}

int check_solve_opts(const rfcmp_solve_opts* in, rfcmp_solve_opts& o) {
  rfcmp_solve_opts_default(&o);
  if (in) o = *in;
  for (int i = 0; i < 8; ++i)
    if (o.reserved[i] != 0) return set_error(RFCMP_ERR_INVALID_ARG, "opts.reserved must be zero");
  if (!(o.tol > 0.0) || o.max_iter < 1 || o.max_iter > 1000000 || o.max_refine < 0 || o.max_refine > 1000 ||
      !(o.inner_tol > 0.0) || o.inner_tol >= 1.0 ||
      (o.precision != RFCMP_PREC_MIXED && o.precision != RFCMP_PREC_FF))
    return set_error(RFCMP_ERR_INVALID_ARG, "invalid solve options");
  return RFCMP_OK;
}

}  // namespace

extern "C" {

int rfcmp_solve(rfcmp_op* op, const rfcmp_c128* e, rfcmp_c128* j, int64_t nrhs, const rfcmp_solve_opts* opts,
                rfcmp_solve_report* report, void* stream) {
  if (!op || !e || !j || nrhs <= 0 || nrhs > 4096) return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  rfcmp_solve_opts o;
  RF_TRY(check_solve_opts(opts, o));
  RF_CUDA(cudaSetDevice(op->ctx->device));
  return solve_impl(op, reinterpret_cast<const double2*>(e), reinterpret_cast<double2*>(j), (int)nrhs, o, report,
                    (cudaStream_t)stream);
}

int rfcmp_solve_host(rfcmp_op* op, const rfcmp_c128* e_host, rfcmp_c128* j_host, int64_t nrhs,
                     const rfcmp_solve_opts* opts, rfcmp_solve_report* report, void* stream) {
  if (!op || !e_host || !j_host || nrhs <= 0 || nrhs > 4096)
    return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  rfcmp_solve_opts o;
  RF_TRY(check_solve_opts(opts, o));
  RF_CUDA(cudaSetDevice(op->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double2) * (size_t)op->top.ne * nrhs;
  double2 *de = nullptr, *dj = nullptr;
  RF_CUDA(cudaMallocAsync(&de, bytes, st));
  RF_CUDA(cudaMallocAsync(&dj, bytes, st));
  RF_CUDA(cudaMemcpyAsync(de, e_host, bytes, cudaMemcpyHostToDevice, st));
  int rc = solve_impl(op, de, dj, (int)nrhs, o, report, st);
  if (rc == RFCMP_OK) {
    cudaError_t err = cudaMemcpyAsync(j_host, dj, bytes, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) rc = set_error(RFCMP_ERR_CUDA, std::string("copy back: ") + cudaGetErrorString(err));
  }
  cudaFreeAsync(de, st);
  cudaFreeAsync(dj, st);
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------- batch sessions
// A multi-column solve whose columns are admitted and retired between refinement sweeps: the
// serving form of continuous batching.  Slots 0..cap-1 hold columns; a sweep runs the columns
// 0..hi-1 (hi one past the highest occupied slot), where free and finished slots are out of the
// solve (the member mask) and only cost their share of the operator products.
struct rfcmp_batch {
  rfcmp_op* op = nullptr;
  int cap = 0;
  rfcmp_solve_opts o{};
  GemvMode inner = GEMV_F32;
  int max_sweeps = 0;
  std::unique_ptr<SolveBuffers> sb;
  std::vector<int> state;  // 0 free, 1 running, 2 finished
  std::vector<int> h_iters, h_sweeps, h_conv;
  std::vector<double> h_res;
  int* dslots = nullptr;     // device copy of the slots of the current admission or release
  double2* stage = nullptr;  // N x cap: right-hand sides b of admitted columns before they move to their slots
  ~rfcmp_batch() {
    if (dslots) dev_free(dslots);
    if (stage) dev_free(stage);
  }
};

namespace {
int batch_hi(const rfcmp_batch* b) {
  int hi = 0;
  for (int c = 0; c < b->cap; ++c)
    if (b->state[c] != 0) hi = c + 1;
  return hi;
}
}  // namespace

extern "C" {

int rfcmp_batch_create(rfcmp_op* op, int32_t capacity, const rfcmp_solve_opts* opts, rfcmp_batch** out) {
  if (!op || !out || capacity < 1 || capacity > 4096) return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  *out = nullptr;
  auto b = std::make_unique<rfcmp_batch>();
  RF_TRY(check_solve_opts(opts, b->o));
  RF_CUDA(cudaSetDevice(op->ctx->device));
  b->op = op;
  b->cap = capacity;
  const bool mixed = b->o.precision == RFCMP_PREC_MIXED;
  b->inner = mixed ? GEMV_F32 : GEMV_FF;
  b->max_sweeps = mixed ? b->o.max_refine : 1;
  RF_TRY(ensure_workspace(op, capacity));
  RF_TRY(alloc_solve_buffers(op, capacity, b->sb));
  RF_TRY(dalloc(&b->sb->member, capacity, b->sb->owned));
  RF_CUDA(cudaMemset(b->sb->member, 0, sizeof(int) * capacity));
  for (double2* v : {b->sb->b, b->sb->i, b->sb->r})  // free slots hold zeros, never stale values
    RF_CUDA(cudaMemset(v, 0, sizeof(double2) * (size_t)op->top.ne * capacity));
  RF_CUDA(dev_malloc((void**)&b->dslots, sizeof(int) * capacity));
  RF_CUDA(dev_malloc((void**)&b->stage, sizeof(double2) * (size_t)op->top.ne * capacity));
  b->state.assign(capacity, 0);
  b->h_iters.assign(capacity, 0);
  b->h_sweeps.assign(capacity, 0);
  b->h_conv.assign(capacity, 0);
  b->h_res.assign(capacity, 0.0);
  KrylovView K = krylov_view(op, *b->sb, capacity);
  RF_K(krylov_params(K, b->o.tol, b->o.inner_tol, b->o.max_iter, b->max_sweeps, mixed, 0));
  RF_CUDA(cudaStreamSynchronize(0));
  *out = b.release();
  return RFCMP_OK;
}

int rfcmp_batch_destroy(rfcmp_batch* b) {
  if (!b) return RFCMP_OK;
  cudaSetDevice(b->op->ctx->device);
  drain_streams(b->op);
  delete b;
  return RFCMP_OK;
}

int rfcmp_batch_admit(rfcmp_batch* b, const rfcmp_c128* e, int32_t n, int32_t* slots, void* stream) {
  if (!b || !e || !slots || n < 1) return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  std::vector<int> free_slots;
  for (int c = 0; c < b->cap && (int)free_slots.size() < n; ++c)
    if (b->state[c] == 0) free_slots.push_back(c);
  if ((int)free_slots.size() < n) return set_error(RFCMP_ERR_INVALID_ARG, "not enough free slots in the batch");
  rfcmp_op* op = b->op;
  RF_CUDA(cudaSetDevice(op->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  RF_TRY(ensure_workspace(op, b->cap));
  RF_TRY(order_stream(op, st));
  SolveBuffers& B = *b->sb;
  const size_t N = op->top.ne;
  // b = -P_o^H T^H P_m e (float-float accurate) for the new columns, then into their slots
  RF_TRY(apply_rhs(op, reinterpret_cast<const double2*>(e), b->stage, n, GEMV_FF, st));
  RF_K(vec_dot(b->stage, b->stage, (int64_t)N, n, B.dots, st));
  for (int q = 0; q < n; ++q) {
    const size_t off = (size_t)free_slots[q] * N;
    RF_CUDA(cudaMemcpyAsync(B.b + off, b->stage + (size_t)q * N, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    RF_CUDA(cudaMemcpyAsync(B.r + off, b->stage + (size_t)q * N, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    RF_CUDA(cudaMemsetAsync(B.i + off, 0, sizeof(double2) * N, st));
  }
  RF_CUDA(cudaMemcpyAsync(b->dslots, free_slots.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  KrylovView K = krylov_view(op, B, b->cap);
  RF_K(krylov_slots(K, b->dslots, n, B.dots, st));
  RF_CUDA(cudaStreamSynchronize(st));  // the slot list on the host is reused by the next call
  for (int q = 0; q < n; ++q) {
    b->state[free_slots[q]] = 1;
    slots[q] = free_slots[q];
  }
  return RFCMP_OK;
}

int rfcmp_batch_step(rfcmp_batch* b, int32_t* finished, int32_t* n_finished, void* stream) {
  if (!b || !finished || !n_finished) return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  *n_finished = 0;
  rfcmp_op* op = b->op;
  RF_CUDA(cudaSetDevice(op->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int hi = batch_hi(b);
  bool running = false;
  for (int c = 0; c < hi; ++c) running |= b->state[c] == 1;
  if (!running) return RFCMP_OK;
  RF_TRY(ensure_workspace(op, b->cap));
  RF_TRY(order_stream(op, st));
  SolveBuffers& B = *b->sb;
  KrylovView K = krylov_view(op, B, hi);
  RF_K(krylov_decide(K, st));
  KrylovCtl h{};
  RF_TRY(read_ctl(B, h, st));
  if (h.live > 0) RF_TRY(eager_sweep(op, B, K, hi, b->inner, b->o.max_iter, st));
  RF_CUDA(cudaMemcpyAsync(b->h_iters.data(), B.iters, sizeof(int) * hi, cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaMemcpyAsync(b->h_sweeps.data(), B.sweeps, sizeof(int) * hi, cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaMemcpyAsync(b->h_conv.data(), B.conv, sizeof(int) * hi, cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaMemcpyAsync(b->h_res.data(), B.res, sizeof(double) * hi, cudaMemcpyDeviceToHost, st));
  int h_err = 0;
  if (op->ws->ms.err) RF_CUDA(cudaMemcpyAsync(&h_err, op->ws->ms.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaStreamSynchronize(st));
  if (h_err) {
    RF_CUDA(cudaMemset(op->ws->ms.err, 0, sizeof(int)));
    return set_error(RFCMP_ERR_DEVICE_TIMEOUT, "a bounded device-side wait gave up (code " + std::to_string(h_err) + ")");
  }
  for (int c = 0; c < hi; ++c) {
    if (b->state[c] != 1) continue;
    if (b->h_conv[c] || b->h_iters[c] >= b->o.max_iter || b->h_sweeps[c] >= b->max_sweeps) {
      b->state[c] = 2;
      finished[(*n_finished)++] = c;
    }
  }
  return RFCMP_OK;
}

int rfcmp_batch_take(rfcmp_batch* b, const int32_t* slots, int32_t n, rfcmp_c128* j, rfcmp_solve_report* reports,
                     void* stream) {
  if (!b || !slots || !j || n < 1 || n > b->cap) return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  for (int q = 0; q < n; ++q) {
    if (slots[q] < 0 || slots[q] >= b->cap) return set_error(RFCMP_ERR_INVALID_ARG, "slot out of range");
    if (b->state[slots[q]] != 2) return set_error(RFCMP_ERR_INVALID_ARG, "slot has no finished column");
    for (int p = 0; p < q; ++p)
      if (slots[p] == slots[q]) return set_error(RFCMP_ERR_INVALID_ARG, "slot listed twice");
  }
  rfcmp_op* op = b->op;
  RF_CUDA(cudaSetDevice(op->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  RF_TRY(ensure_workspace(op, b->cap));
  RF_TRY(order_stream(op, st));
  SolveBuffers& B = *b->sb;
  const size_t N = op->top.ne;
  // the finished columns of i side by side, then j = P_o i for all of them in one application
  for (int q = 0; q < n; ++q)
    RF_CUDA(cudaMemcpyAsync(b->stage + (size_t)q * N, B.i + (size_t)slots[q] * N, sizeof(double2) * N,
                            cudaMemcpyDeviceToDevice, st));
  RF_TRY(apply_Po(op, b->stage, reinterpret_cast<double2*>(j), n, false, GEMV_FF, st));
  if (reports) {
    for (int q = 0; q < n; ++q) {
      const int c = slots[q];
      reports[q].converged = b->h_conv[c];
      reports[q].iterations = b->h_iters[c];
      reports[q].refinements = b->h_sweeps[c];
      reports[q].reserved = 0;
      reports[q].residual = b->h_res[c];
    }
  }
  RF_CUDA(cudaMemcpyAsync(b->dslots, slots, sizeof(int) * n, cudaMemcpyHostToDevice, st));
  KrylovView K = krylov_view(op, B, b->cap);
  RF_K(krylov_slots(K, b->dslots, n, nullptr, st));
  RF_CUDA(cudaStreamSynchronize(st));  // the slot list on the host may go out of scope
  for (int q = 0; q < n; ++q) b->state[slots[q]] = 0;
  return RFCMP_OK;
}

int rfcmp_batch_counts(const rfcmp_batch* b, int32_t* running, int32_t* finished, int32_t* free_slots) {
  if (!b) return set_error(RFCMP_ERR_INVALID_ARG, "NULL batch");
  int r = 0, f = 0, e = 0;
  for (int s : b->state) (s == 1 ? r : (s == 2 ? f : e))++;
  if (running) *running = r;
  if (finished) *finished = f;
  if (free_slots) *free_slots = e;
  return RFCMP_OK;
}

int rfcmp_gemm_bf16x3(const float* A, int64_t lda, const float* B, int64_t ldb, float* D, int64_t ldd, int64_t M,
                      int64_t N, int64_t K, int accumulate, void* stream) {
  if (!A || !B || !D || M <= 0 || N <= 0 || K <= 0 || lda < K || ldb < K || ldd < N || M > (1 << 30) ||
      N > (1 << 30) || K > (1 << 30))
    return set_error(RFCMP_ERR_INVALID_ARG, "invalid GEMM arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const long long ldp = (K + 7) / 8 * 8;  // plane row stride: 16-byte multiple
  __nv_bfloat16* pl = nullptr;
  int* err = nullptr;
  const size_t na = (size_t)M * ldp, nb = (size_t)N * ldp;
  RF_CUDA(cudaMallocAsync(&pl, sizeof(__nv_bfloat16) * 2 * (na + nb), st));
  RF_CUDA(cudaMallocAsync(&err, sizeof(int), st));
  RF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  RF_CUDA(cudaMemsetAsync(pl, 0, sizeof(__nv_bfloat16) * 2 * (na + nb), st));
  SplitOperand a, b;
  a.hi = pl;
  a.lo = pl + na;
  a.rows = (int)M;
  a.ld = ldp;
  b.hi = pl + 2 * na;
  b.lo = pl + 2 * na + nb;
  b.rows = (int)N;
  b.ld = ldp;
  RF_K(split_bf16_f32(A, lda, (int)M, (int)K, const_cast<__nv_bfloat16*>(a.hi), const_cast<__nv_bfloat16*>(a.lo),
                      ldp, st));
  RF_K(split_bf16_f32(B, ldb, (int)N, (int)K, const_cast<__nv_bfloat16*>(b.hi), const_cast<__nv_bfloat16*>(b.lo),
                      ldp, st));
  RF_K(gemm_bf16x3(&a, &b, nullptr, 1, (int)M, (int)N, (int)K, D, ldd, accumulate != 0, err, st));
  int h_err = 0;
  RF_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaFreeAsync(pl, st));
  RF_CUDA(cudaFreeAsync(err, st));
  RF_CUDA(cudaStreamSynchronize(st));
  if (h_err) return set_error(RFCMP_ERR_DEVICE_TIMEOUT, "GEMM kernel wait timed out (code " + std::to_string(h_err) + ")");
  return RFCMP_OK;
}

int rfcmp_farfield(rfcmp_op* op, const rfcmp_c128* j, int64_t nrhs, const double* dirs, int64_t ndir,
                   double* rcs_dbsm, void* stream) {
  if (!op || !j || !dirs || !rcs_dbsm || nrhs <= 0 || ndir <= 0 || nrhs > 65535 || ndir > (1 << 20))
    return set_error(RFCMP_ERR_INVALID_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  double* dd = nullptr;
  double2* dn = nullptr;
  RF_CUDA(cudaMallocAsync(&dd, sizeof(double) * 3 * ndir, st));
  RF_CUDA(cudaMallocAsync(&dn, sizeof(double2) * 3 * ndir * nrhs, st));
  RF_CUDA(cudaMemcpyAsync(dd, dirs, sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, st));
  RF_K(launch_farfield(op->g, op->k, reinterpret_cast<const double2*>(j), (int)nrhs, dd, (int)ndir, dn, st));
  std::vector<double2> h(3 * ndir * nrhs);
  RF_CUDA(cudaMemcpyAsync(h.data(), dn, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaFreeAsync(dd, st));
  RF_CUDA(cudaFreeAsync(dn, st));
  RF_CUDA(cudaStreamSynchronize(st));
  const double k = op->k;
  for (int64_t r = 0; r < nrhs; ++r)
    for (int64_t d = 0; d < ndir; ++d) {
      const double* u = dirs + 3 * d;
      const double2* n = &h[(r * ndir + d) * 3];
      double2 dot = make_double2(u[0] * n[0].x + u[1] * n[1].x + u[2] * n[2].x,
                                 u[0] * n[0].y + u[1] * n[1].y + u[2] * n[2].y);
      double s = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double pr = n[a].x - u[a] * dot.x, pi = n[a].y - u[a] * dot.y;
        s += pr * pr + pi * pi;
      }
      const double sigma = k * k / (4.0 * M_PI) * s;
      rcs_dbsm[r * ndir + d] = 10.0 * std::log10(std::max(sigma, 1e-300));
    }
  return RFCMP_OK;
}

}  // extern "C"
