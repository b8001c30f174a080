// Internal declarations shared by the translation units of librfcmp.
// Host topology (topology.cpp), kernels (k_assembly.cu, k_linalg.cu) and the
// C ABI (capi.cu).  Nothing here is part of the public interface.
#pragma once

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/rfcmp.h"

namespace rfcmp {

// Launch accounting: every kernel of the library adds one to its translation unit's device
// counter from block 0, thread 0 as its first statement, so the count covers every launch
// whatever the kernel does next.  Each .cu file defines a reader (RF_LAUNCH_READER); the C ABI
// sums them (rfcmp_launch_count).
#ifdef __CUDACC__
static __device__ unsigned long long g_rf_launches;
#define RF_COUNT_LAUNCH()                                                                      \
  do {                                                                                         \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
      atomicAdd(&::rfcmp::g_rf_launches, 1ULL);                                                \
  } while (0)
#define RF_LAUNCH_READER(fn)                                                              \
  unsigned long long fn() {                                                                \
    unsigned long long v = 0;                                                              \
    if (cudaMemcpyFromSymbol(&v, ::rfcmp::g_rf_launches, sizeof(v)) != cudaSuccess) v = 0; \
    return v;                                                                              \
  }
#endif
unsigned long long launches_assembly();
unsigned long long launches_exact();
unsigned long long launches_factor();
unsigned long long launches_gemm();
unsigned long long launches_gemv_stream();
unsigned long long launches_linalg();
unsigned long long launches_krylov();
unsigned long long launches_hmatrix();

// ---------------------------------------------------------------- op accessors
// Read-only view of an operator's T_A for translation units outside capi.cu.
struct OpTaView {
  const float2* TA = nullptr;
  int n = 0;
  int device = 0;
};
bool op_ta_view(const rfcmp_op* op, OpTaView* out);
struct Topology;
// Read-only view of an operator's dense T_A and V, its mesh and its context's accounting, for the
// compressed form (k_hmatrix.cu).
struct OpDenseView {
  const float2* TA = nullptr;
  const float2* V = nullptr;
  int n = 0, nc = 0;      // rows of T_A (RWG functions) and V (cells)
  int ldN = 0, ldC = 0;   // their row strides (elements); both triangles are stored
  int device = 0;
  const Topology* top = nullptr;
  const double* verts = nullptr;        // mesh vertices, 3 per vertex
  std::atomic<uint64_t>* ctx_bytes = nullptr;
  std::atomic<int>* ctx_live = nullptr;  // objects that must be destroyed before the context
  uint64_t budget = 0;                   // the context's HBM budget (0: none)
};
bool op_dense_view(rfcmp_op* op, OpDenseView* out);
// Records the message returned by rfcmp_last_error() for the calling thread; returns code.
int set_error(int code, const std::string& msg);

// ---------------------------------------------------------------- profiling
// RAII bracket of one launch by CUDA events on its stream (no-op when disabled).
class ProfScope {
 public:
  ProfScope(const char* family, double bytes, double flops, cudaStream_t s);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  int slot_ = -1;
  cudaStream_t s_ = nullptr;
  cudaEvent_t a_ = nullptr, b_ = nullptr;  // this launch's own start / end events
  uint64_t gen_ = 0;                        // profiling generation the slot belongs to
  // launches captured into a graph: device timestamps instead of events
  bool captured_ = false;
  int scope_ = 0;
  double bytes_ = 0.0, flops_ = 0.0;
};

// ---------------------------------------------------------------- host topology
// Edge numbering and signs follow include/rfcmp.h (Sec. 2, Eq. RWGdef, Eq. qHofj).
struct Topology {
  int64_t nv = 0, nc = 0, ne = 0;  // nv: loop functions (the interior vertices)
  int64_t nv_mesh = 0;             // vertices of the mesh
  int genus = 0;
  int boundaries = 0;                // boundary curves (0: a closed surface)
  std::vector<int32_t> loop_of;      // nv_mesh: loop index of a vertex, -1 on the boundary
  std::vector<int32_t> loop_verts;   // nv: mesh vertex of each loop function
  std::vector<int32_t> edge_loops;   // ne x 2: loop indices of (v1, v2), -1 on the boundary
  std::vector<int32_t> tris;        // nc x 3
  std::vector<int32_t> edge_verts;  // ne x 2 (v1, v2): c^+ traverses v1 -> v2
  std::vector<int32_t> edge_cells;  // ne x 2 (c^+, c^-)
  std::vector<int32_t> edge_free;   // ne x 2 (r^+, r^-)
  std::vector<int32_t> cell_edges;  // nc x 3, edge opposite local vertex i
  std::vector<int8_t> cell_sign;    // nc x 3, +1 if the cell is c^+ of that edge
  // Lambda^T gather: for vertex v, entries [vtx_ptr[v], vtx_ptr[v+1]) of vtx_edge / vtx_sign
  std::vector<int32_t> vtx_ptr, vtx_edge;
  std::vector<int8_t> vtx_sign;
  // Sigma^T Sigma as CSR (cell graph Laplacian: the cell's RWG edges on the diagonal, -1 per
  // shared edge)
  std::vector<int32_t> lap_ptr, lap_col;
  std::vector<double> lap_val;
  // unordered near pairs (s <= t) of cells sharing at least one vertex
  std::vector<int32_t> near_pairs;  // P x 2
  uint64_t hash = 0;                // of the connectivity only
};

// Builds the topology; returns RFCMP_OK or a mesh error with a message.
int build_topology(const int32_t* tris, int64_t nc, int64_t nv, Topology& out, std::string& err);

// G_l~p (dual piecewise linear x primal pulse, Sec. 3) as CSR over the cells, from the case
// formula of Sec. 3 (diagonal, cells sharing an edge, cells sharing only a vertex).
void gtp_matrix_csr(const Topology& top, std::vector<int32_t>& ptr, std::vector<int32_t>& col,
                    std::vector<double>& val);

// G_ll (P1 mass matrix) as CSR over the loop (interior) vertices, local block
// A/12 [[2,1,1],[1,2,1],[1,1,2]] restricted to them.
void mass_matrix_csr(const Topology& top, const double* verts, std::vector<int32_t>& ptr,
                     std::vector<int32_t>& col, std::vector<double>& val);

// ---------------------------------------------------------------- device geometry
// Per-cell data for the assembly kernels; structure of arrays, FP32 copies of
// quantities relative to the centroid plus FP64 copies for the near pairs.
struct DeviceGeometry {
  int32_t nc = 0, ne = 0, nv = 0;
  int32_t ldN = 0, ldC = 0;  // padded row strides (elements) of T_A and V
  float rq_max = 0.f;        // largest distance of a quadrature point from its cell's centroid (+ margin)
  float rq_mean = 0.f;       // that distance per cell, averaged over the cells
  // FP32 (far pairs)
  float* cen_hi = nullptr;   // nc x 3 (centroid rounded to FP32)
  float* cen_lo = nullptr;   // nc x 3 (centroid - cen_hi)
  float* rho = nullptr;      // nc x 7 x 3 quadrature points minus centroid
  float* wq = nullptr;       // nc x 7 weight x area
  float* aloc = nullptr;     // nc x 3 x 3 free vertex of local basis i minus centroid
  float* inv_area = nullptr; // nc
  // FP64 (near pairs, excitation, far field)
  double* verts = nullptr;    // nv x 3
  double* cen64 = nullptr;    // nc x 3
  double* area64 = nullptr;   // nc
  double* qp64 = nullptr;     // nc x 7 x 3 quadrature points
  // topology
  int32_t* tris = nullptr;        // nc x 3
  int32_t* cell_edges = nullptr;  // nc x 3
  int8_t* cell_sign = nullptr;    // nc x 3
  int32_t* edge_cells = nullptr;  // ne x 2
  int32_t* edge_loops = nullptr;  // ne x 2 loop indices of the edge ends (-1 on the boundary)
  int32_t* edge_free = nullptr;   // ne x 2
  int32_t* vtx_ptr = nullptr;     // nv + 1
  int32_t* vtx_edge = nullptr;
  int8_t* vtx_sign = nullptr;
  int32_t* lap_ptr = nullptr;     // nc + 1
  int32_t* lap_col = nullptr;
  double* lap_val = nullptr;
  int32_t* near_pairs = nullptr;  // n_near x 2
  int32_t n_near = 0;
};

// ---------------------------------------------------------------- kernels (k_assembly.cu)
// T_A (ne x ne) and V (nc x nc), complex64 row-major, must be zeroed by the caller.
// min_blocks: resident CTAs per SM the register allocation is sized for (1, 2 or 3; 0 = 2)
cudaError_t launch_assemble_far(const DeviceGeometry& g, float k, float2* TA, float2* V, int min_blocks,
                                cudaStream_t s);
cudaError_t launch_assemble_near(const DeviceGeometry& g, double k, float2* TA, float2* V, cudaStream_t s);
// T_A is accumulated in its upper triangle; this copies it to the lower one (bit-identical symmetry)
cudaError_t launch_mirror_upper(float2* M, int n, int ld, cudaStream_t s);
// e (ne x nrhs complex128), khat/pol device nrhs x 3
cudaError_t launch_rhs_voltage_gap(const DeviceGeometry& g, const double* origin, const double* normal, double2 v,
                                   double2* e, cudaStream_t s);
cudaError_t launch_rhs_planewave(const DeviceGeometry& g, double k, const double* khat, const double* pol,
                                 int nrhs, double2* e, cudaStream_t s);
// radiation vector N(rhat) for nrhs currents and ndir directions -> out (ndir x nrhs x 3 complex)
cudaError_t launch_farfield(const DeviceGeometry& g, double k, const double2* j, int nrhs, const double* dirs,
                            int ndir, double2* out, cudaStream_t s);

// ---------------------------------------------------------------- tensor-core GEMM (k_gemm.cu)
// A BF16 operand split in two planes (hi = bf16(x), lo = bf16(x - hi)), row-major with K
// contiguous, `rows` rows, row stride `ld` elements (ld * 2 bytes a multiple of 16).
struct SplitOperand {
  const __nv_bfloat16* hi = nullptr;
  const __nv_bfloat16* lo = nullptr;
  int rows = 0;
  long long ld = 0;
};
// D[M x N] = sum_g (negate[g] ? -1 : 1) A_g B_g^T (+ D), three BF16 products per K step into an
// FP32 tensor-memory accumulator (tcgen05).  nseg 1 or 2.  err_dev receives a nonzero code if a
// bounded device-side wait gave up.
// bn selects the N tile (32, 64 or 128); 0 picks it from N.  With upper, only the 128 x 128 tiles
// on or above the diagonal are computed (for a result known to be symmetric).
cudaError_t gemm_bf16x3(const SplitOperand* A, const SplitOperand* B, const int* negate, int nseg, int M, int N,
                        int K, float* D, long long ldd, bool accumulate, int* err_dev, cudaStream_t s, int bn = 0,
                        bool upper = false);
cudaError_t split_bf16_f32(const float* src, long long ld_src, int rows, int cols, __nv_bfloat16* hi,
                           __nv_bfloat16* lo, long long ld_dst, cudaStream_t s);

// BF16 planes of the resident blocks for the multi-right-hand-side products.
struct CplxPlanes {  // complex n x n: Re hi/lo, Im hi/lo, row stride ldp; ih = rh + n ldp, il = rl + n ldp
  __nv_bfloat16 *rh = nullptr, *rl = nullptr, *ih = nullptr, *il = nullptr;
  int n = 0;
  long long ldp = 0;
};
struct RealPlanes {  // real n x n: hi/lo, row stride ldp
  __nv_bfloat16 *h = nullptr, *l = nullptr;
  int n = 0;
  long long ldp = 0;
};
// Scratch of the multi-RHS products: BF16 planes of X (4 x cap_cols x cap_ld) and the FP32
// products (2 x cap_n x cap_cols); err receives device-side timeout codes.
struct MrhsScratch {
  __nv_bfloat16* xb = nullptr;
  float* D = nullptr;  // 4 x cap_cols x cap_n
  int* err = nullptr;
  int cap_cols = 0, cap_n = 0;
  long long cap_ld = 0;
  int bn = 0;  // GEMM N tile (32, 64, 128; 0 = by column count)
  // exact-digit products (float-float accurate multi-column products)
  __nv_bfloat16* xd = nullptr;  // EXACT_DIGITS planes of 2 cap_cols x cap_ld
  int* xe = nullptr;            // 2 cap_cols row exponents
  double* D64 = nullptr;        // 4 x cap_cols x cap_n
};

// Exact-digit operands: every row r scaled by 2^e[r] and written as EXACT_DIGITS signed 8-bit
// digits, plane p of rows x ldp BF16 at d + p * plane_stride.
constexpr int EXACT_DIGITS = 6;
struct ExactOperand {
  __nv_bfloat16* d = nullptr;
  int* e = nullptr;
  int rows = 0;
  long long ldp = 0;
  long long plane_stride = 0;
};
// digit planes of a complex64 matrix (n x n, row stride ld) as 2n rows [Re; Im]
cudaError_t exact_digits_c64(const float2* M, int n, long long ld, const ExactOperand& out, cudaStream_t s);
// digit planes of an FP64-accurate real matrix given as FP32 hi + lo planes
cudaError_t exact_digits_f32pair(const float* hi, const float* lo, int n, long long ld, const ExactOperand& out,
                                 cudaStream_t s);
// Y = scale * op(T) X (+ Y) and Y = scale * P X (+ Y), float-float accurate (about 2^-48 of the
// row and column scales per term), X, Y complex128 column-major n x nr.
cudaError_t exact_cplx_gemm(const ExactOperand& T, int n, const double2* X, double2* Y, int nr, bool conj,
                            double2 scale, bool accumulate, MrhsScratch& w, cudaStream_t s);
cudaError_t exact_real_gemm(const ExactOperand& P, int n, const double2* X, double2* Y, int nr, double scale,
                            bool accumulate, MrhsScratch& w, cudaStream_t s);
cudaError_t split_c64_planes(const float2* M, int n, long long ld, const CplxPlanes& P, cudaStream_t s);
// Y = scale * op(T) X (+ Y) with op = conj if conj; X, Y complex128 column-major n x nr.
cudaError_t cplx_gemm(const CplxPlanes& T, const double2* X, double2* Y, int nr, bool conj, double2 scale,
                      bool accumulate, MrhsScratch& w, cudaStream_t s);
// Y = scale * P X (+ Y) with a real P.
cudaError_t real_gemm(const RealPlanes& P, const double2* X, double2* Y, int nr, double scale, bool accumulate,
                      MrhsScratch& w, cudaStream_t s);
cudaError_t split_bf16_f64(const double* src, long long ld_src, int rows, int cols, __nv_bfloat16* hi,
                           __nv_bfloat16* lo, long long ld_dst, cudaStream_t s);

// ---------------------------------------------------------------- kernels (k_linalg.cu)
enum GemvMode { GEMV_F32 = 0, GEMV_FF = 1 };

// Device scratch of the GEMV: x converted to FP32 hi (and lo) padded to ld, and the output the
// persistent CTAs add their scaled FP64 row sums into.  Calls sharing a scratch must not overlap
// on the device.
struct GemvScratch {
  float2* xh = nullptr;   // cap_cols x cap_ld
  float2* xl = nullptr;   // cap_cols x cap_ld
  double2* out = nullptr; // y of the current product (set per call): CTAs add scale * partial sums
  double scale = 1.0;     // real factor of the current product
  int cap_n = 0, cap_ld = 0, cap_cols = 0;
  int chunk = 0;          // columns per work unit (multiple of 256; 0 = 1024)
  int ctas_per_sm = 0;    // persistent CTAs per SM (0 = occupancy maximum)
  int* err = nullptr;     // set when a bounded device-side wait of the streaming GEMV gives up
  bool symmetric = false; // every matrix this scratch serves is symmetric: read the upper triangle
};
// Streaming FP32-mode GEMV of a symmetric matrix (k_gemv_stream.cu; w.symmetric must be set): the
// prepared x (w.xh) times the complex64 or FP32 matrix, w.scale times it added into the FP64
// output w.out, the upper triangle streamed by bulk copies; NR = 1 or 2.
template <int NR>
cudaError_t gemv_stream_c64(const float2* M, int ld, int n, bool conj, GemvScratch& w, cudaStream_t s);
template <int NR>
cudaError_t gemv_stream_r32(const float* M, int ld, int n, GemvScratch& w, cudaStream_t s);
// Float-float streaming GEMV of one column of a complex64 M (x split in w.xh + w.xl).
cudaError_t gemv_stream_c64_ff(const float2* M, int ld, int n, bool conj, GemvScratch& w, cudaStream_t s);
int padded_ld(int n);

// Device memory from the device's stream-ordered pool, which keeps freed memory mapped: the
// large buffers of operators, factor builds and solve workspaces come and go once per operator
// or per wavenumber, and the pool turns their allocation and release into bookkeeping instead of
// page-table work.  Both calls synchronise like cudaMalloc / cudaFree (the memory is usable on
// any stream on return; a free waits for the device to go idle first).
cudaError_t dev_malloc(void** p, size_t bytes);
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}
cudaError_t dev_free(void* p);
// Returns the pool's unused memory of the current device to the driver.
void dev_pool_trim();

// y[:, r] = scale * op(M) x[:, r] (+ y[:, r] if accumulate), r < nrhs; M n x n complex64
// row-major with rows padded to padded_ld(n) (symmetric, so rows are columns); op = conj if
// conjugate.  x, y complex128 column-major with leading dimension n.
// fed: the kernel that produced x already wrote its split into w.xh (and w.xl) and zeroed y
// (GemvFeed), so the split is skipped; nrhs is then 1, 2 or 4.
cudaError_t gemv_c64(const float2* M, int n, const double2* x, double2* y, int nrhs, bool conjugate,
                     double2 scale, bool accumulate, GemvMode mode, GemvScratch& w, cudaStream_t s,
                     bool fed = false);
// y = op(M) x through the same kernels with no allocation of any kind (no profiling events,
// no cached launch-grid table).
cudaError_t gemv_c64_plain(const float2* M, int n, const double2* x, double2* y, int nrhs, bool conjugate,
                           GemvMode mode, GemvScratch& w, cudaStream_t s);
// y = scale * (Mhi [+ Mlo]) x with a real symmetric n x n matrix in FP32 hi/lo planes.
cudaError_t gemv_r32(const float* Mhi, const float* Mlo, int n, const double2* x, double2* y, int nrhs,
                     double scale, bool accumulate, GemvMode mode, GemvScratch& w, cudaStream_t s,
                     bool fed = false);

// What a sparse kernel writes besides its output when a GEMV reads that output next: the FP32
// split of each value exactly as the GEMV's own split would form it (hi, and lo for float-float
// products; zero padding up to ld), and the zeroed output of that GEMV (and of a second GEMV of
// the same vector).  All null: nothing besides the output.
struct GemvFeed {
  float2* xh = nullptr;
  float2* xl = nullptr;
  int ld = 0;
  double2* y = nullptr;
  double2* y2 = nullptr;
};

// sparse transforms (Sec. 2, Eq. qHofj); all complex128, nrhs columns
cudaError_t sigma_t(const DeviceGeometry& g, const double2* x, double2* out, int nrhs, cudaStream_t s,
                    const GemvFeed& feed = GemvFeed());  // N_C
cudaError_t lambda_t(const DeviceGeometry& g, const double2* x, double2* out, int nrhs, cudaStream_t s,
                     const GemvFeed& feed = GemvFeed());  // N_V
cudaError_t lap_apply(const DeviceGeometry& g, const double2* z, double2* out, int nrhs, cudaStream_t s,
                      const GemvFeed& feed = GemvFeed());  // Sigma^T Sigma z

// Fused edge-space combination: out = a*x + b*(Sigma zs) + c*(Lambda zl) + d*(Sigma zs2) + e*w
// with complex coefficients; any input may be null (its term is dropped).
struct EdgeCombo {
  const double2* x = nullptr;   double2 a{0, 0};
  const double2* zs = nullptr;  double2 b{0, 0};   // N_C vector through Sigma
  const double2* zl = nullptr;  double2 c{0, 0};   // N_V vector through Lambda
  const double2* zs2 = nullptr; double2 d{0, 0};   // second N_C vector through Sigma
  const double2* w = nullptr;   double2 e{0, 0};   // second edge vector
};
cudaError_t edge_combo(const DeviceGeometry& g, const EdgeCombo& c, double2* out, int nrhs, cudaStream_t s,
                       const GemvFeed& feed = GemvFeed());

// q = scale * diag(area) (z + w - mean(w)); mean over each column of w (N_C).  w may be null.
cudaError_t star_middle(const DeviceGeometry& g, const double2* z, const double2* w, double scale, double2* q,
                        int nrhs, double* scratch_mean, cudaStream_t s, const GemvFeed& feed = GemvFeed());

// q = a z + b (w - mean(w)) over the cells, per column; z may be null; scratch holds 2 x nrhs doubles
cudaError_t cell_combo(const DeviceGeometry& g, const double2* z, double2 a, const double2* w, double2 b, double2* q,
                       int nrhs, double* scratch_mean, cudaStream_t s);

// out = Pi diag(area) Pi w, Pi = I - 1 1^T / N_C (per column); scratch holds 4 x nrhs doubles
cudaError_t pgp_apply(const DeviceGeometry& g, const double2* w, double2* out, int nrhs, double* scratch,
                      cudaStream_t s);

// vector kernels (length n per column, nrhs columns)
cudaError_t vec_dot(const double2* a, const double2* b, int64_t n, int nrhs, double2* out, cudaStream_t s);  // out[r] = a^H b
cudaError_t vec_axpy_cols(const double* coef, bool negate, const double2* x, double2* y, int64_t n, int nrhs,
                          const int* active, cudaStream_t s);   // y += (+/-coef[r]) x
cudaError_t vec_xpby_cols(const double2* x, const double* coef, double2* y, int64_t n, int nrhs,
                          const int* active, cudaStream_t s);   // y = x + coef[r] y
cudaError_t vec_copy(const double2* x, double2* y, int64_t n, cudaStream_t s);
cudaError_t vec_copy_scale_cols(const double2* x, const double* coef, double2* y, int64_t n, int nrhs,
                               cudaStream_t s);  // y[:, r] = coef[r] x[:, r]
cudaError_t vec_scale(double2* y, double2 a, int64_t n, cudaStream_t s);
// CG scalar step on device: alpha = rr/pAp etc. (see k_linalg.cu)
cudaError_t cg_scalars_alpha(const double* rr, const double2* pAp, double* alpha, const int* active, int nrhs,
                             cudaStream_t s);
cudaError_t cg_scalars_beta(const double2* rr_new2, double* rr, double* beta, const int* active, int nrhs,
                            cudaStream_t s);

// ---------------------------------------------------------------- device-resident CG (k_krylov.cu)
// Control block of one solve (device).  Written by the solve's kernels; the host reads it only
// in the eager (non-graph) driver and never in the middle of a captured solve.
struct KrylovCtl {
  double tol, inner_tol, tol2;  // outer tolerance, inner reduction asked per sweep, (inner rel tol)^2
  int max_iter, max_sweeps, mixed;
  int sweep;                    // refinement sweeps done
  int passes, max_passes;       // inner iterations of this sweep and their bound
  int live;                     // active columns after the last decision
  int go;                       // 1 while another sweep is due
  unsigned int gticket;         // columns finished in the current launch
};
constexpr int KRYLOV_MAX_G = 32;  // blocks per column of the column kernels
// Device pointers of one solve's per-column state (passed by value to the kernels).  With graph
// set, the kernels set the WHILE conditions h_outer (refinement sweeps) and h_inner (CG iterations).
struct KrylovView {
  KrylovCtl* ctl = nullptr;
  double *bb = nullptr, *rr = nullptr, *rho = nullptr, *r0 = nullptr, *alpha = nullptr, *beta = nullptr,
         *res = nullptr;
  int *active = nullptr, *conv = nullptr, *iters = nullptr, *sweeps = nullptr;
  double2* part = nullptr;       // nr x G partial sums
  unsigned int* ticket = nullptr;  // nr per-column tickets
  const int* member = nullptr;   // batch sessions: 1 for the columns of running requests (null: all)
  int64_t n = 0;                 // rows (edges)
  int nr = 0, G = 1;
  int graph = 0;
  cudaGraphConditionalHandle h_outer = 0, h_inner = 0;
};
int krylov_blocks_per_column(int64_t n);
cudaError_t krylov_params(const KrylovView& K, double tol, double inner_tol, int max_iter, int max_sweeps, bool mixed,
                          cudaStream_t s);
// r = b - t and the sweep decision (init: r = b, i = 0, bb = ||b||^2, no t)
cudaError_t krylov_refine_residual(const KrylovView& K, const double2* b, const double2* t, double2* r, double2* i,
                                   bool init, cudaStream_t s);
cudaError_t krylov_cg_start(const KrylovView& K, const double2* r, double2* d, double2* rin, double2* p,
                            cudaStream_t s);
cudaError_t krylov_cg_pap(const KrylovView& K, const double2* p, const double2* Ap, cudaStream_t s);
cudaError_t krylov_cg_update(const KrylovView& K, const double2* p, const double2* Ap, double2* d, double2* rin,
                             cudaStream_t s);
cudaError_t krylov_cg_direction(const KrylovView& K, const double2* rin, double2* p, cudaStream_t s);
cudaError_t krylov_add(const KrylovView& K, const double2* d, double2* i, cudaStream_t s);
// the sweep decision alone (active mask, inner tolerance) from the current rr, bb, iters, sweeps
cudaError_t krylov_decide(const KrylovView& K, cudaStream_t s);
// batch admission: for the n new columns at slots[q] (device), bb = rr = dots[q].x, counters 0,
// member 1; for the n columns at slots[q] with dots == nullptr: member 0, bb = rr = 0 (a freed slot)
cudaError_t krylov_slots(const KrylovView& K, const int* slots, int n, const double2* dots, cudaStream_t s);

// Smoothed-aggregation multigrid hierarchy (host side, amg.cpp).
struct AmgLevelHost {
  int n = 0, nc = 0;       // rows of this level, rows of the next
  double omega = 0.0;      // Jacobi weight 4 / (3 rho)
  std::vector<double> diag;
  std::vector<int32_t> A_ptr, A_col, P_ptr, P_col, R_ptr, R_col;  // A (n x n), P (n x nc), R = P^T
  std::vector<double> A_val, P_val, R_val;
};
struct AmgHierarchy {
  std::vector<AmgLevelHost> levels;
  int coarse_n = 0;
  std::vector<double> coarse_inv;  // dense pseudo-inverse of the coarsest matrix
};
int build_amg(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col, const std::vector<double>& val, int n,
              int max_coarse, AmgHierarchy& H, std::string& err);

// Dense inverse of a sparse SPD matrix (or of the singular cell Laplacian restricted to 1^perp,
// with project = true: columns e_c - 1/n, result with zero column means = the pseudo-inverse),
// by block CG, preconditioned by one multigrid V(1,1) cycle when H is given.  A in CSR (device,
// n x n, FP64); output in FP32 hi + lo planes (n rows, padded_ld(n) stride).  Work buffers are
// allocated inside.  *iters receives the iteration count of the slowest column block.
// With Xd (and project), the result goes to Xd (FP64, n rows, padded_ld(n) stride) as
// X - colmean + 1/n, an approximation of (L + 1 1^T / n)^{-1}, instead of the FP32 planes.
cudaError_t dense_inverse_block_cg(const int32_t* ptr, const int32_t* col, const double* val, int n, bool project,
                                   const AmgHierarchy* H, double tol, int max_iter, float* Xhi, float* Xlo,
                                   int* iters, cudaStream_t s, double* Xd = nullptr);
// Newton-Schulz refinement of X ~ M^{-1} (k_factor.cu) for M = L + 1 1^T / n (project: writes
// (Sigma^T Sigma)^+ = sym(X) - 1 1^T / n) or M = L (writes sym(X)) to the FP32 hi + lo planes.
cudaError_t newton_schulz_pseudo_inverse(const int32_t* ptr, const int32_t* col, const double* val, int n,
                                         bool project, double* X, long long ldx, int max_steps, double tol, float* Xhi,
                                         float* Xlo, int* steps_done, double* final_residual, cudaStream_t s);
// X = c D^{-1} for the diagonal D of a CSR matrix (n x n, row stride ldx; the rest of X zeroed)
cudaError_t jacobi_start(const int32_t* ptr, const int32_t* col, const double* val, int n, double c, double* X,
                         long long ldx, cudaStream_t s);

}  // namespace rfcmp
