/*
 * rfcmp.h -- C ABI of the GB300 library for the RWG-discretised EFIE and the
 * refinement-free Calderon multiplicative preconditioner (RF-CMP) of
 * Adrian, Andriulli, Eibert, "On a refinement-free Calderon multiplicative
 * preconditioner for the electric field integral equation" (arXiv 1803.08333).
 *
 * Problem (Sec. 2): a PEC surface Gamma, triangulated, closed or open; RWG
 * functions f_n (not divided by the edge length, Eq. RWGdef) on the edges
 * shared by two cells (an edge of one cell is a boundary edge of an open
 * surface and carries none); loop functions on the interior vertices (every
 * vertex of a closed surface); wavenumber k; e^{-i w t};
 * current j normalised by the wave impedance.  With
 *   [T_A]_mn  = int int f_m(r) . f_n(r') G(r,r'),    G = e^{ikR}/(4 pi R),
 *   V_st      = int int p_s(r) p_t(r') G(r,r'),      p_s = 1/A_s on cell s,
 *   T_Phi     = Sigma V Sigma^T                       (Sec. 3, Eq. TPhiandV),
 *   T         = i k T_A + T_Phi / (i k),
 *   e_n       = int f_n . E^i,
 * the EFIE is T j = -e.  RF-CMP (Sec. 3 Eq. NewFormulation, with the
 * numerical variant of Sec. 4) solves the Hermitian positive definite system
 *   P_o^H T^H P_m T P_o i = -P_o^H T^H P_m e,   j = P_o i,
 *   P_o  = P_LH / alpha + i P_S / beta,
 *   P_m  = Lambda G_ll^{-1} Lambda^T / alpha^2 + P_LH / gamma
 *        + Sigma (Sigma^T Sigma)^+ G_pp^{-1} (Sigma^T Sigma)^+ Sigma^T / beta^2,
 *   P_S  = Sigma (Sigma^T Sigma)^+ Sigma^T,  P_LH = I - P_S      (Sec. 2),
 * by conjugate gradients (Sec. 4).
 *
 * Conventions shared by every entry point
 *  - Return value: 0 (RFCMP_OK) on success, a negative rfcmp_status otherwise;
 *    rfcmp_last_error() gives a message for the calling thread.
 *  - Mesh arrays are HOST pointers; the library copies them.  Triangles are
 *    int32 vertex triples, counter-clockwise about the outward normal.
 *  - Edge numbering: edges sorted by (smaller vertex id, larger vertex id);
 *    c_n^+ is the lower-index cell of edge n, c_n^- the other.
 *    Sigma[n, c^+] = +1, Sigma[n, c^-] = -1; with c^+ listed
 *    counter-clockwise as (v1, v2, r^+), Lambda[n, v1] = +1, Lambda[n, v2] = -1.
 *  - Vectors passed to apply / precondition / solve are DEVICE pointers to
 *    complex128 (rfcmp_c128), column-major with nrhs columns of length N
 *    (edges) unless stated otherwise; the caller owns them.  Work is queued
 *    on `stream` (a cudaStream_t, NULL = legacy default stream); entry points
 *    that return host results synchronise that stream.
 *  - An rfcmp_op is not thread-safe; different ops may be used from
 *    different threads.  rfcmp_ctx create/destroy are thread-safe.
 *  - Device memory of an op is allocated by the library on the context's
 *    device and counted against the context's HBM budget.  Allocations and
 *    frees are queued on the legacy default stream (a stream-ordered pool that
 *    keeps freed memory mapped), never with a host synchronisation: blocking
 *    streams are ordered with that stream by CUDA's rules; for a non-blocking
 *    stream an entry point makes it wait for the library's allocations, and
 *    memory an op frees waits for every non-blocking stream the op was used on.
 */
#ifndef RFCMP_H
#define RFCMP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest k times the diagonal of the vertices' bounding box that rfcmp_op_create accepts.  The
 * far-pair assembly (FP32) reduces k R by whole multiples of pi/2 with a product that stays exact
 * below 2^16 multiples (k R < 1.029e5); beyond this bound the phase would be silently wrong.  The
 * FP32 phase error itself grows as k R * 2^-24 (6e-3 rad at the bound). */
#define RFCMP_MAX_K_EXTENT 1.0e5

typedef struct rfcmp_ctx rfcmp_ctx;
typedef struct rfcmp_op rfcmp_op;
typedef struct { double re, im; } rfcmp_c128;

typedef enum {
  RFCMP_OK = 0,
  RFCMP_ERR_INVALID_ARG = -1,
  RFCMP_ERR_MESH_NOT_MANIFOLD = -2, /* an edge of three or more cells, a pinched boundary vertex, no
                                       interior vertex, or a bad index */
  RFCMP_ERR_MESH_ORIENTATION = -3,  /* neighbouring cells not consistently oriented */
  RFCMP_ERR_OUT_OF_BUDGET = -4,     /* the op would exceed the context's HBM budget */
  RFCMP_ERR_CUDA = -5,              /* a CUDA call failed (message in rfcmp_last_error) */
  RFCMP_ERR_DEVICE_TIMEOUT = -6,    /* a bounded device-side wait gave up */
  RFCMP_ERR_NOT_CONVERGED = -7,     /* only with rfcmp_solve_opts.fail_on_nonconvergence */
  RFCMP_ERR_NO_DEVICE = -8          /* no usable CUDA device of compute capability 10.3 */
} rfcmp_status;

/* which operator rfcmp_apply applies */
typedef enum {
  RFCMP_APPLY_T = 0,     /* y = T x = (i k T_A + Sigma V Sigma^T / (i k)) x          (Sec. 2) */
  RFCMP_APPLY_T_A = 1,   /* y = T_A x                                                 (Sec. 2) */
  RFCMP_APPLY_T_PHI = 2, /* y = Sigma V Sigma^T x                          (Sec. 3, Eq. TPhiandV) */
  RFCMP_APPLY_T_ADJ = 3, /* y = T^H x = conj(T conj(x))                    (Sec. 3.4, T^dagger) */
  RFCMP_APPLY_A = 4,     /* y = P_o^H T^H P_m T P_o x (low-frequency-stable order)   (Sec. 3, Sec. 4) */
  RFCMP_APPLY_A_INNER = 5 /* the same operator in the inner-iteration arithmetic of a MIXED solve:
                            FP32 products (FP32 GEMV, or the split-BF16 tensor-core GEMM from
                            rfcmp_plan.mrhs_min columns on); what the autotuner times */
} rfcmp_apply_which;

/* which preconditioner factor rfcmp_precondition applies */
typedef enum {
  RFCMP_PREC_P_O = 0,     /* P_o                 (Sec. 4, first display) */
  RFCMP_PREC_P_O_ADJ = 1, /* P_o^H */
  RFCMP_PREC_P_M = 2,     /* P_m = P_mL + P_mS   (Sec. 4, first display) */
  RFCMP_PREC_P_SIGMA = 3, /* P_S = Sigma (Sigma^T Sigma)^+ Sigma^T   (Sec. 2) */
  RFCMP_PREC_P_LAMBDAH = 4, /* P_LH = I - P_S                         (Sec. 2) */
  RFCMP_PREC_P_GSIGMA = 5   /* P_gS = Sigma (Sigma^T Sigma)^+ G_l~p^{-1} Sigma^T (Sec. 3, Eq. Pgs);
                               only for an op created with outer = RFCMP_OUTER_GSIGMA */
} rfcmp_prec_which;

/* the star part of the outer preconditioner P_o */
typedef enum {
  RFCMP_OUTER_SIGMA = 0,  /* P_o = P_LH / alpha + i P_S / beta (numerical variant, Sec. 4); the default */
  RFCMP_OUTER_GSIGMA = 1  /* P_o = P_LH / alpha + i P_gS / beta with P_gS of Eq. Pgs (Sec. 3) and the
                             mixed Gram matrix G_l~p of the dual piecewise linear functions and the
                             primal pulses (the case formula of Sec. 3); with RFCMP_SCALE_K this is
                             the formulation of Sec. 3, P_o = P_LH / sqrt k + i P_gS sqrt k.  The
                             current j = P_o i is the same; the conditioning differs */
} rfcmp_outer;

/* how alpha, beta, gamma are chosen */
typedef enum {
  RFCMP_SCALE_POWER = 0, /* norms of Sec. 4, second display, estimated iteratively (Lanczos); the default */
  RFCMP_SCALE_K = 1,     /* alpha = sqrt k, beta = 1/sqrt k, gamma = k (Sec. 4, third display) */
  RFCMP_SCALE_FIXED = 2  /* the values given in rfcmp_op_opts */
} rfcmp_scaling;

/* arithmetic of the solve */
typedef enum {
  RFCMP_PREC_MIXED = 0, /* FP32-data / FP32-accumulate inner CG, float-float residual refinement */
  RFCMP_PREC_FF = 1     /* every application float-float accurate (FP64-equivalent), no refinement */
} rfcmp_precision;

typedef struct {
  int32_t scaling;      /* rfcmp_scaling; default RFCMP_SCALE_POWER */
  int32_t power_steps;  /* maximum iteration steps for each norm (a Lanczos iteration whose largest
                           Ritz value converges to the spectral norm the power iteration of
                           Sec. 4 estimates); default 30 */
  double alpha, beta, gamma; /* used with RFCMP_SCALE_FIXED */
  double factor_tol;    /* accuracy of the dense-inverse builds of (Sigma^T Sigma)^+ and
                           G_ll^{-1}: relative residual per column for a block-CG build, largest
                           entry of I - M X (at least 1e-12, the FP64 rounding level of tens of
                           thousands of cells) for a Newton-Schulz refinement; default 1e-13 */
  double power_rtol;    /* a norm iteration stops once its estimate changes by at most power_rtol
                           (relative) between two steps, after at least 2 and at most power_steps
                           steps; 0 = always power_steps; default 1e-3 */
  const rfcmp_op* scaling_start; /* NULL, or an op on the same mesh: the norm iterations start
                           from its final Ritz vectors instead of the splitmix64 vectors (a
                           frequency sweep converges in a few steps); default NULL */
  int32_t outer;        /* rfcmp_outer; default RFCMP_OUTER_SIGMA.  RFCMP_OUTER_GSIGMA builds the
                           dense G_l~p^{-1} (N_C x N_C, FP32 hi + lo planes, cached per connectivity
                           in the context) at rfcmp_op_create */
  int32_t reserved[7];  /* must be zero */
} rfcmp_op_opts;

typedef struct {
  double tol;           /* stop when ||b - A i|| / ||b|| <= tol on the preconditioned system; default 1e-6 */
  int32_t max_iter;     /* total CG iterations per right-hand side, 1..1000000; default 2000 */
  int32_t max_refine;   /* refinement sweeps (MIXED), 0..1000; default 24 (a column stops at its own
                           tolerance: 2-3 sweeps at low frequency, 12 for 1024 plane waves at ka = 10
                           on 90750 unknowns, where split-BF16 inner products meet a harder system) */
  double inner_tol;     /* relative reduction asked of each inner CG (MIXED); default 1e-4 */
  int32_t precision;    /* rfcmp_precision; default RFCMP_PREC_MIXED */
  int32_t fail_on_nonconvergence; /* nonzero: return RFCMP_ERR_NOT_CONVERGED if any column fails */
  int32_t reserved[8];  /* must be zero */
} rfcmp_solve_opts;

typedef struct {
  int32_t converged;    /* 1 if the column reached tol */
  int32_t iterations;   /* CG iterations spent on this column (all sweeps) */
  int32_t refinements;  /* refinement sweeps (accurate residual evaluations) */
  int32_t reserved;
  double residual;      /* final ||b - A i|| / ||b||, float-float accurate */
} rfcmp_solve_report;

typedef struct {
  int64_t n_edges;     /* RWG functions N: the edges shared by two cells */
  int64_t n_vertices;  /* loop functions: the interior vertices (all vertices of a closed surface) */
  int64_t n_cells;
  int32_t genus;
  int32_t boundaries;  /* boundary curves of an open surface (0: closed) */
  double k, alpha, beta, gamma;
  uint64_t device_bytes;    /* device memory held by the op */
  double ms_assembly;       /* T_A and V assembly (device time) */
  double ms_factors;        /* dense (Sigma^T Sigma)^+ and G_ll^{-1} (0 when shared from the context cache) */
  double ms_scaling;        /* alpha, beta, gamma power iterations */
  int32_t factor_iterations_lplus; /* block-CG iterations of the (Sigma^T Sigma)^+ build */
  int32_t factor_iterations_gll;   /* block-CG iterations of the G_ll^{-1} build */
} rfcmp_op_info;

/* ----------------------------------------------------------------------------
 * Context: one CUDA device, an HBM budget, and a cache of the k-independent
 * topology factors ((Sigma^T Sigma)^+ depends on the mesh connectivity only,
 * G_ll^{-1} on the mesh geometry) shared by ops on the same mesh.
 *  device            CUDA ordinal; the device must be sm_103 (GB300).
 *  hbm_budget_bytes  upper bound on device memory held by all ops of this
 *                    context (0 = no bound).
 * Errors: RFCMP_ERR_INVALID_ARG, RFCMP_ERR_NO_DEVICE, RFCMP_ERR_CUDA.
 */
int rfcmp_ctx_create(int device, uint64_t hbm_budget_bytes, rfcmp_ctx** out);
/* Frees the factor cache.  Every op of the context must be destroyed first. */
int rfcmp_ctx_destroy(rfcmp_ctx* ctx);
/* Drops the cached topology factors (ops keep their own references). */
int rfcmp_ctx_clear_cache(rfcmp_ctx* ctx);
/* Bytes currently held by the ops and the cache of this context. */
uint64_t rfcmp_ctx_bytes_in_use(const rfcmp_ctx* ctx);

/* ----------------------------------------------------------------------------
 * Operator: mesh + wavenumber -> resident T_A (N x N) and V (N_C x N_C),
 * complex64, row-major (both complex symmetric); dense (Sigma^T Sigma)^+
 * (N_C x N_C) and G_ll^{-1} (N_V x N_V, the interior vertices) as FP32 hi + lo planes; alpha, beta,
 * gamma.  Assembly (Sec. 2 definitions): 7 x 7 product of the 7-point rule
 * on far cell pairs in FP32; on near pairs (a shared vertex) closed-form
 * integration of 1/(4 pi R) over the source cell plus the 7-point rule for
 * (e^{ikR} - 1)/(4 pi R), in FP64, averaged over both orders.
 *  verts  nv x 3 float64 (host: every mesh vertex), tris N_C x 3 int32 (host).  Open
 *         surfaces need at least one interior vertex; the theory variant (opts.outer =
 *         RFCMP_OUTER_GSIGMA) needs a closed surface (RFCMP_ERR_INVALID_ARG otherwise).
 *  k      wavenumber > 0 (rad/m, c = 1); k times the diagonal of the bounding box of verts at
 *         most RFCMP_MAX_K_EXTENT (RFCMP_ERR_INVALID_ARG otherwise).
 *  opts   NULL for the defaults.
 * All work runs on the context device's legacy default stream; the call
 * returns when the op is ready.
 * Errors: RFCMP_ERR_INVALID_ARG, RFCMP_ERR_MESH_NOT_MANIFOLD,
 * RFCMP_ERR_MESH_ORIENTATION, RFCMP_ERR_OUT_OF_BUDGET, RFCMP_ERR_CUDA.
 */
int rfcmp_op_create(rfcmp_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t nc,
                    double k, const rfcmp_op_opts* opts, rfcmp_op** out);
int rfcmp_op_info_get(const rfcmp_op* op, rfcmp_op_info* out);
int rfcmp_op_destroy(rfcmp_op* op);
/* Releases what op built for wide products (the BF16 planes of the tensor-core inner products,
 * the exact-digit planes of the accurate ones) and its solve workspace; the assembled T_A and V,
 * the shared factors and the scaling stay.  The next wide call rebuilds them.  The memory returns
 * to the pool behind the work already queued with op; the host does not wait.  (The paper has no
 * counterpart: memory management for resident operators.)
 * Errors: RFCMP_ERR_INVALID_ARG, RFCMP_ERR_CUDA. */
int rfcmp_op_trim(rfcmp_op* op);

/* Copies an internal matrix to a caller-owned DEVICE buffer of dst_bytes bytes.
 *  which 0: T_A, N x N complex64 row-major      (8 N^2 bytes)
 *        1: V, N_C x N_C complex64 row-major    (8 N_C^2 bytes)
 *        2: (Sigma^T Sigma)^+, N_C x N_C float64 (hi + lo)  (8 N_C^2 bytes)
 *        3: G_ll^{-1}, N_V x N_V float64 (hi + lo)         (8 N_V^2 bytes)
 *        4: G_l~p^{-1}, N_C x N_C float64 (hi + lo)        (8 N_C^2 bytes; RFCMP_OUTER_GSIGMA ops)
 * Errors: RFCMP_ERR_INVALID_ARG (unknown which, dst_bytes too small), RFCMP_ERR_CUDA. */
int rfcmp_op_export(const rfcmp_op* op, int which, void* dst, uint64_t dst_bytes, void* stream);

/* Topology read-back for tests: edge table in the library's numbering.
 *  edge_verts  N x 2 int32 (v1, v2)    edge_cells  N x 2 int32 (c^+, c^-)   (host, caller-owned) */
int rfcmp_op_edges(const rfcmp_op* op, int32_t* edge_verts, int32_t* edge_cells);

/* Plane-wave excitation e_n = int f_n . pol e^{i k khat . r} dS (Sec. 2), 7-point rule, FP64.
 *  khat, pol  nrhs x 3 float64 (host); khat unit vectors, pol real polarisations.
 *  e          DEVICE, N x nrhs complex128, column-major. */
int rfcmp_rhs_planewave(rfcmp_op* op, const double* khat, const double* pol, int64_t nrhs,
                        rfcmp_c128* e, void* stream);

/* Voltage-gap (delta-gap) excitation, the second excitation of the paper's Fokker experiment
 * (Sec. 4; the paper gives no formula).  Reading: an impressed field V delta(s) u across the
 * closed line of mesh edges cut by the plane through `origin` with normal `normal` -- the edges
 * whose two cells have their centroids on opposite sides -- u the in-surface normal of that line
 * towards the side `normal` points to.  The flux of an RWG function (Eq. RWGdef, no edge-length
 * factor) through its own edge is 1, so e_n = +V where c_n^+ lies on the negative side, -V where
 * it lies on the positive side, 0 off the gap (e = V Sigma chi, chi the indicator of the
 * negative side's cells).
 *  origin, normal  HOST 3 float64 each; normal nonzero (need not be unit length).
 *  e               DEVICE, N complex128 (one column).
 * Errors: RFCMP_ERR_INVALID_ARG (NULL, zero or non-finite plane), RFCMP_ERR_CUDA. */
int rfcmp_rhs_voltage_gap(rfcmp_op* op, const double* origin, const double* normal, rfcmp_c128 voltage,
                          rfcmp_c128* e, void* stream);

/* y = op(x) for nrhs columns (see rfcmp_apply_which).  Float-float accurate
 * accumulation over the stored complex64 matrices.  x and y must not alias. */
int rfcmp_apply(rfcmp_op* op, int which, const rfcmp_c128* x, rfcmp_c128* y, int64_t nrhs, void* stream);

/* y = P(x) (see rfcmp_prec_which); float-float accurate.  x and y must not alias. */
int rfcmp_precondition(rfcmp_op* op, int which, const rfcmp_c128* x, rfcmp_c128* y, int64_t nrhs,
                       void* stream);

/* Solves T j = -e through the RF-CMP system by CG (Sec. 4), nrhs columns.
 *  e  DEVICE N x nrhs; j DEVICE N x nrhs (output); report HOST nrhs entries (output, may be NULL).
 *  opts NULL for the defaults.  Synchronises `stream` before returning.
 * Errors: RFCMP_ERR_INVALID_ARG, RFCMP_ERR_CUDA, RFCMP_ERR_NOT_CONVERGED (opt-in). */
int rfcmp_solve(rfcmp_op* op, const rfcmp_c128* e, rfcmp_c128* j, int64_t nrhs, const rfcmp_solve_opts* opts,
                rfcmp_solve_report* report, void* stream);

/* The same solve with HOST e and j (copies inside the call; pinned memory is faster). */
int rfcmp_solve_host(rfcmp_op* op, const rfcmp_c128* e_host, rfcmp_c128* j_host, int64_t nrhs,
                     const rfcmp_solve_opts* opts, rfcmp_solve_report* report, void* stream);

/* ----------------------------------------------------------------------------
 * Batch sessions: continuous batching of one operator's solves (the paper has no counterpart;
 * the serving form of the solve above).  A session holds `capacity` column slots of one RF-CMP
 * CG solve with refinement; excitations are admitted into free slots at any time between
 * sweeps, every rfcmp_batch_step runs one refinement sweep (inner CG to the sweep's tolerance,
 * then the accurate residual) over all running columns together, and finished columns are
 * taken out one by one, freeing their slots for the next admissions.  A column's arithmetic is
 * that of rfcmp_solve (the same kernels, its own scalars and stopping test); columns that share
 * a sweep share the operator products.  The op must not be used by another call while a step
 * runs; a session keeps its own solve vectors (capacity x N complex128, several copies).
 */
typedef struct rfcmp_batch rfcmp_batch;
/* opts as for rfcmp_solve (NULL: defaults).  Errors: RFCMP_ERR_INVALID_ARG, RFCMP_ERR_CUDA. */
int rfcmp_batch_create(rfcmp_op* op, int32_t capacity, const rfcmp_solve_opts* opts, rfcmp_batch** out);
int rfcmp_batch_destroy(rfcmp_batch* b);
/* Admits n excitations e (DEVICE, N x n complex128, column-major) into free slots, whose
 * indices go to slots (HOST, n).  Errors: RFCMP_ERR_INVALID_ARG (fewer than n free slots). */
int rfcmp_batch_admit(rfcmp_batch* b, const rfcmp_c128* e, int32_t n, int32_t* slots, void* stream);
/* One refinement sweep over the running columns.  The slots whose column finished in this
 * sweep (converged, or out of iterations or sweeps) go to finished (HOST, up to capacity) and
 * their count to *n_finished.  Synchronises the stream. */
int rfcmp_batch_step(rfcmp_batch* b, int32_t* finished, int32_t* n_finished, void* stream);
/* Takes the columns of n finished slots (HOST list, no repeats): j = P_o i for all of them in one
 * application (DEVICE, N x n complex128, column-major, in the order of slots) and their reports
 * (HOST, n, may be NULL); the slots become free.  Synchronises the stream.
 * Errors: RFCMP_ERR_INVALID_ARG (a slot out of range, repeated, or without a finished column). */
int rfcmp_batch_take(rfcmp_batch* b, const int32_t* slots, int32_t n, rfcmp_c128* j, rfcmp_solve_report* reports,
                     void* stream);
/* Slots running, finished (not yet taken) and free; any pointer may be NULL. */
int rfcmp_batch_counts(const rfcmp_batch* b, int32_t* running, int32_t* finished, int32_t* free_slots);

/* Bistatic radar cross section sigma = (k^2 / 4 pi) |N - rhat (rhat . N)|^2,
 * N(rhat) = int j e^{-i k rhat . r} dS (7-point rule, FP64), in dBsm.
 *  j DEVICE N x nrhs; dirs HOST ndir x 3 unit vectors; rcs_dbsm HOST ndir x nrhs (column-major). */
int rfcmp_farfield(rfcmp_op* op, const rfcmp_c128* j, int64_t nrhs, const double* dirs, int64_t ndir,
                   double* rcs_dbsm, void* stream);

/* ----------------------------------------------------------------------------
 * D = A B^T (+ D) on the tensor cores in split BF16 (the engine of the multi-RHS products).
 * The paper has no counterpart; it is exported so the engine can be checked on its own.
 *  A  DEVICE float32, M x K row-major, row stride lda elements
 *  B  DEVICE float32, N x K row-major, row stride ldb elements
 *  D  DEVICE float32, M x N row-major, row stride ldd elements; accumulate != 0 adds to D
 * Each operand is split into two BF16 planes (hi = bf16(x), lo = bf16(x - hi)); every K step
 * accumulates hi*hi + hi*lo + lo*hi in FP32 (tcgen05.mma, tensor-memory accumulator), about
 * 2^-16 relative accuracy per product.  Temporary planes are allocated on `stream`.
 * Errors: RFCMP_ERR_INVALID_ARG, RFCMP_ERR_CUDA, RFCMP_ERR_DEVICE_TIMEOUT (a bounded wait of
 * the kernel gave up; the context stays usable). */
int rfcmp_gemm_bf16x3(const float* A, int64_t lda, const float* B, int64_t ldb, float* D, int64_t ldd, int64_t M,
                      int64_t N, int64_t K, int accumulate, void* stream);

/* ----------------------------------------------------------------------------
 * y = T_A x without allocating anything (the paper has no counterpart).
 * For callers that cannot allocate device memory where they need this product: a serving
 * loop whose HBM is partitioned up front by its own pool, or a latency-critical path that
 * must not call cudaMalloc/cudaFree, which can synchronise the device.  rfcmp_apply
 * allocates the operator's work buffers on first use; this entry point never does.  Its
 * scratch (x in FP32 hi/lo and an FP64 row accumulator, 4 MiB) is a file-scope device array
 * that every GPU which loads the library holds until the process exits.
 *  op     an operator created earlier (its T_A is read; nothing of op is modified)
 *  x, y   DEVICE, N x nrhs complex128, column-major; must not alias
 *  nrhs   1..4, with padded_N x nrhs <= 131072 (padded_N = N rounded up to a multiple of 64;
 *         N = 30720 allows nrhs <= 4, N = 90750 allows nrhs = 1)
 * Float-float accurate accumulation, like rfcmp_apply with RFCMP_APPLY_T_A.
 * The first call on each device (with the op's device current) looks up the scratch
 * address with cudaGetSymbolAddress; make that first call before any stream capture.
 * Every call shares the one scratch array (it is cleared where it must start at zero):
 * calls that overlap on the GPU race, so issue them on one stream or serialise them.
 * Errors: RFCMP_ERR_INVALID_ARG (NULL, nrhs or size beyond the limits), RFCMP_ERR_CUDA.
 */
int rfcmp_apply_ta_noalloc(const rfcmp_op* op, const rfcmp_c128* x, rfcmp_c128* y, int64_t nrhs, void* stream);

/* ----------------------------------------------------------------------------
 * Kernel plans (the paper has no counterpart; they choose launch shapes, never
 * arithmetic that changes a float-float result).  A zero field means the
 * built-in choice.  The autotuner measures candidates through rfcmp_apply
 * (RFCMP_APPLY_A_INNER) and keeps the best per (N, nrhs, precision).
 */
typedef struct {
  int32_t mrhs_min;         /* inner-iteration products of at least this many columns run on the
                               tensor cores (split-BF16 GEMM), narrower ones on the FP32 GEMV;
                               1..65536, default 4 */
  int32_t gemm_bn;          /* GEMM N tile: 32, 64 or 128 columns; default by column count */
  int32_t gemv_chunk;       /* register-pipelined GEMV work unit width in matrix columns: a multiple
                               of 256 in [256, 8192]; default 1024.  Nonzero (like gemv_ctas_per_sm)
                               selects that kernel also where the default is the streaming one (one
                               or two FP32 columns of the symmetric blocks, one float-float column
                               of T_A or V), whose shape is fixed */
  int32_t gemv_ctas_per_sm; /* persistent GEMV CTAs per SM, 1..8; default the occupancy maximum */
  int32_t far_min_blocks;   /* far-pair assembly CTAs per SM its registers are sized for: 1 to 4;
                               default 3 (read at rfcmp_op_create) */
  int32_t exact_min;        /* float-float accurate products of at least this many columns run as
                               exact-digit tensor-core products (each value as 6 signed 8-bit digits
                               under a power-of-two row scale, integer level sums exact in the FP32
                               accumulators; about 2^-48 of the row and column maxima per term),
                               narrower ones on the float-float GEMV; 1..65536, default 4 */
  int32_t reserved[2];      /* must be zero */
} rfcmp_plan;
/* Fills plan with zeros (every field at its built-in choice). */
void rfcmp_plan_default(rfcmp_plan* plan);
/* The plan that operators created afterwards in ctx start with.
 * Errors: RFCMP_ERR_INVALID_ARG (NULL ctx or a field out of range). */
int rfcmp_ctx_set_plan(rfcmp_ctx* ctx, const rfcmp_plan* plan);
/* Replaces the plan of op for its later calls (NULL: built-in choices).  Not thread-safe
 * against calls on the same op.  Errors: RFCMP_ERR_INVALID_ARG. */
int rfcmp_op_set_plan(rfcmp_op* op, const rfcmp_plan* plan);
int rfcmp_op_get_plan(const rfcmp_op* op, rfcmp_plan* out);

/* ----------------------------------------------------------------------------
 * Profiling counters (the paper has no counterpart; measurement support).
 * When enabled, every launch of an instrumented kernel family is bracketed by
 * CUDA events on the stream it is launched on; rfcmp_profile_read
 * synchronises the device and reports per family the launch count, the sum
 * of the event durations and the algorithmic bytes and FLOPs of those
 * launches (GEMV: the matrix plus the vectors it reads and writes; far-pair
 * assembly: 49 kernel evaluations per unique pair at 54 FLOPs each).
 */
typedef struct {
  char name[40];
  int64_t launches;
  double total_ms;
  double bytes;
  double flops;
} rfcmp_profile_entry;
/* Clears the counters; nonzero enables, zero disables. */
int rfcmp_profile_enable(int enable);
/* Copies up to max_entries families into out (host) and their number into *n_entries. */
int rfcmp_profile_read(rfcmp_profile_entry* out, int max_entries, int* n_entries);

/* Kernel launches of this library since it was loaded, over all devices of the process:
 * every kernel adds one to a device counter from its first block and thread.  Synchronises
 * the current device.  Errors: RFCMP_ERR_INVALID_ARG (out is NULL). */
int rfcmp_launch_count(uint64_t* out);

/* Device memory of the library's stream-ordered pool on the current device (the paper has no
 * counterpart: memory accounting for large operators): bytes in use now and at most since the
 * last reset, bytes the pool holds mapped now and at most.  Any pointer may be NULL.
 * rfcmp_pool_reset_high restarts both high-water marks.  Errors: RFCMP_ERR_CUDA. */
int rfcmp_pool_stats(uint64_t* used, uint64_t* used_high, uint64_t* reserved, uint64_t* reserved_high);
int rfcmp_pool_reset_high(void);
/* Hands the memory the pool holds but no buffer uses back to the driver (synchronises the device). */
int rfcmp_pool_trim(void);

/* How rfcmp_solve runs its loop (the paper has no counterpart; the arithmetic is the same
 * either way, so the results are identical).  Nonzero (the default, unless the environment
 * variable RFCMP_SOLVE_GRAPHS is "0" when the first solve starts): refinement sweeps and CG
 * iterations run as one CUDA graph per op with nested WHILE conditional nodes, whose conditions
 * the solve's own kernels set on the device (convergence test, active-column mask, inner
 * tolerance); the host launches it and synchronises once per solve.  The graph is captured on
 * the op's first solve of a shape and reused while the shape, the op's buffers, its plan and the
 * profiling state stay the same.  Zero: the same kernels launched one by one, the host reading
 * the device's decision after every iteration.  Process-wide; returns the previous setting. */
int rfcmp_set_solve_graphs(int enable);

const char* rfcmp_strerror(int status);
const char* rfcmp_last_error(void);

/* Fills opts with the defaults documented above. */
void rfcmp_op_opts_default(rfcmp_op_opts* opts);
void rfcmp_solve_opts_default(rfcmp_solve_opts* opts);

/* ----------------------------------------------------------------------------
 * Compressed operators (Sec. 4: the system matrix compressed by an adaptive cross
 * approximation at tolerance 1e-4; at extremely low frequency the vector potential stored and
 * compressed apart from the scalar potential).  T_A (RWG functions) and V (cells) each become a
 * symmetric hierarchical matrix: a cluster tree of the index set (recursive bisection at the
 * middle position of the items sorted along the largest extent of their centres; an item's
 * support box spans the vertices of its cells), the blocks of the block tree on and above the
 * block diagonal, an admissible block (min(diam a, diam b) <= eta * dist(a, b) > 0 for the two
 * clusters' boxes, which couples only cells that share no vertex) stored as rank-r crosses
 * U^T Vt found by ACA with partial pivoting on the device (stop after the cross whose size
 * ||u|| ||v|| is at most eps ||S_r||_F) when r (m + n) < m n, every other block dense.  A block off the diagonal also
 * stands for its transpose below it, so the compressed T_A and V stay exactly complex symmetric.
 * The compressed form is built from an op's resident dense T_A and V (the op remains valid and
 * unchanged); assembling the compressed form without the dense matrices is not provided.
 */
typedef struct rfcmp_hm rfcmp_hm;

typedef enum {
  RFCMP_HM_T_A = 0, /* the vector-potential block T_A (N x N) */
  RFCMP_HM_V = 1    /* the scalar-potential block V (N_C x N_C) */
} rfcmp_hm_which;

typedef struct {
  double eps;        /* ACA stopping tolerance per block, in (0, 1) (default 1e-4, the paper's) */
  double eta;        /* admissibility parameter > 0 (default 1) */
  int32_t leaf;      /* largest cluster that is not split, in [8, 1024] (default 32) */
  int32_t max_rank;  /* crosses per block, in [1, 256] (default 64); an admissible block whose
                        crosses reach it without meeting the stopping rule is stored dense */
  int32_t reserved[6];  /* must be zero */
} rfcmp_hm_opts;

typedef struct {
  int64_t n[2];               /* rows of T_A (N) and V (N_C), indexed by rfcmp_hm_which */
  int64_t lowrank_blocks[2];  /* blocks stored as crosses (on and above the block diagonal) */
  int64_t dense_blocks[2];    /* blocks stored dense, capped ones included */
  int64_t capped_blocks[2];   /* admissible blocks the rank cap left dense */
  int64_t small_blocks[2];    /* admissible blocks stored dense because their crosses would take
                                 at least the block's own entries (rank (m + n) >= m n) */
  int64_t bytes[2];           /* device bytes of each compressed matrix */
  int32_t max_rank[2];        /* largest rank of a low-rank block */
  int32_t reserved[6];
} rfcmp_hm_info;

void rfcmp_hm_opts_default(rfcmp_hm_opts* opts);

/* Host only (no device work): the cluster tree and the symmetric block list of n items.
 *  centres, sup_lo, sup_hi  n x 3 float64 each (host): item centres and support boxes.
 *  leaf, eta                as in rfcmp_hm_opts (leaf in [1, 65536], eta >= 0).
 *  perm       n int32 (host, caller-owned): cluster order -> item index.
 *  blocks     5 int32 per block (host, caller-owned) or NULL to query the count: r0, r1, c0, c1
 *             (half-open ranges of the cluster order, r0 <= c0) and 1 if admissible else 0,
 *             ordered by (r0, c0); capacity = blocks the array holds.
 *  n_blocks   receives the number of blocks.
 * Errors: RFCMP_ERR_INVALID_ARG (NULL, non-finite coordinates, argument out of range, capacity
 * too small). */
int rfcmp_hm_partition(const double* centres, const double* sup_lo, const double* sup_hi, int64_t n, int32_t leaf,
                       double eta, int32_t* perm, int32_t* blocks, int64_t capacity, int64_t* n_blocks);

/* Compresses op's T_A and V (opts NULL for the defaults).  Runs on the context device's legacy
 * default stream and returns when the compressed form is ready.  Its bytes count against the
 * context's budget; destroy it before the context.
 * Errors: RFCMP_ERR_INVALID_ARG, RFCMP_ERR_OUT_OF_BUDGET (the build's peak: the crosses' slots
 * and, at worst, every block dense), RFCMP_ERR_CUDA. */
int rfcmp_hm_create(rfcmp_op* op, const rfcmp_hm_opts* opts, rfcmp_hm** out);

/* y = H x for nrhs columns, H the compressed T_A or V (which), FP32 factors with FP64
 * accumulation.  x, y DEVICE, n x nrhs complex128 column-major (n = N or N_C), not aliased;
 * nrhs in [1, 65535]; stream NULL for the legacy default stream.  Several streams may run
 * products of one hm at once.  Errors: RFCMP_ERR_INVALID_ARG, RFCMP_ERR_CUDA. */
int rfcmp_hm_apply(rfcmp_hm* hm, int which, const rfcmp_c128* x, rfcmp_c128* y, int64_t nrhs, void* stream);

/* Block counts, ranks and bytes of both compressed matrices.  Errors: RFCMP_ERR_INVALID_ARG. */
int rfcmp_hm_info_get(const rfcmp_hm* hm, rfcmp_hm_info* out);

/* Frees the compressed form after the products queued on its streams. */
int rfcmp_hm_destroy(rfcmp_hm* hm);

#ifdef __cplusplus
}
#endif
#endif /* RFCMP_H */
