// Allocation-free application of T_A (rfcmp_apply_ta_noalloc in include/rfcmp.h).
//
// The paper has no counterpart: this entry point exists for callers that cannot allocate
// device memory at the point where they need a product with T_A -- a serving loop whose HBM
// was partitioned up front by its own pool, or a latency-critical path that must not call
// cudaMalloc/cudaFree because those calls can synchronise the device.  rfcmp_apply allocates
// the operator's work buffers lazily on first use; this variant never does: the GEMV scratch
// (x in FP32 hi/lo, the FP64 row accumulator) lives in the file-scope array below, which every
// GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "rfcmp_internal.h"

namespace rfcmp {

namespace {

// Capacity in complex entries: x (padded row length x columns) and y (rows x columns).
constexpr long long NOALLOC_MAX = 131072;
constexpr size_t NOALLOC_BYTES = (size_t)NOALLOC_MAX * (2 * sizeof(float2) + sizeof(double2));  // 4 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch per device ordinal, filled on the first call made with
// that device current.  In host code the symbol name is only a host-side stand-in.
constexpr int MAX_DEVICES = 64;
void* g_scratch_addr[MAX_DEVICES] = {};
std::mutex g_setup_mu;

int scratch_for_device(int dev, void** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return set_error(RFCMP_ERR_INVALID_ARG, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return set_error(RFCMP_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return RFCMP_OK;
}

}  // namespace

}  // namespace rfcmp

using namespace rfcmp;

extern "C" int rfcmp_apply_ta_noalloc(const rfcmp_op* op, const rfcmp_c128* x, rfcmp_c128* y, int64_t nrhs,
                                      void* stream) {
  OpTaView v;
  if (!op_ta_view(op, &v) || !x || !y) return set_error(RFCMP_ERR_INVALID_ARG, "NULL argument");
  if (nrhs < 1 || nrhs > 4) return set_error(RFCMP_ERR_INVALID_ARG, "nrhs must be 1 to 4");
  const long long ld = padded_ld(v.n);
  if (ld * nrhs > NOALLOC_MAX)
    return set_error(RFCMP_ERR_INVALID_ARG, "padded N x nrhs = " + std::to_string(ld * nrhs) +
                                                " exceeds the allocation-free scratch of 131072 complex entries");
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return set_error(RFCMP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (cur != v.device && (e = cudaSetDevice(v.device)) != cudaSuccess)
    return set_error(RFCMP_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  void* base = nullptr;
  int rc = scratch_for_device(v.device, &base);
  if (rc == RFCMP_OK) {
    unsigned char* b = static_cast<unsigned char*>(base);
    GemvScratch w;
    w.xh = reinterpret_cast<float2*>(b);
    w.xl = reinterpret_cast<float2*>(b + NOALLOC_MAX * sizeof(float2));
    // the GEMV runs column chunks of at most 4; each chunk uses ld x cols of x (hi and lo) and
    // adds its partial sums straight into y
    w.cap_cols = (int)nrhs;
    w.cap_ld = (int)(NOALLOC_MAX / nrhs);
    w.cap_n = w.cap_ld;
    e = gemv_c64_plain(v.TA, v.n, reinterpret_cast<const double2*>(x), reinterpret_cast<double2*>(y), (int)nrhs,
                       false, GEMV_FF, w, (cudaStream_t)stream);
    if (e != cudaSuccess) rc = set_error(RFCMP_ERR_CUDA, std::string("T_A product: ") + cudaGetErrorString(e));
  }
  if (cur != v.device) cudaSetDevice(cur);
  return rc;
}
