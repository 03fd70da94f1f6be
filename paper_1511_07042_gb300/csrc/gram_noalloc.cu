// bmg_gram_noalloc: the tall-skinny Gram product G = X^T Y without any device
// allocation.
//
// bmg_gram obtains the buffer for its per-block partial sums from cudaMalloc on
// every call (and frees it again, which also waits for the device).  Some callers
// cannot do that: a host framework that has reserved all device memory for its own
// pool, a service that runs under a fixed device-memory budget, or a caller on a
// path where the implicit device-wide wait of cudaFree is not acceptable.  For them
// this entry point keeps the partial sums in one fixed array compiled into the
// library (kScratchDoubles doubles, 4 MiB), which every GPU that loads the library
// holds until the process exits.  The caller still provides X, Y and G.
//
// The array is shared by every call in the process.  Its contents are fully
// rewritten by each call before they are read, so nothing needs clearing, but two
// calls whose work overlaps on the GPU (for instance on two streams) race on it and
// give wrong results: order such calls on one stream or synchronise between them.
#include <mutex>

#include "common.cuh"

namespace bmg {
namespace {

constexpr size_t kScratchDoubles = size_t(1) << 19;   // 4 MiB of partial sums
static_assert(160 * 160 <= kScratchDoubles, "one k x k partial of the largest block fits the array");
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_gram_scratch[kScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_gram_scratch on the current device, looked up once per device
// (the host-side symbol is only a handle, not a device address).
double* scratch_for_current_device() {
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) fail(BMG_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    check_cuda(cudaGetSymbolAddress(&p, g_gram_scratch), "cudaGetSymbolAddress(g_gram_scratch)");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  return g_scratch_ptr[dev];
}

}  // namespace
}  // namespace bmg

using namespace bmg;

extern "C" bmg_status bmg_gram_noalloc(const double* X, const double* Y, int n, int k, int ld, double* G,
                                       void* stream) {
  try {
    if (!X || !Y || !G) fail(BMG_ERR_INVALID_ARG, "bmg_gram_noalloc: null pointer");
    if (n < 1 || k < 1 || ld < k || ld > kGramMaxLd)
      fail(BMG_ERR_INVALID_ARG, "bmg_gram_noalloc: need n >= 1 and 1 <= k <= ld <= 800");
    if (k > 160)
      fail(BMG_ERR_INVALID_ARG, "bmg_gram_noalloc: k = " + std::to_string(k) +
                                    " exceeds the maximum of 160 supported by the Gram kernel");
    const size_t kk = (size_t)k * k;
    double* scratch = scratch_for_current_device();
    // The array bounds the number of row blocks that run in parallel, not k: each
    // block keeps a k x k partial, so k = 160 allows 20 blocks (where bmg_gram runs up
    // to 304) and each block then sums n / 20 rows.
    int parts = gram_parts(n);
    const int cap = (int)(kScratchDoubles / kk);
    if (parts > cap) parts = cap;
    gram(X, Y, n, k, ld, G, scratch, parts, (cudaStream_t)stream);
    return BMG_OK;
  } catch (const BmgException& e) {
    set_error(e.msg);
    return e.code;
  } catch (...) {
    set_error("bmg_gram_noalloc: unexpected failure");
    return BMG_ERR_CUDA;
  }
}
