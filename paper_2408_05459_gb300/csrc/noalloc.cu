// ancka_discretize_noalloc: Discretize that allocates no device memory.
//
// Some callers cannot allocate device memory while they run: real-time or
// safety-critical code that reserves all memory at start-up and has no
// failure path for an allocation later; programs where another allocator
// (a framework's caching allocator, a memory pool sized to the whole GPU)
// already owns nearly all device memory, so a cudaMalloc would fail; and
// latency-critical loops that avoid cudaMalloc/cudaFree because freeing
// synchronises the device.  For them this entry point keeps Discretize's
// scratch -- the row-normalised copy of the block, per-CTA partial sums and
// the k x k state -- in the fixed device array below, sized when the library
// is built.  Every GPU that loads the library holds the array until the
// process exits.
//
// The first call on a device looks up the array's device address (a CUDA
// runtime query, no allocation), so make that first call before any stream
// capture.  Every call waits for its stream before returning: it reads the
// inner-iteration count and an error flag back to the host.  All calls
// share the one array and leave their contents in it;
// each call resets the state it needs, but two calls whose work overlaps on
// the GPU (different streams, or different host threads) race on it.
#include <mutex>

#include "common.cuh"

// 32 MiB of scratch per device, shared by every call of this entry point.
static constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_discretize_scratch[kNoAllocScratchBytes];

namespace ancka {
namespace {

std::mutex g_scratch_mu;
void* g_scratch_ptr[64] = {nullptr};

// Device address of the scratch array on the current device.  The host-side
// name g_discretize_scratch is only a stand-in, so the address is looked up
// once per device (with that device current) and cached.
ancka_status scratch_for_current_device(void** out) {
  int dev = 0;
  ANCKA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return ANCKA_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_discretize_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return ANCKA_OK;
}

}  // namespace
}  // namespace ancka

extern "C" ancka_status ancka_discretize_noalloc(const float* Qk, int64_t n, int32_t k, int32_t ldq,
                                                 int32_t max_iter, int32_t* labels, int32_t* iters,
                                                 void* stream) {
  using namespace ancka;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ANCKA_TRY(ancka_device_check());
  if (!Qk || !labels) {
    set_error("Qk or labels is NULL");
    return ANCKA_ERR_INVALID_ARG;
  }
  if (n < 1 || n >= (int64_t(1) << 31) - 1 || k < 1 || k > 64 || ldq < k || max_iter < 1 || max_iter > 1000) {
    set_error("ancka_discretize_noalloc: need 1 <= n < 2^31-1, 1 <= k <= 64, ldq >= k, 1 <= max_iter <= 1000");
    return ANCKA_ERR_INVALID_ARG;
  }
  const size_t need = discretize_scratch_bytes(n, k);
  if (need > kNoAllocScratchBytes) {
    set_error("ancka_discretize_noalloc: n = %lld, k = %d needs %zu bytes of scratch, more than the fixed %zu "
              "(about n * round_up(k, 4) * 4 bytes); use ancka_discretize",
              (long long)n, k, need, kNoAllocScratchBytes);
    return ANCKA_ERR_INVALID_ARG;
  }
  void* scratch = nullptr;
  ANCKA_TRY(scratch_for_current_device(&scratch));
  int32_t* it_dev = nullptr;
  int32_t* err_dev = nullptr;
  ANCKA_TRY(discretize_scratch(scratch, kNoAllocScratchBytes, Qk, n, k, ldq, max_iter, labels, &it_dev, &err_dev, s));
  int32_t hit = 0, he = 0;
  ANCKA_CUDA(cudaMemcpyAsync(&hit, it_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaMemcpyAsync(&he, err_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaStreamSynchronize(s));
  if (he) {
    set_error("ancka_discretize_noalloc: a grid barrier wait expired");
    return ANCKA_ERR_TIMEOUT;
  }
  if (iters) *iters = hit;
  return ANCKA_OK;
}
