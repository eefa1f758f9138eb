// sw_selftest_wait: the library's bounded device waits, made to run out.
// Every wait between warps or CTAs in the kernels gives up after a clock
// budget, reports SW_ETIMEOUT and returns, so that a failure leaves the CUDA
// context usable.  This entry point runs the two wait helpers the kernels use
// against a condition that nothing fulfils, so that a test can check that
// they give up and report it, without faulting or hanging a GPU.
#include <cstdio>

#include "devutil.cuh"
#include "internal.h"
#include "../../include/swgb.h"

namespace swgb {
namespace {

__global__ void wait_selftest_kernel(int which, long long budget, const int32_t *flag, int32_t *status) {
  __shared__ uint64_t bar;
  if (which == 0) {
    // a progress counter that nothing raises (the pair-band kernel's waits)
    const int32_t v = wait_flag_value(flag, 1, budget);
    *status = v >= 1 ? SW_OK : SW_ETIMEOUT;
  } else {
    // an mbarrier phase that nothing completes (the profile-chunk waits of
    // the inter- and intra-task kernels; their fixed budget of ~1 s)
    mbar_init(&bar, 1);
    fence_mbar_init();
    *status = mbar_wait_bounded(&bar, 0u) ? SW_OK : SW_ETIMEOUT;
  }
}

int st_fail(int code, const char *msg) { return set_last_error(code, msg); }

int st_cuda(cudaError_t e, const char *what) {
  char buf[256];
  snprintf(buf, sizeof buf, "sw_selftest_wait: %s: %s", what, cudaGetErrorString(e));
  return set_last_error(e == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, buf);
}

}  // namespace
}  // namespace swgb

using namespace swgb;

extern "C" int sw_selftest_wait(int32_t which, int64_t budget_cycles, int32_t *status_out, void *stream) {
  clear_last_error();
  if (!status_out) return st_fail(SW_EINVAL, "sw_selftest_wait: null status_out");
  if (which != 0 && which != 1) return st_fail(SW_EINVAL, "sw_selftest_wait: which must be 0 or 1");
  if (which == 0 && (budget_cycles <= 0 || budget_cycles > ((int64_t)1 << 32)))
    return st_fail(SW_EINVAL, "sw_selftest_wait: budget_cycles must lie in (0, 2^32]");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t *d = nullptr;  // [0] the flag, [1] the status
  cudaError_t e = cudaMallocAsync((void **)&d, 2 * sizeof(int32_t), s);
  if (e != cudaSuccess) return st_cuda(e, "device allocation");
  e = cudaMemsetAsync(d, 0, 2 * sizeof(int32_t), s);
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 1, 0, s>>>(which, (long long)budget_cycles, d, d + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(status_out, d + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return st_cuda(e, "run");
  return SW_OK;
}
