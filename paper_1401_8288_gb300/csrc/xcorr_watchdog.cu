// xcorr_watchdog.cu -- a self-test of the failure path of the bounded waits.
//
// Every wait in the library's kernels is bounded: a wait that runs out raises
// the CTA's abort flag, records a code in the plan's status word and lets the
// kernel return, so a stalled pipeline surfaces as XCORR_ERR_DEVICE instead of
// a hung GPU.  This kernel exercises exactly that path with a wait that can
// never complete (an mbarrier nothing arrives at), so a deployment or a test
// can check it without any real fault.
#include "sm103_ptx.cuh"
#include "xcorr_internal.h"

namespace xc {
namespace {

__global__ void watchdog_selftest_kernel(int* status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // one arrival would complete phase 0; none ever comes
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0, &abort_flag, status, DEV_TIMEOUT_FULL);
}

}  // namespace
}  // namespace xc

extern "C" xcorr_status xcorr_watchdog_selftest(xcorr_plan plan, void* stream) {
  xcorr_status st = xc::plan_check(plan);
  if (st != XCORR_OK) return st;
  xc::watchdog_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(plan->status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return xc::set_error(XCORR_ERR_CUDA, std::string("watchdog kernel: ") + cudaGetErrorString(e));
  return XCORR_OK;
}
