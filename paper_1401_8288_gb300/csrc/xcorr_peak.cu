// xcorr_peak.cu -- measured dense arithmetic rates of this device, used to
// state the X kernels' fraction of peak.  Each probe keeps its operands on
// chip (shared memory or registers) so only the arithmetic pipe is timed:
//   kind 0: tcgen05 kind::f8f6f4 E4M3 x E4M3 -> F32, M = 128, N = 256
//   kind 1: tcgen05 kind::f16 BF16 x BF16 -> F32, M = 128, N = 256
//   kind 2: the int8 tensor path GB300 offers, warp-level mma.sync m16n8k32 s8
//   kind 3: the CUDA-core int8 dot product (dp4a)
// One CTA per SM, timed with CUDA events after a warm-up launch.
#include <cuda_runtime.h>

#include "sm103_ptx.cuh"
#include "xcorr_internal.h"

namespace xc {
namespace {

template <bool E4M3>
__global__ void __launch_bounds__(128, 1) tc_rate_kernel(int iters, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t done;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x / 32;
  if (threadIdx.x == 0) {
    mbar_init(&done, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&tslot, 256);
  // small finite operand values (bytes <= 0x3F are finite in E4M3 and BF16)
  for (int k = threadIdx.x; k < 384 * 128; k += blockDim.x) sm[k] = static_cast<uint8_t>((k * 7) & 0x3F);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (threadIdx.x == 0) {
    const uint32_t id = instr_desc(E4M3 ? kTypeE4M3 : kTypeBF16, false, 128, 256, false);
    const uint64_t a = smem_desc_sw128(smem_u32(sm), 16, 1024);
    const uint64_t b = smem_desc_sw128(smem_u32(sm + 128 * 128), 16, 1024);
    for (int r = 0; r < iters; ++r) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (E4M3)
          mma_f8f6f4(tmem, a + 2 * k, b + 2 * k, id, (r | k) != 0);
        else
          mma_f16(tmem, a + 2 * k, b + 2 * k, id, (r | k) != 0);
      }
    }
    mma_commit(&done);
  }
  __syncthreads();
  volatile int never = 0;
  mbar_wait(&done, 0, &never, status, DEV_TIMEOUT_DRAIN);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

__global__ void __launch_bounds__(256) mma_sync_s8_rate_kernel(int iters, int* sink) {
  uint32_t a0 = 0x01020304u ^ threadIdx.x, a1 = 0x05060708u, a2 = 0x0102F3F4u, a3 = 0x7F800101u ^ blockIdx.x;
  uint32_t b0 = 0x11223344u, b1 = 0x0A0B0C0Du ^ threadIdx.x;
  int c[8][4] = {};
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+r"(c[q][0]), "+r"(c[q][1]), "+r"(c[q][2]), "+r"(c[q][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  int s = 0;
  for (int q = 0; q < 8; ++q) s += c[q][0] + c[q][1] + c[q][2] + c[q][3];
  if (s == 0x7FFFFFFF) sink[0] = s;
}

__global__ void __launch_bounds__(256) dp4a_rate_kernel(int iters, int* sink) {
  int a[8], c[8] = {};
  int b = 0x01020304 ^ static_cast<int>(threadIdx.x);
  for (int q = 0; q < 8; ++q) a[q] = (0x05060708 * (q + 1)) ^ static_cast<int>(blockIdx.x);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] = __dp4a(a[q], b, c[q]);
    b = __dp4a(b, b, b) | 1;
  }
  int s = 0;
  for (int q = 0; q < 8; ++q) s += c[q];
  if (s == 0x7FFFFFFF) sink[0] = s;
}

}  // namespace
}  // namespace xc

extern "C" xcorr_status xcorr_measure_peak(int kind, double* tops) {
  using namespace xc;
  if (!tops || kind < 0 || kind > 3) return XCORR_ERR_INVALID_ARG;
  *tops = 0.0;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int* buf = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&buf, 256);
  if (e == cudaSuccess) e = cudaMemset(buf, 0, 256);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int smem = 160 * 1024;  // one CTA per SM for the tcgen05 probes
  if (e == cudaSuccess && kind == 0)
    e = cudaFuncSetAttribute(tc_rate_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess && kind == 1)
    e = cudaFuncSetAttribute(tc_rate_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int iters = kind <= 1 ? 4000 : (kind == 2 ? 20000 : 100000);
  const int blocks = kind <= 1 ? nsm : 4 * nsm;
  auto launch = [&](int it) {
    if (kind == 0) tc_rate_kernel<true><<<blocks, 128, smem>>>(it, buf);
    else if (kind == 1) tc_rate_kernel<false><<<blocks, 128, smem>>>(it, buf);
    else if (kind == 2) mma_sync_s8_rate_kernel<<<blocks, 256>>>(it, buf);
    else dp4a_rate_kernel<<<blocks, 256>>>(it, buf);
  };
  float best = 1e30f;
  if (e == cudaSuccess) {
    launch(iters / 10);
    e = cudaDeviceSynchronize();
  }
  for (int rep = 0; e == cudaSuccess && rep < 3; ++rep) {
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) best = ms;
  }
  int code = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&code, buf, sizeof(int), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (e != cudaSuccess) return XCORR_ERR_CUDA;
  if (code != 0) return XCORR_ERR_DEVICE;
  double ops;
  if (kind <= 1) ops = 2.0 * 128 * 256 * (kind == 0 ? 32 : 16) * 4.0 * iters * blocks;
  else if (kind == 2) ops = 2.0 * 16 * 8 * 32 * 8.0 * iters * blocks * 8;  // 8 warps x 8 chains
  else ops = 8.0 * 9 * (double)iters * blocks * 256;                      // 9 dp4a per iteration
  *tops = ops / (best * 1e-3) / 1e12;
  return XCORR_OK;
}
