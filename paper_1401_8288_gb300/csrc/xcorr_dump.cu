// xcorr_dump.cu -- the cross-dump accumulation: the GPU integrates K samples
// per dump and further integration happens downstream (Sec. 2.4, Sec. 4: 1024
// spectra on the GPU, then 119 more on the CPU).  Here that downstream sum is
// kept exact on the device: each dump's int32 integration is widened and added
// into a caller-owned int64 buffer.
#include "xcorr_internal.h"

namespace xc {
namespace {

__global__ void __launch_bounds__(256) fold_wide_i64_kernel(const int4* __restrict__ acc,
                                                            longlong2* __restrict__ out, int64_t n4) {
  // one int4 of the accumulator = two (re, im) pairs = two longlong2 of the output
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int4 a = __ldg(acc + q);
    longlong2 o0 = out[2 * q], o1 = out[2 * q + 1];
    o0.x += a.x;
    o0.y += a.y;
    o1.x += a.z;
    o1.y += a.w;
    out[2 * q] = o0;
    out[2 * q + 1] = o1;
  }
}

__global__ void fold_wide_i64_tail(const int2* __restrict__ acc, longlong2* __restrict__ out, int64_t first,
                                   int64_t n) {
  const int64_t q = first + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < n) {
    longlong2 o = out[q];
    o.x += acc[q].x;
    o.y += acc[q].y;
    out[q] = o;
  }
}

// Float visibilities: widen each dump into a double running sum, the FP64
// cross-dump accumulation for integrations longer than one FP32 dump.
__global__ void __launch_bounds__(256) fold_wide_f64_kernel(const float2* __restrict__ acc,
                                                            double2* __restrict__ out, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = __ldg(acc + q);
    double2 o = out[q];
    o.x += a.x;
    o.y += a.y;
    out[q] = o;
  }
}

}  // namespace

cudaError_t launch_fold_wide_f64(const float2* acc, double* out, int64_t n_pairs_total, cudaStream_t stream) {
  int64_t blocks = (n_pairs_total + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  if (blocks < 1) blocks = 1;
  fold_wide_f64_kernel<<<(unsigned)blocks, 256, 0, stream>>>(acc, reinterpret_cast<double2*>(out), n_pairs_total);
  return cudaGetLastError();
}

cudaError_t launch_fold_wide_i64(const int2* acc, int64_t* out, int64_t n_pairs_total, cudaStream_t stream) {
  const int64_t n4 = n_pairs_total / 2;
  if (n4 > 0) {
    int64_t blocks = (n4 + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    fold_wide_i64_kernel<<<(unsigned)blocks, 256, 0, stream>>>(reinterpret_cast<const int4*>(acc),
                                                               reinterpret_cast<longlong2*>(out), n4);
  }
  if (n_pairs_total % 2)
    fold_wide_i64_tail<<<1, 32, 0, stream>>>(acc, reinterpret_cast<longlong2*>(out), 2 * n4, n_pairs_total);
  return cudaGetLastError();
}

}  // namespace xc
