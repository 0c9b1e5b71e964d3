// xcorr_noalloc.cu -- a one-shot 4-bit correlation that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need a
// correlation.  A real-time capture loop is one: cudaMalloc and cudaFree may
// synchronise the whole device, and that stalls the streams that are draining
// the network into the ring buffers.  A process whose device memory is owned
// by another framework's fixed pool is another.  For them this file offers one
// entry point, xcorr_correlate_ci4_noalloc.  It runs the same tensor-core
// X-stage as a plan (the unpack into E4M3 planes, then the tcgen05 kernel),
// but its staging planes live in a fixed array that is part of the library's
// device image: kScratchBytes on every GPU that loads the library, held until
// the process exits.  The caller still provides the input and the output.
#include <mutex>
#include <string>

#include "xcorr_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB per device
constexpr size_t kStatusBytes = 256;               // kernel status word, then the planes

// The scratch array.  In host code this name is only a stand-in for the
// device object: the kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

// The array's device address belongs to the module as loaded in one CUDA context: after a
// cudaDeviceReset, or in a caller's own driver-API context, the module is loaded again and the
// array sits elsewhere.  So the address is cached per device together with the context it was
// looked up in, and looked up again on every call whose stream is not being captured (a cheap
// runtime call); a stream under capture reuses the address cached for this device and context.
struct ScratchEntry {
  CUcontext ctx = nullptr;
  void* addr = nullptr;
};
std::mutex g_scratch_mu;
ScratchEntry g_scratch[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

xcorr_status current_context(CUcontext* out) {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  if (!fn) return xc::set_error(XCORR_ERR_CUDA, "cuCtxGetCurrent is not available from the driver");
  if (fn(out) != CUDA_SUCCESS) return xc::set_error(XCORR_ERR_CUDA, "cuCtxGetCurrent failed");
  return XCORR_OK;
}

// Device address of the scratch array for the current device and context.
xcorr_status scratch_address(cudaStream_t stream, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return xc::set_error(XCORR_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return xc::set_error(XCORR_ERR_UNSUPPORTED, "device ordinal above 63");
  CUcontext ctx = nullptr;
  xcorr_status st = current_context(&ctx);
  if (st != XCORR_OK) return st;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
    cudaGetLastError();  // the query itself is refused while another stream captures: keep the cache
    cs = cudaStreamCaptureStatusActive;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchEntry& en = g_scratch[dev];
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return xc::set_error(XCORR_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") +
                                               cudaGetErrorString(e));
    en.ctx = ctx;
    en.addr = p;
  } else if (!en.addr || en.ctx != ctx) {
    return xc::set_error(XCORR_ERR_INVALID_ARG,
                         "the stream is being captured and this device and context have no scratch address yet: "
                         "make one call outside the capture first");
  }
  *out = en.addr;
  return XCORR_OK;
}

}  // namespace

extern "C" xcorr_status xcorr_correlate_ci4_noalloc(const void* d_in, int n_time, int n_channels,
                                                    int n_stations, void* d_out, int* d_status,
                                                    void* stream) {
  if (!d_in || !d_out) return xc::set_error(XCORR_ERR_INVALID_ARG, "d_in and d_out must not be NULL");
  if (n_time < 1 || n_channels < 1 || n_stations < 1)
    return xc::set_error(XCORR_ERR_INVALID_ARG, "n_time, n_channels and n_stations must be >= 1");
  if (n_time > xc::kMaxIntegrationCI4)
    return xc::set_error(XCORR_ERR_OVERFLOW, "n_time exceeds the exact int32 bound of 16,777,215 samples");
  if (n_stations > (1 << 20))
    return xc::set_error(XCORR_ERR_INVALID_ARG, "n_stations must be at most 2^20");
  const int n_inputs = 2 * n_stations;
  const int ni_pad = (n_inputs + 15) / 16 * 16;
  const size_t planes = size_t(2) * size_t(n_channels) * size_t(n_time) * size_t(ni_pad);
  if (planes > kScratchBytes - kStatusBytes)
    return xc::set_error(XCORR_ERR_INVALID_ARG,
                         "this correlation needs " + std::to_string(planes) +
                             " bytes of staging planes (2 * n_channels * n_time * N_i rounded up to 16); "
                             "the fixed scratch array holds " +
                             std::to_string(kScratchBytes - kStatusBytes) + " bytes: use a plan instead");
  int dev = 0, major = 0, minor = 0, n_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return xc::set_error(XCORR_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
  if (major != 10 || minor != 3) return xc::set_error(XCORR_ERR_UNSUPPORTED, "needs an sm_103a (GB300) device");

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  xcorr_status st = scratch_address(s, &scratch);
  if (st != XCORR_OK) return st;
  int* status = static_cast<int*>(scratch);
  uint8_t* plane_buf = static_cast<uint8_t*>(scratch) + kStatusBytes;

  // The array keeps the previous call's contents: the status word must start at zero.
  // (The planes need no clearing: the unpack writes every element the X kernel reads.)
  e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e != cudaSuccess) return xc::set_error(XCORR_ERR_CUDA, std::string("status clear: ") + cudaGetErrorString(e));
  e = xc::launch_unpack_ci4_e4m3(static_cast<const uint8_t*>(d_in), plane_buf, n_time, n_channels, n_inputs, ni_pad,
                                 n_time, n_sms, s);
  if (e != cudaSuccess) return xc::set_error(XCORR_ERR_CUDA, std::string("unpack launch: ") + cudaGetErrorString(e));
  CUtensorMap tmap;
  std::string err;
  if (!xc::encode_plane_tmap(&tmap, plane_buf, 1, n_inputs, ni_pad, n_time, n_time, 2 * n_channels,
                             xc::tc_stage_samples(1, 0), &err))
    return xc::set_error(XCORR_ERR_CUDA, err);
  xc::TcLaunch L;
  L.elem_bytes = 1;
  L.variant = 0;
  L.n_time = n_time;
  L.chan0 = 0;
  L.n_chan = n_channels;
  L.n_inputs = n_inputs;
  L.window_samples = xc::kTcWindowCI4;
  L.accumulate = false;
  L.out = d_out;
  L.status = status;
  L.num_sms = n_sms;
  e = xc::launch_xcorr_tc(&tmap, L, s);
  if (e != cudaSuccess)
    return xc::set_error(XCORR_ERR_CUDA, std::string("X kernel launch: ") + cudaGetErrorString(e));
  if (d_status) {
    e = cudaMemcpyAsync(d_status, status, sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return xc::set_error(XCORR_ERR_CUDA, std::string("status copy: ") + cudaGetErrorString(e));
  }
  return XCORR_OK;
}
