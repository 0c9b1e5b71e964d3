// xcorr_unpack.cu -- the unpack step of Sec. 2.4 ("pads the data from four to
// eight bits" and completes the corner turn, Fig. 5), GB300 style.
//
// Input: 4+4-bit complex samples [time][channel][input] (input = 2*station+pol).
// Output: two planes per channel, real and imaginary, each [time][input] of
// E4M3 codes: plane (c, comp) row t holds the N_i inputs of time t.  Every
// 4-bit code in [-8, 7] is exactly representable in E4M3, so the tensor-core
// X kernel multiplies the true integers.  The planes stay input-contiguous:
// the X kernel reads them as MN-major operands, so the tensor memory access
// itself performs the transpose of the corner turn and this kernel is a pure
// element-wise decode with 128-bit loads and stores.
#include <cudaTypedefs.h>

#include <cstring>

#include "xcorr_internal.h"

namespace xc {
namespace {

// E4M3 codes of 0..7 and of -8..-1, four per word, lowest byte first.
constexpr uint32_t kPos0 = 0x44403800u;  // 0, 1, 2, 3
constexpr uint32_t kPos1 = 0x4E4C4A48u;  // 4, 5, 6, 7
constexpr uint32_t kNeg0 = 0xCACCCED0u;  // -8, -7, -6, -5
constexpr uint32_t kNeg1 = 0xB8C0C4C8u;  // -4, -3, -2, -1

// Byte-wise table lookup: `lo3` holds a 3-bit index in the low bits of each
// byte, `neg` is 0xFF in the bytes whose 4-bit code is negative.
__device__ __forceinline__ uint32_t e4m3_of_nibbles(uint32_t lo3, uint32_t neg) {
  uint32_t sel = lo3 | (lo3 >> 4);                  // pack the four indices into 16 bits
  sel = (sel & 0xFFu) | ((sel >> 8) & 0xFF00u);
  const uint32_t pos = __byte_perm(kPos0, kPos1, sel);
  const uint32_t ngt = __byte_perm(kNeg0, kNeg1, sel);
  return (ngt & neg) | (pos & ~neg);
}

// Four CI4 samples (one per byte) -> four E4M3 real parts and four imaginary parts.
__device__ __forceinline__ void ci4_to_e4m3(uint32_t v, uint32_t& re, uint32_t& im) {
  re = e4m3_of_nibbles((v >> 4) & 0x07070707u, ((v >> 7) & 0x01010101u) * 0xFFu);
  im = e4m3_of_nibbles(v & 0x07070707u, ((v >> 3) & 0x01010101u) * 0xFFu);
}

// Channels [c0, c0 + nc) of every time row, 16 inputs per thread (N_i a
// multiple of 16 and a 16-byte aligned input); grid-stride over the rows.
__global__ void __launch_bounds__(256) unpack_ci4_e4m3_vec(const uint8_t* __restrict__ in,
                                                           uint8_t* __restrict__ planes, int64_t n_rows,
                                                           int n_chan, int c0, int nc, int q_per_row,
                                                           int ni_pad, int64_t comp_stride) {
  const int64_t total = n_rows * q_per_row;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = q / q_per_row;  // row = t * nc + (c - c0)
    const int k = static_cast<int>(q - row * q_per_row);
    const int64_t t = row / nc;
    const int c = c0 + static_cast<int>(row - t * nc);
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(in + ((t * n_chan + c) * q_per_row + k) * 16));
    uint4 r, m;
    ci4_to_e4m3(v.x, r.x, m.x);
    ci4_to_e4m3(v.y, r.y, m.y);
    ci4_to_e4m3(v.z, r.z, m.z);
    ci4_to_e4m3(v.w, r.w, m.w);
    uint8_t* dst = planes + (2 * (int64_t)c) * comp_stride + t * ni_pad + 16 * (int64_t)k;
    *reinterpret_cast<uint4*>(dst) = r;
    *reinterpret_cast<uint4*>(dst + comp_stride) = m;
  }
}

// Any input count and alignment: one byte per thread.
__global__ void __launch_bounds__(256) unpack_ci4_e4m3_byte(const uint8_t* __restrict__ in,
                                                            uint8_t* __restrict__ planes,
                                                            int64_t n_rows, int n_chan, int c0, int nc,
                                                            int n_inputs, int ni_pad, int64_t comp_stride) {
  const int64_t total = n_rows * n_inputs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = q / n_inputs;
    const int i = static_cast<int>(q - row * n_inputs);
    const int64_t t = row / nc;
    const int c = c0 + static_cast<int>(row - t * nc);
    uint32_t re, im;
    ci4_to_e4m3(in[(t * n_chan + c) * n_inputs + i], re, im);
    uint8_t* dst = planes + (2 * (int64_t)c) * comp_stride + t * ni_pad + i;
    dst[0] = static_cast<uint8_t>(re);
    dst[comp_stride] = static_cast<uint8_t>(im);
  }
}

}  // namespace

cudaError_t launch_unpack_ci4_e4m3_channels(const uint8_t* in, uint8_t* planes, int n_time, int n_chan,
                                            int c0, int nc, int n_inputs, int ni_pad, int max_time,
                                            int num_sms, cudaStream_t stream) {
  const int64_t n_rows = (int64_t)n_time * nc;
  const int64_t comp_stride = (int64_t)max_time * ni_pad;
  const int threads = 256;
  const bool vec = (n_inputs % 16 == 0) && (reinterpret_cast<uintptr_t>(in) % 16 == 0);
  const int64_t work = vec ? n_rows * (n_inputs / 16) : n_rows * n_inputs;
  int64_t blocks = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (vec)
    unpack_ci4_e4m3_vec<<<(unsigned)blocks, threads, 0, stream>>>(in, planes, n_rows, n_chan, c0, nc,
                                                                 n_inputs / 16, ni_pad, comp_stride);
  else
    unpack_ci4_e4m3_byte<<<(unsigned)blocks, threads, 0, stream>>>(in, planes, n_rows, n_chan, c0, nc,
                                                                  n_inputs, ni_pad, comp_stride);
  return cudaGetLastError();
}

cudaError_t launch_unpack_ci4_e4m3(const uint8_t* in, uint8_t* planes, int n_time, int n_chan,
                                   int n_inputs, int ni_pad, int max_time, int num_sms,
                                   cudaStream_t stream) {
  return launch_unpack_ci4_e4m3_channels(in, planes, n_time, n_chan, 0, n_chan, n_inputs, ni_pad, max_time,
                                         num_sms, stream);
}

// ------------------------------------------------------------ tensor map ---
namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled_fn(std::string* err) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      if (err) *err = "cuTensorMapEncodeTiled is not available from the driver";
      return nullptr;
    }
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}
}  // namespace

bool encode_plane_tmap(CUtensorMap* map, void* planes, int n_inputs, int ni_pad, int n_time,
                       int max_time, int n_chan, std::string* err) {
  auto fn = encode_tiled_fn(err);
  if (!fn) return false;
  std::memset(map, 0, sizeof(*map));
  // dim0: input (contiguous), dim1: time, dim2: channel * 2 + component.  Rows
  // past n_inputs and times past n_time read as zeros.
  cuuint64_t dims[3] = {(cuuint64_t)n_inputs, (cuuint64_t)n_time, (cuuint64_t)n_chan * 2};
  cuuint64_t strides[2] = {(cuuint64_t)ni_pad, (cuuint64_t)ni_pad * (cuuint64_t)max_time};
  cuuint32_t box[3] = {128, (cuuint32_t)kTcStageT, 1};
  cuuint32_t elem_strides[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, planes, dims, strides, box, elem_strides,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r);
    return false;
  }
  return true;
}

}  // namespace xc
