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
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "ci4_decode.cuh"
#include "xcorr_internal.h"

namespace xc {
namespace {

// Channels [c0, c0 + nc) of every time row, 16 inputs per thread (N_i a
// multiple of 16 and a 16-byte aligned input); grid-stride over the rows.
// Idx is the type of the flat index: 32-bit whenever the work fits, since the
// two divisions per 16 bytes cost several times more in 64-bit arithmetic.
template <typename Idx>
__global__ void __launch_bounds__(256) unpack_ci4_e4m3_vec(const uint8_t* __restrict__ in,
                                                           uint8_t* __restrict__ planes, int64_t n_rows,
                                                           int n_chan, int c0, int nc, int q_per_row,
                                                           int ni_pad, int64_t comp_stride) {
  const Idx total = static_cast<Idx>(n_rows * q_per_row);
  for (Idx q = blockIdx.x * static_cast<Idx>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<Idx>(gridDim.x) * blockDim.x) {
    const Idx row = q / static_cast<Idx>(q_per_row);  // row = t * nc + (c - c0)
    const int k = static_cast<int>(q - row * q_per_row);
    const int64_t t = static_cast<int64_t>(row / static_cast<Idx>(nc));
    const int c = c0 + static_cast<int>(row - static_cast<Idx>(t) * nc);
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
  const bool idx32 = work + (int64_t)blocks * threads < (INT64_C(1) << 32);
  if (vec && idx32)
    unpack_ci4_e4m3_vec<uint32_t><<<(unsigned)blocks, threads, 0, stream>>>(in, planes, n_rows, n_chan, c0, nc,
                                                                           n_inputs / 16, ni_pad, comp_stride);
  else if (vec)
    unpack_ci4_e4m3_vec<int64_t><<<(unsigned)blocks, threads, 0, stream>>>(in, planes, n_rows, n_chan, c0, nc,
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

bool encode_plane_tmap(CUtensorMap* map, void* planes, int elem_bytes, int n_inputs, int ni_pad,
                       int n_time, int max_time, int n_planes_total, int box_t, std::string* err) {
  auto fn = encode_tiled_fn(err);
  if (!fn) return false;
  std::memset(map, 0, sizeof(*map));
  // dim0: input (contiguous), dim1: time, dim2: channel * planes + plane.  Inputs
  // past n_inputs and times past n_time read as zeros.
  const cuuint64_t row = (cuuint64_t)ni_pad * elem_bytes;
  cuuint64_t dims[3] = {(cuuint64_t)n_inputs, (cuuint64_t)n_time, (cuuint64_t)n_planes_total};
  cuuint64_t strides[2] = {row, row * (cuuint64_t)max_time};
  cuuint32_t box[3] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_t, 1};
  cuuint32_t elem_strides[3] = {1, 1, 1};
  CUresult r = fn(map, elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, planes,
                  dims, strides, box, elem_strides, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r);
    return false;
  }
  return true;
}

namespace {
// The raw-input maps are pure functions of their arguments and are rebuilt by every execute;
// the last few are kept per host thread, so that an execute that repeats an earlier one (the
// usual case: the same buffer every integration) skips the driver's encode.
struct RawMapMemo {
  const void* in = nullptr;
  int n_inputs = 0, n_chan = 0, row_chans = 0, n_time = 0, box_t = 0, box_i = 0, packed = -1;
  CUtensorMap map;
};
constexpr int kRawMapMemo = 4;
thread_local RawMapMemo t_raw_memo[kRawMapMemo];
thread_local int t_raw_memo_next = 0;

RawMapMemo* raw_memo_find(const void* in, int n_inputs, int n_chan, int row_chans, int n_time, int box_t, int box_i,
                          int packed) {
  for (RawMapMemo& m : t_raw_memo)
    if (m.packed == packed && m.in == in && m.n_inputs == n_inputs && m.n_chan == n_chan &&
        m.row_chans == row_chans && m.n_time == n_time && m.box_t == box_t && m.box_i == box_i)
      return &m;
  return nullptr;
}

void raw_memo_put(const CUtensorMap& map, const void* in, int n_inputs, int n_chan, int row_chans, int n_time,
                  int box_t, int box_i, int packed) {
  RawMapMemo& m = t_raw_memo[t_raw_memo_next];
  t_raw_memo_next = (t_raw_memo_next + 1) % kRawMapMemo;
  m.in = in;
  m.n_inputs = n_inputs;
  m.n_chan = n_chan;
  m.row_chans = row_chans;
  m.n_time = n_time;
  m.box_t = box_t;
  m.box_i = box_i;
  m.packed = packed;
  m.map = map;
}

}  // namespace

bool encode_raw_ci4_tmap(CUtensorMap* map, const void* in, int n_inputs, int n_chan, int row_chans, int n_time,
                         int box_t, std::string* err, int box_i) {
  if (const RawMapMemo* m = raw_memo_find(in, n_inputs, n_chan, row_chans, n_time, box_t, box_i, 0)) {
    *map = m->map;
    return true;
  }
  auto fn = encode_tiled_fn(err);
  if (!fn) return false;
  std::memset(map, 0, sizeof(*map));
  if (box_i != 128 && box_i != 64) {
    if (err) *err = "raw input box must be 128 or 64 inputs wide";
    return false;
  }
  // the caller's [t][c][i] bytes: dim0 input, dim1 channel, dim2 time; a box is
  // box_i inputs x 1 channel x box_t samples = box_t rows of box_i bytes, swizzled
  // at the row width (128- or 64-byte pattern)
  cuuint64_t dims[3] = {(cuuint64_t)n_inputs, (cuuint64_t)n_chan, (cuuint64_t)n_time};
  cuuint64_t strides[2] = {(cuuint64_t)n_inputs, (cuuint64_t)n_inputs * (cuuint64_t)row_chans};
  cuuint32_t box[3] = {(cuuint32_t)box_i, 1, (cuuint32_t)box_t};
  cuuint32_t elem_strides[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(in), dims, strides, box, elem_strides,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, box_i == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled (raw input) failed with CUresult " + std::to_string((int)r);
    return false;
  }
  raw_memo_put(*map, in, n_inputs, n_chan, row_chans, n_time, box_t, box_i, 0);
  return true;
}

bool encode_raw_ci4_packed_tmap(CUtensorMap* map, const void* in, int n_inputs, int n_chan, int row_chans,
                                int n_time, int box_t, std::string* err) {
  if (const RawMapMemo* m = raw_memo_find(in, n_inputs, n_chan, row_chans, n_time, box_t, 128, 1)) {
    *map = m->map;
    return true;
  }
  auto fn = encode_tiled_fn(err);
  if (!fn) return false;
  std::memset(map, 0, sizeof(*map));
  // the caller's [t][c][i] bytes with channel and input merged into one dimension of n_chan *
  // n_inputs bytes (dim0), an extent-1 dimension (dim1, so that the kernels' 3-D loads serve),
  // and time (dim2); a box is box_t rows of 128 bytes, consecutive channels side by side
  const cuuint64_t row = (cuuint64_t)n_inputs * (cuuint64_t)row_chans;
  cuuint64_t dims[3] = {(cuuint64_t)n_inputs * (cuuint64_t)n_chan, 1, (cuuint64_t)n_time};
  cuuint64_t strides[2] = {row, row};
  cuuint32_t box[3] = {128, 1, (cuuint32_t)box_t};
  cuuint32_t elem_strides[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(in), dims, strides, box, elem_strides,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled (packed raw input) failed with CUresult " + std::to_string((int)r);
    return false;
  }
  raw_memo_put(*map, in, n_inputs, n_chan, row_chans, n_time, box_t, 128, 1);
  return true;
}

// ----------------------------------------------------- int8 and float input --
namespace {

__device__ __forceinline__ uint32_t bf16_bits(float f) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(f)));
}

// Eight int8 samples (16 bytes: re, im interleaved) -> eight BF16 real parts
// and eight imaginary parts, exact (|v| <= 128 needs 8 significant bits).
// Idx as for unpack_ci4_e4m3_vec.
template <typename Idx>
__global__ void __launch_bounds__(256) unpack_ci8_bf16_vec(const int8_t* __restrict__ in,
                                                           uint16_t* __restrict__ planes, int64_t n_rows,
                                                           int n_chan, int c0, int nc, int q_per_row,
                                                           int ni_pad, int64_t comp_stride) {
  const Idx total = static_cast<Idx>(n_rows * q_per_row);
  for (Idx q = blockIdx.x * static_cast<Idx>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<Idx>(gridDim.x) * blockDim.x) {
    const Idx row = q / static_cast<Idx>(q_per_row);
    const int k = static_cast<int>(q - row * q_per_row);
    const int64_t t = static_cast<int64_t>(row / static_cast<Idx>(nc));
    const int c = c0 + static_cast<int>(row - static_cast<Idx>(t) * nc);
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(in + ((t * n_chan + c) * q_per_row + k) * 16));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t re[4], im[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {  // word h holds samples 2h, 2h + 1: re0 im0 re1 im1
      const float r0 = static_cast<float>(static_cast<int8_t>(w[h] & 0xFF));
      const float i0 = static_cast<float>(static_cast<int8_t>((w[h] >> 8) & 0xFF));
      const float r1 = static_cast<float>(static_cast<int8_t>((w[h] >> 16) & 0xFF));
      const float i1 = static_cast<float>(static_cast<int8_t>(w[h] >> 24));
      re[h] = bf16_bits(r0) | (bf16_bits(r1) << 16);
      im[h] = bf16_bits(i0) | (bf16_bits(i1) << 16);
    }
    uint16_t* dst = planes + (2 * (int64_t)c) * comp_stride + t * ni_pad + 8 * (int64_t)k;
    *reinterpret_cast<uint4*>(dst) = make_uint4(re[0], re[1], re[2], re[3]);
    *reinterpret_cast<uint4*>(dst + comp_stride) = make_uint4(im[0], im[1], im[2], im[3]);
  }
}

__global__ void __launch_bounds__(256) unpack_ci8_bf16_elem(const int8_t* __restrict__ in,
                                                            uint16_t* __restrict__ planes, int64_t n_rows,
                                                            int n_chan, int c0, int nc, int n_inputs,
                                                            int ni_pad, int64_t comp_stride) {
  const int64_t total = n_rows * n_inputs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = q / n_inputs;
    const int i = static_cast<int>(q - row * n_inputs);
    const int64_t t = row / nc;
    const int c = c0 + static_cast<int>(row - t * nc);
    const int64_t s = (t * n_chan + c) * n_inputs + i;
    uint16_t* dst = planes + (2 * (int64_t)c) * comp_stride + t * ni_pad + i;
    dst[0] = static_cast<uint16_t>(bf16_bits(static_cast<float>(in[2 * s])));
    dst[comp_stride] = static_cast<uint16_t>(bf16_bits(static_cast<float>(in[2 * s + 1])));
  }
}

// Float input, one thread per (channel, window, input): find the window's
// largest magnitude max < 2^(E+1), quantise each component to the integer
// M = rint(x 2^(22-E)) (|M| < 2^23, error <= 2^-23 max), and write the
// balanced base-256 digits of M = d0 2^16 + d1 2^8 + d2 (|d_p| <= 128, exact
// BF16 values) to planes re_p = p and im_p = 3 + p.  E goes to exps.
//
// Edges.  The maximum is taken over the components' bit patterns with the
// sign cleared: for non-negative floats they order as the values do, and the
// patterns of infinities and NaNs lie above every finite one, so one integer
// maximum also finds a non-finite sample.  Such a window gets E =
// kExpNonFinite and zero digits; the X kernel's drain turns every block that
// involves it into NaN.  A window whose maximum is subnormal gets that
// maximum's own exponent (down to -149), so its samples keep 23-bit integers
// like any other window's and no finite input is flushed.  2^(22-E) spans
// 2^-105 .. 2^171, past the float range, so it is applied as two exact
// power-of-two factors.
__device__ __forceinline__ uint32_t abs_bits(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }

__device__ __forceinline__ int window_exponent(uint32_t max_bits) {
  if (max_bits >= 0x7F800000u) return kExpNonFinite;
  if (max_bits >= 0x00800000u) return static_cast<int>(max_bits >> 23) - 127;  // normal
  if (max_bits == 0u) return kExpMin;
  return (31 - __clz(static_cast<int>(max_bits))) - 149;  // subnormal m 2^-149: floor(log2 m) - 149
}

// The two factors of 2^(22 - e), each in [2^-53, 2^86]; zero for a non-finite window.
__device__ __forceinline__ void window_scale(int e, float& s1, float& s2) {
  if (e == kExpNonFinite) {
    s1 = s2 = 0.f;
    return;
  }
  const int n = 22 - e, a = n >> 1;
  s1 = pow2i(a);
  s2 = pow2i(n - a);
}

__device__ __forceinline__ void digits_of(float x, float s1, float s2, uint16_t (&d)[3]) {
  const int m = __float2int_rn((x * s1) * s2);
  const int d2 = ((m + 128) & 255) - 128;
  const int m1 = (m - d2) >> 8;
  const int d1 = ((m1 + 128) & 255) - 128;
  const int d0 = (m1 - d1) >> 8;
  d[0] = __bfloat16_as_ushort(__float2bfloat16_rn(static_cast<float>(d0)));
  d[1] = __bfloat16_as_ushort(__float2bfloat16_rn(static_cast<float>(d1)));
  d[2] = __bfloat16_as_ushort(__float2bfloat16_rn(static_cast<float>(d2)));
}

// Any 4-byte aligned input: the components are read as single floats.
__global__ void __launch_bounds__(256) unpack_cf32_digits_kernel(const float* __restrict__ in,
                                                                 uint16_t* __restrict__ planes,
                                                                 int16_t* __restrict__ exps, int n_time, int n_chan,
                                                                 int c0, int nc, int n_inputs, int ni_pad,
                                                                 int64_t comp_stride, int window, int exp_windows) {
  const int n_w = (n_time + window - 1) / window;
  const int64_t total = (int64_t)nc * n_w * n_inputs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = static_cast<int>(q % n_inputs);
    const int64_t rest = q / n_inputs;
    const int w = static_cast<int>(rest % n_w);
    const int c = c0 + static_cast<int>(rest / n_w);
    const int t0 = w * window, t1 = min(n_time, t0 + window);
    uint32_t mb = 0u;
#pragma unroll 8
    for (int t = t0; t < t1; ++t) {
      const float* v = in + 2 * (((int64_t)t * n_chan + c) * n_inputs + i);
      mb = max(mb, max(abs_bits(__ldg(v)), abs_bits(__ldg(v + 1))));
    }
    const int e = window_exponent(mb);
    exps[((int64_t)c * exp_windows + w) * ni_pad + i] = static_cast<int16_t>(e);
    float s1, s2;
    window_scale(e, s1, s2);
    uint16_t* base = planes + (6 * (int64_t)c) * comp_stride + i;
#pragma unroll 4
    for (int t = t0; t < t1; ++t) {
      const float* v = in + 2 * (((int64_t)t * n_chan + c) * n_inputs + i);
      uint16_t dr[3], dm[3];
      digits_of(__ldg(v), s1, s2, dr);
      digits_of(__ldg(v + 1), s1, s2, dm);
      uint16_t* row = base + (int64_t)t * ni_pad;
#pragma unroll
      for (int pc = 0; pc < 3; ++pc) {
        row[pc * comp_stride] = dr[pc];
        row[(3 + pc) * comp_stride] = dm[pc];
      }
    }
  }
}

// As unpack_cf32_digits_kernel for two neighbouring inputs per thread (an even
// input count and a 16-byte aligned input): 16-byte loads of (re, im) pairs and
// 4-byte stores of two digits, half the instructions per byte.
__global__ void __launch_bounds__(256) unpack_cf32_digits_x2_kernel(const float4* __restrict__ in,
                                                                    uint16_t* __restrict__ planes,
                                                                    int16_t* __restrict__ exps, int n_time,
                                                                    int n_chan, int c0, int nc, int n_inputs,
                                                                    int ni_pad, int64_t comp_stride, int window,
                                                                    int exp_windows) {
  const int n_w = (n_time + window - 1) / window;
  const int half = n_inputs / 2;
  const int64_t total = (int64_t)nc * n_w * half;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i2 = static_cast<int>(q % half);
    const int64_t rest = q / half;
    const int w = static_cast<int>(rest % n_w);
    const int c = c0 + static_cast<int>(rest / n_w);
    const int t0 = w * window, t1 = min(n_time, t0 + window);
    const float4* col = in + (int64_t)c * half + i2;  // inputs 2 i2, 2 i2 + 1 of channel c, time 0
    const int64_t row_step = (int64_t)n_chan * half;  // float4s from one sample to the next
    uint32_t mb0 = 0u, mb1 = 0u;
#pragma unroll 8
    for (int t = t0; t < t1; ++t) {
      const float4 v = __ldg(col + t * row_step);
      mb0 = max(mb0, max(abs_bits(v.x), abs_bits(v.y)));
      mb1 = max(mb1, max(abs_bits(v.z), abs_bits(v.w)));
    }
    const int e0 = window_exponent(mb0), e1 = window_exponent(mb1);
    int16_t* ex = exps + ((int64_t)c * exp_windows + w) * ni_pad + 2 * i2;
    ex[0] = static_cast<int16_t>(e0);
    ex[1] = static_cast<int16_t>(e1);
    float s0a, s0b, s1a, s1b;
    window_scale(e0, s0a, s0b);
    window_scale(e1, s1a, s1b);
    uint32_t* base = reinterpret_cast<uint32_t*>(planes + (6 * (int64_t)c) * comp_stride + 2 * i2);
    const int64_t cs = comp_stride / 2;  // in uint32 units (comp_stride is a multiple of 16)
#pragma unroll 4
    for (int t = t0; t < t1; ++t) {
      const float4 v = __ldg(col + t * row_step);
      uint16_t r0[3], m0[3], r1[3], m1[3];
      digits_of(v.x, s0a, s0b, r0);
      digits_of(v.y, s0a, s0b, m0);
      digits_of(v.z, s1a, s1b, r1);
      digits_of(v.w, s1a, s1b, m1);
      uint32_t* row = base + (int64_t)t * (ni_pad / 2);
#pragma unroll
      for (int pc = 0; pc < 3; ++pc) {
        row[pc * cs] = r0[pc] | (static_cast<uint32_t>(r1[pc]) << 16);
        row[(3 + pc) * cs] = m0[pc] | (static_cast<uint32_t>(m1[pc]) << 16);
      }
    }
  }
}

// Float input read once: a CTA stages one (channel, window, 32 inputs) slice -- the window's
// samples x 32 inputs x 8 bytes, 96 KB for a 384-sample window -- in shared memory with 16-byte
// asynchronous copies (each time row of the slice is 256 contiguous bytes), takes each input's window maximum
// from it, then writes the digits from it.  The two-read kernels above read every float twice
// from HBM: with a CTA per (channel, window, 256 input pairs) the slices in flight far exceed
// L2.  Here two CTAs of 256 threads share an SM, so one loads while the other converts.  Thread
// (pair q, time group g) handles inputs 2q, 2q + 1 of the slice at samples g, g + 16, ...; a warp
// covers two time rows of 16 pairs (512 contiguous bytes), conflict-free.  Needs n_inputs % 32
// == 0 and a 16-byte aligned input; same arithmetic as the other kernels, so the same results.
constexpr int kTileInputs = 32;
constexpr int kTilePairs = kTileInputs / 2;
constexpr int kTileGroups = 16;
constexpr int kTileThreads = kTilePairs * kTileGroups;
__global__ void __launch_bounds__(kTileThreads, 2) unpack_cf32_digits_tile_kernel(
    const float4* __restrict__ in, uint16_t* __restrict__ planes, int16_t* __restrict__ exps, int n_time, int n_chan,
    int c0, int nc, int n_inputs, int ni_pad, int64_t comp_stride, int window, int exp_windows) {
  extern __shared__ float4 slice[];  // [window][kTilePairs]
  __shared__ uint32_t part[2][kTileGroups][kTilePairs];
  __shared__ int win_e[2][kTilePairs];
  const int n_w = (n_time + window - 1) / window;
  const int n_groups = n_inputs / kTileInputs;
  const int half = n_inputs / 2;
  const int q = threadIdx.x % kTilePairs, g = threadIdx.x / kTilePairs;
  for (int64_t blk = blockIdx.x; blk < (int64_t)nc * n_w * n_groups; blk += gridDim.x) {
    const int ig = static_cast<int>(blk % n_groups);
    const int64_t rest = blk / n_groups;
    const int w = static_cast<int>(rest % n_w);
    const int c = c0 + static_cast<int>(rest / n_w);
    const int t0 = w * window, len = min(n_time, t0 + window) - t0;
    // the slice's rows into shared memory, once: asynchronous 16-byte copies, all of a thread's
    // rows in flight together
    const float4* col = in + (int64_t)c * half + ig * kTilePairs + q;
    const int64_t row_step = (int64_t)n_chan * half;
    for (int r = g; r < len; r += kTileGroups) {
      const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(&slice[r * kTilePairs + q]));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(col + (t0 + r) * row_step)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    uint32_t mb0 = 0u, mb1 = 0u;
    for (int r = g; r < len; r += kTileGroups) {
      const float4 v = slice[r * kTilePairs + q];
      mb0 = max(mb0, max(abs_bits(v.x), abs_bits(v.y)));
      mb1 = max(mb1, max(abs_bits(v.z), abs_bits(v.w)));
    }
    part[0][g][q] = mb0;
    part[1][g][q] = mb1;
    __syncthreads();
    if (threadIdx.x < 2 * kTilePairs) {
      const int k = threadIdx.x / kTilePairs, pq = threadIdx.x % kTilePairs;
      uint32_t m = 0u;
#pragma unroll
      for (int gg = 0; gg < kTileGroups; ++gg) m = max(m, part[k][gg][pq]);
      const int e = window_exponent(m);
      win_e[k][pq] = e;
      exps[((int64_t)c * exp_windows + w) * ni_pad + ig * kTileInputs + 2 * pq + k] = static_cast<int16_t>(e);
    }
    __syncthreads();
    float s0a, s0b, s1a, s1b;
    window_scale(win_e[0][q], s0a, s0b);
    window_scale(win_e[1][q], s1a, s1b);
    uint32_t* base = reinterpret_cast<uint32_t*>(planes + (6 * (int64_t)c) * comp_stride + ig * kTileInputs + 2 * q);
    const int64_t cs = comp_stride / 2;  // in uint32 units (comp_stride is a multiple of 16)
    for (int r = g; r < len; r += kTileGroups) {
      const float4 v = slice[r * kTilePairs + q];
      uint16_t r0[3], m0[3], r1[3], m1[3];
      digits_of(v.x, s0a, s0b, r0);
      digits_of(v.y, s0a, s0b, m0);
      digits_of(v.z, s1a, s1b, r1);
      digits_of(v.w, s1a, s1b, m1);
      uint32_t* row = base + (int64_t)(t0 + r) * (ni_pad / 2);
#pragma unroll
      for (int pc = 0; pc < 3; ++pc) {
        row[pc * cs] = r0[pc] | (static_cast<uint32_t>(r1[pc]) << 16);
        row[(3 + pc) * cs] = m0[pc] | (static_cast<uint32_t>(m1[pc]) << 16);
      }
    }
    __syncthreads();  // the slice is refilled by the next block of work
  }
}

int64_t grid_for(int64_t work, int num_sms) {
  int64_t blocks = (work + 255) / 256;
  const int64_t cap = (int64_t)num_sms * 16;
  if (blocks > cap) blocks = cap;
  return blocks < 1 ? 1 : blocks;
}

}  // namespace

cudaError_t launch_unpack_ci8_bf16(const int8_t* in, uint16_t* planes, int n_time, int n_chan, int c0, int nc,
                                   int n_inputs, int ni_pad, int max_time, int num_sms, cudaStream_t stream) {
  const int64_t n_rows = (int64_t)n_time * nc;
  const int64_t comp_stride = (int64_t)max_time * ni_pad;
  const bool vec = (n_inputs % 8 == 0) && (reinterpret_cast<uintptr_t>(in) % 16 == 0);
  const int64_t work = n_rows * (n_inputs / 8), blocks = grid_for(work, num_sms);
  if (vec && work + blocks * 256 < (INT64_C(1) << 32))
    unpack_ci8_bf16_vec<uint32_t><<<(unsigned)blocks, 256, 0, stream>>>(in, planes, n_rows, n_chan, c0, nc,
                                                                       n_inputs / 8, ni_pad, comp_stride);
  else if (vec)
    unpack_ci8_bf16_vec<int64_t><<<(unsigned)blocks, 256, 0, stream>>>(in, planes, n_rows, n_chan, c0, nc,
                                                                      n_inputs / 8, ni_pad, comp_stride);
  else
    unpack_ci8_bf16_elem<<<(unsigned)grid_for(n_rows * n_inputs, num_sms), 256, 0, stream>>>(
        in, planes, n_rows, n_chan, c0, nc, n_inputs, ni_pad, comp_stride);
  return cudaGetLastError();
}

cudaError_t launch_unpack_cf32_digits(const float* in, uint16_t* planes, int16_t* exps, int n_time, int n_chan,
                                      int c0, int nc, int n_inputs, int ni_pad, int max_time, int window,
                                      int exp_windows, cudaStream_t stream) {
  const int64_t comp_stride = (int64_t)max_time * ni_pad;
  if (n_inputs % kTileInputs == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0) {
    // read once through shared memory: 2 CTAs per SM, each looping over its slices
    const size_t smem = (size_t)window * kTilePairs * sizeof(float4);
    static int attr_device = -1;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && attr_device != dev) {
      e = cudaFuncSetAttribute(unpack_cf32_digits_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e == cudaSuccess) attr_device = dev;
    }
    if (e != cudaSuccess) return e;
    const int64_t slices = (int64_t)nc * ((n_time + window - 1) / window) * (n_inputs / kTileInputs);
    const int64_t grid = slices < 2LL * sms ? slices : 2LL * sms;
    unpack_cf32_digits_tile_kernel<<<(unsigned)grid, kTileThreads, smem, stream>>>(
        reinterpret_cast<const float4*>(in), planes, exps, n_time, n_chan, c0, nc, n_inputs, ni_pad, comp_stride,
        window, exp_windows);
    return cudaGetLastError();
  }
  const bool x2 = n_inputs % 2 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0;
  const int64_t work = (int64_t)nc * ((n_time + window - 1) / window) * (x2 ? n_inputs / 2 : n_inputs);
  int64_t blocks = (work + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > (1 << 20)) blocks = 1 << 20;
  if (x2)
    unpack_cf32_digits_x2_kernel<<<(unsigned)blocks, 256, 0, stream>>>(
        reinterpret_cast<const float4*>(in), planes, exps, n_time, n_chan, c0, nc, n_inputs, ni_pad, comp_stride,
        window, exp_windows);
  else
    unpack_cf32_digits_kernel<<<(unsigned)blocks, 256, 0, stream>>>(in, planes,
                                                                    exps, n_time, n_chan, c0, nc, n_inputs, ni_pad,
                                                                    comp_stride, window, exp_windows);
  return cudaGetLastError();
}

}  // namespace xc
