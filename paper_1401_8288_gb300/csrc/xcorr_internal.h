// xcorr_internal.h -- plan state and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "xcorr.h"

namespace xc {

// Exactness bounds of one integration held in int32 (sum of per-sample
// products; the largest |Re| or |Im| contribution of one sample is
// 2 * 8 * 8 = 128 for 4-bit codes in [-8, 7] and 2 * 128 * 128 for int8).
constexpr int64_t kMaxIntegrationCI4 = (INT64_C(2147483647)) / 128;    // 16,777,215
constexpr int64_t kMaxIntegrationCI8 = (INT64_C(2147483647)) / 32768;  // 65,535

// The tensor path accumulates exact products in FP32 tensor memory and drains
// it every window.  Integer input stays exact while every partial sum of a
// window is an integer below 2^24: per sample at most 128 (4-bit) or 32768
// (int8) per accumulator, so windows of 130,944 (4-bit: 16,760,832) and 384
// (int8: 12,582,912) samples.  Float input is quantised per 384-sample window
// into integer digits whose products are at most 2^14 (2 * 384 * 2^14 < 2^24).
// Windows are multiples of every stage height (128, 96, 64 rows for E4M3;
// 64, 48, 32 for BF16).
constexpr int kTcWindowCI4 = 130944;
constexpr int kTcWindowBF16 = 384;
// Offset-binary 4-bit operands u = t + 8 in [0, 15]: |sum_t (u_re u_re' + u_im u_im')| <= 450 T
// stays below 2^24 for T <= 37,282; rounded down to a multiple of 384 (every stage height).
constexpr int kFusedWindowCI4 = 37248;
constexpr int kTcVariants = 3;     // planes-path stage shapes: 64 KB x 3, 48 KB x 4, 32 KB x 6
constexpr int kFusedVariants = 11;  // fused 4-bit kernel shapes (the tuning's stage_variant range)
constexpr int kDefaultFusedVariant = 4;  // 4-bit plans before any tuning: A in tensor memory, 128 x (2 + 2)
constexpr int kSmallFusedVariant = 10;   // ... for small problems: the same kernel, channels packed, time split
// The planes path's shape for a tuning's stage_variant (3 exists only for the fused kernel).
inline int planes_variant(int v) { return v >= kTcVariants ? 1 : v; }
constexpr int64_t kMaxIntegrationCF32 = INT64_C(16777216);  // FP32 per dump, widen beyond
// Float input: window exponents E = floor(log2(largest magnitude of the window)), so every
// component is below 2^(E+1), lie in [kExpMin, 127] (int16); a window of zeros takes kExpMin.
// A subnormal maximum gets its own exponent too, so the window's 23-bit quantisation keeps its
// full length (a subnormal m 2^-149 is the integer m 2^(-127 - E) on that window's grid).  A
// window holding a NaN or an infinity is marked kExpNonFinite, and every block that involves
// it drains as NaN.
constexpr int kExpMin = -149;
constexpr int kExpNonFinite = -256;

// 2^n as a float for -149 <= n <= 127 (subnormal below -126), built from its bits.
__host__ __device__ __forceinline__ float pow2i(int n) {
  union {
    uint32_t u;
    float f;
  } v;
  v.u = n >= -126 ? static_cast<uint32_t>(n + 127) << 23 : 1u << (n + 149);
  return v.f;
}

enum ExecMode : int { MODE_STORE = 0, MODE_ADD = 1, MODE_ATOMIC = 2 };

// The tensor path splits the channels of an execute into groups: the unpack
// of group g + 1 runs on one internal stream while the X kernel of group g
// runs on another, so the HBM-bound unpack hides under the tensor-bound X.
constexpr int kMaxGroups = 8;
constexpr int kProfileEvents = 2 + 2 * kMaxGroups;  // per timed execute

}  // namespace xc

struct xcorr_plan_s {
  xcorr_config cfg{};
  int device = 0;
  int num_sms = 0;
  int n_inputs = 0;  // N_i
  int ni_pad = 0;    // plane row pitch (inputs), multiple of 16
  int64_t n_pairs = 0;
  int engine = 0;
  int64_t max_integration = 0;
  int64_t samples = 0;  // samples integrated since the last reset
  bool fresh = true;    // the accumulator holds nothing of the current integration
  int sticky = 0;       // a kernel failure was seen: every call fails until destroy

  void* acc = nullptr;         // [C][P] (re, im): int32 (integer input) or float (float input)
  void* planes = nullptr;      // tensor path: [C][planes_per_chan][max_time][ni_pad] numbers
  int16_t* exps = nullptr;     // float input: window exponents [C][exp_windows][ni_pad]
  int exp_windows = 0;
  size_t planes_bytes = 0;
  int elem_bytes = 1;          // plane numbers: 1 = E4M3, 2 = BF16
  int planes_per_chan = 2;     // re pieces then im pieces
  int window_samples = 0;      // drain window of the tensor X kernel
  int* status = nullptr;       // device status word
  int* status_host = nullptr;  // pinned mirror, refreshed by every dump
  size_t device_bytes = 0;

  // tuning of the tensor path (xcorr_plan_set_tuning / xcorr_autotune); 0 = automatic
  int tune_variant = 0;        // stage shape, 0 .. kFusedVariants - 1 (see planes_variant)
  int tune_groups = 0;         // channel groups, 0 = heuristic
  int tune_x_streams = 2;      // X launches alternate over 1 or 2 streams
  int tune_unfused = 0;        // 4-bit input: 1 = always through planes, 0 = fuse the unpack when possible


  CUtensorMap tmap{};          // planes, for tmap_ntime / tmap_variant
  int tmap_ntime = -1;
  int tmap_variant = -1;

  // internal streams of the tensor path (forked from and joined to the caller's stream)
  cudaStream_t s_unpack = nullptr;
  cudaStream_t s_x[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_unpacked[xc::kMaxGroups] = {};
  cudaEvent_t ev_x_done[2] = {nullptr, nullptr};
  // host-to-host executes: device copy of the input, the copy-out stream and
  // per-group events (made on first use)
  void* host_stage = nullptr;
  size_t host_stage_bytes = 0;
  cudaStream_t s_down = nullptr;
  cudaEvent_t ev_up[xc::kMaxGroups] = {};
  cudaEvent_t ev_group_done[xc::kMaxGroups] = {};
  cudaEvent_t ev_down = nullptr;

  // timing (xcorr_profile_enable): kProfileEvents per timed execute -- start,
  // end of the last unpack, then (begin, end) of each X launch
  cudaEvent_t* prof_events = nullptr;
  int prof_cap = 0;
  int64_t prof_count = 0;
  int* prof_ngroups = nullptr;  // groups used by each timed execute
};

namespace xc {

// Launchers; each returns the launch's cudaError_t.
cudaError_t launch_unpack_ci4_e4m3(const uint8_t* in, uint8_t* planes, int n_time, int n_chan,
                                   int n_inputs, int ni_pad, int max_time, int num_sms,
                                   cudaStream_t stream);
// The same for channels [c0, c0 + nc) only.
cudaError_t launch_unpack_ci4_e4m3_channels(const uint8_t* in, uint8_t* planes, int n_time, int n_chan,
                                            int c0, int nc, int n_inputs, int ni_pad, int max_time,
                                            int num_sms, cudaStream_t stream);

// Channels [chan0, chan0 + n_chan) of the planes described by tmap; acc points
// at channel 0 of the packed accumulator.
// One launch of the tensor-core X kernel over channels [chan0, chan0 + n_chan).
struct TcLaunch {
  int elem_bytes = 1;       // 1: E4M3 planes (kind::f8f6f4), 2: BF16 planes (kind::f16)
  int variant = 0;          // stage shape, 0 .. kTcVariants - 1
  bool float_out = false;   // float accumulator (float input) or exact int32
  int n_time = 0, chan0 = 0, n_chan = 0, n_inputs = 0;
  int planes_per_chan = 2;  // re planes then im planes: 2 (one piece) or 6 (three)
  int n_pairs_k = 1;        // plane pairs on the virtual K axis
  int pair_p[8] = {0}, pair_q[8] = {0};
  int window_samples = kTcWindowCI4;  // samples per drained block
  const int16_t* exps = nullptr;      // float input: window exponents [C][exp_windows][ni_pad]
  int exp_windows = 0, ni_pad = 0;
  bool accumulate = false;  // add into out (else the first block stores)
  void* out = nullptr;      // int2 or float2 [C][P]
  int* status = nullptr;
  int num_sms = 0;
};
int tc_stage_samples(int elem_bytes, int variant);

// One subarray of a batch, as the batch X kernel reads it from device memory
// (host and device share this layout; it inherits the tensor map's alignment).
struct SubDescHost {
  CUtensorMap tmap;  // its E4M3 planes
  void* out;         // its int2 [C][P] visibilities
  int64_t n_pairs;
  int n_inputs, n_kt, n_tw, pad;
};
// A subarray of a batch run by the fused 4-bit kernel (A operand in tensor memory).
struct TaSubDesc {
  CUtensorMap tmap;  // its raw CI4 input: boxes of 128 inputs x 1 channel x the stage height
  int2* out;         // its int2 [C][P] visibilities
  int64_t n_pairs;
  int n_inputs, n_tile_pairs, n_kt, accumulate;
};
static_assert(sizeof(TaSubDesc) % 64 == 0, "tensor maps in a descriptor array stay 64-byte aligned");
cudaError_t launch_xcorr_tc_fused_ta_batch(const TaSubDesc* subs, const uint4* items, int n_items, int variant,
                                           int* status, int num_sms, cudaStream_t stream);
// One launch of the batch X kernel over items (subarray, channel, I, J).
cudaError_t launch_xcorr_tc_batch(const void* subs, const uint4* items, int n_items, int variant, int* status,
                                  int num_sms, cudaStream_t stream);
cudaError_t launch_xcorr_tc(const CUtensorMap* tmap, const TcLaunch& launch, cudaStream_t stream);

cudaError_t launch_xcorr_cuda_core(int fmt, const void* in, int n_time, int n_chan, int n_inputs,
                                   int2* acc, int mode, int ksplit, cudaStream_t stream);

// Choose the CUDA-core kernel's split of the time axis (1 = no split).
int cuda_core_ksplit(int n_time, int n_chan, int n_inputs, int num_sms);

// The autotuners' cache (xcorr_tune_cache.cpp): a problem's key on the current device, and the
// shape recorded for it.
struct TuneKey {
  std::string scope, device;  // "plan" or "batch"; the device's name
  int sms = 0, fmt = 0, n_inputs = 0, n_channels = 0, n_time = 0;
};
TuneKey tune_key(const char* scope, int fmt, int n_inputs, int n_channels, int n_time);
bool tune_cache_get(const TuneKey& key, xcorr_tuning* tuning, float* ms);
void tune_cache_put(const TuneKey& key, const xcorr_tuning& tuning, float ms);

// Record the calling thread's error message (read by xcorr_last_error) and return st.
xcorr_status set_error(xcorr_status st, const std::string& msg);
// For the library's other front ends (streams): the plan checks of every call,
// one execute of n_time samples into `target` (store when target_fresh, else
// add; the plan's own accumulator is untouched unless it is the target), and
// a read of the device status word (DEVICE if a kernel gave up a wait).
xcorr_status plan_check(xcorr_plan plan);
xcorr_status execute_into(xcorr_plan plan, const void* d_in, int n_time, void* target, bool target_fresh,
                          cudaStream_t s);
xcorr_status read_device_status(xcorr_plan plan);

cudaError_t launch_fold_wide_i64(const int2* acc, int64_t* out, int64_t n_pairs_total,
                                 cudaStream_t stream);

// Encode the 3-D tensor map over planes of elem_bytes-byte numbers (dims:
// input, time, channel * planes_per_chan + plane), box 128 bytes x box_t rows.
bool encode_plane_tmap(CUtensorMap* map, void* planes, int elem_bytes, int n_inputs, int ni_pad,
                       int n_time, int max_time, int n_planes_total, int box_t, std::string* err);


// Tensor map over n_chan channels of a CI4 input [t][c][i] whose time rows hold
// row_chans channels (n_inputs % 16 == 0, 16-byte aligned pointer to the first
// channel): boxes of box_i (128 or 64) inputs x 1 channel x box_t samples,
// swizzled at the box's row width (the fused kernels' raw tiles, and their L2
// prefetches).
bool encode_raw_ci4_tmap(CUtensorMap* map, const void* in, int n_inputs, int n_chan, int row_chans, int n_time,
                         int box_t, std::string* err, int box_i = 128);
// The same input with channel and input merged into one dimension (boxes of 128 bytes: 128 /
// n_inputs channels side by side per time row), for the small-problem layout that packs
// channels into one tile (n_inputs % 16 == 0, 16-byte aligned pointer).
bool encode_raw_ci4_packed_tmap(CUtensorMap* map, const void* in, int n_inputs, int n_chan, int row_chans,
                                int n_time, int box_t, std::string* err);
// The fused 4-bit X kernel (unpack on chip, offset-binary operands): one
// launch per kFusedWindowCI4 samples; n_inputs % 16 == 0, `in` 16-byte aligned.
int fused_stage_samples(int variant);
int fused_launches(int n_time);
// `in` points at the first of n_chan channels; time rows hold row_chans channels.
// Variants 0-3 decode both operands into shared memory; 4-6 run the kernel
// with the A operand in tensor memory (its variants 0-2); 7-9 run the CTA-pair
// kernel (its variants 0-2); 10 runs the tensor-memory-A kernel's small-problem
// layout (its variant 3: channels packed per tile, time split over the SMs).
cudaError_t launch_xcorr_tc_fused_ci4(const uint8_t* in, int row_chans, int variant, int n_time, int n_chan,
                                      int n_inputs, int2* out, bool accumulate, int* status, int num_sms,
                                      cudaStream_t stream);

int fused_ta_stage_samples(int variant);
cudaError_t launch_xcorr_tc_fused_ta_ci4(const uint8_t* in, int row_chans, int variant, int n_time, int n_chan,
                                         int n_inputs, int2* out, bool accumulate, int* status, int num_sms,
                                         cudaStream_t stream);

// The fused 4-bit kernel on CTA pairs (xcorr_tc_fused_pair.cu): two SMs share
// one column tile through a cta_group::2 MMA.
int fused_pair_stage_samples(int variant);
cudaError_t launch_xcorr_tc_fused_pair_ci4(const uint8_t* in, int row_chans, int variant, int n_time, int n_chan,
                                           int n_inputs, int2* out, bool accumulate, int* status, int num_sms,
                                           cudaStream_t stream);

// int8 (re, im) samples -> two BF16 planes [c][2][t][ni_pad] (exact).
cudaError_t launch_unpack_ci8_bf16(const int8_t* in, uint16_t* planes, int n_time, int n_chan, int c0,
                                   int nc, int n_inputs, int ni_pad, int max_time, int num_sms,
                                   cudaStream_t stream);
// float (re, im) samples -> six BF16 planes [c][6][t][ni_pad] of integer digits
// (re digits 0-2, im digits 0-2) and one exponent per (channel, window, input).
cudaError_t launch_unpack_cf32_digits(const float* in, uint16_t* planes, int16_t* exps, int n_time, int n_chan,
                                      int c0, int nc, int n_inputs, int ni_pad, int max_time, int window,
                                      int exp_windows, cudaStream_t stream);
cudaError_t launch_fold_wide_f64(const float2* acc, double* out, int64_t n_pairs_total, cudaStream_t stream);

}  // namespace xc
