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

// The tensor path accumulates E4M3 products in FP32 tensor memory, exact while
// every partial sum stays below 2^24: at most 128 * W for a window of W
// samples.  W = 130,944 keeps 128 * W = 16,760,832 < 2^24.
constexpr int kTcStageT = 64;  // samples per pipeline stage (TMA box height)
constexpr int kTcWindowSamples = 130944;
constexpr int kTcMaxKblocksPerWindow = kTcWindowSamples / kTcStageT;
static_assert(kTcWindowSamples % kTcStageT == 0, "window must hold whole stages");

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

  int2* acc = nullptr;         // [C][P] (re, im) int32
  uint8_t* planes = nullptr;   // tensor path: E4M3 planes [C][2][max_time][ni_pad]
  size_t planes_bytes = 0;
  int* status = nullptr;       // device status word
  int* status_host = nullptr;  // pinned mirror, refreshed by every dump
  size_t device_bytes = 0;

  CUtensorMap tmap{};  // planes, for the n_time of the last tensor execute
  int tmap_ntime = -1;

  // internal streams of the tensor path (forked from and joined to the caller's stream)
  cudaStream_t s_unpack = nullptr;
  cudaStream_t s_x[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_unpacked[xc::kMaxGroups] = {};
  cudaEvent_t ev_x_done[2] = {nullptr, nullptr};

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
cudaError_t launch_xcorr_tc_e4m3(const CUtensorMap* tmap, int n_time, int chan0, int n_chan,
                                 int n_inputs, int2* acc, bool accumulate, int* status,
                                 int num_sms, cudaStream_t stream);

cudaError_t launch_xcorr_cuda_core(int fmt, const void* in, int n_time, int n_chan, int n_inputs,
                                   int2* acc, int mode, int ksplit, cudaStream_t stream);

// Choose the CUDA-core kernel's split of the time axis (1 = no split).
int cuda_core_ksplit(int n_time, int n_chan, int n_inputs, int num_sms);

// Record the calling thread's error message (read by xcorr_last_error) and return st.
xcorr_status set_error(xcorr_status st, const std::string& msg);

cudaError_t launch_fold_wide_i64(const int2* acc, int64_t* out, int64_t n_pairs_total,
                                 cudaStream_t stream);

// Encode the 3-D tensor map over the E4M3 planes (dims: input, time, channel*2+component).
bool encode_plane_tmap(CUtensorMap* map, void* planes, int n_inputs, int ni_pad, int n_time,
                       int max_time, int n_chan, std::string* err);

}  // namespace xc
