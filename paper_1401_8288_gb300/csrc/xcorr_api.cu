// xcorr_api.cu -- the C ABI (xcorr.h): plan validation, device memory owned
// by the plan, kernel selection, tuning and stream-ordered launches.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "xcorr_internal.h"
#include "xcorr_nvtx.h"

namespace {

thread_local std::string g_last_error;

xcorr_status fail(xcorr_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

xcorr_status cuda_fail(cudaError_t e, const char* what) {
  return fail(XCORR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int64_t n_pairs_of(int n_inputs) { return (int64_t)n_inputs * (n_inputs + 1) / 2; }

// Checks common to every call on a live plan.
xcorr_status plan_ok(xcorr_plan plan) {
  if (!plan) return fail(XCORR_ERR_INVALID_ARG, "plan is NULL");
  if (!plan->sticky && plan->status_host && *const_cast<volatile int*>(plan->status_host) != 0)
    plan->sticky = *plan->status_host;
  if (plan->sticky)
    return fail(XCORR_ERR_DEVICE, "a kernel of this plan reported failure code " + std::to_string(plan->sticky) +
                                      " (a bounded wait ran out); destroy the plan");
  cudaError_t e = cudaSetDevice(plan->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return XCORR_OK;
}

void free_profile(xcorr_plan plan) {
  if (plan->prof_events) {
    for (int64_t k = 0; k < (int64_t)xc::kProfileEvents * plan->prof_cap; ++k)
      if (plan->prof_events[k]) cudaEventDestroy(plan->prof_events[k]);
    delete[] plan->prof_events;
  }
  delete[] plan->prof_ngroups;
  plan->prof_events = nullptr;
  plan->prof_ngroups = nullptr;
  plan->prof_cap = 0;
  plan->prof_count = 0;
}

void release(xcorr_plan plan) {
  free_profile(plan);
  if (plan->s_unpack) cudaStreamDestroy(plan->s_unpack);
  for (auto& sx : plan->s_x)
    if (sx) cudaStreamDestroy(sx);
  if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
  for (auto& ev : plan->ev_unpacked)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : plan->ev_x_done)
    if (ev) cudaEventDestroy(ev);
  plan->s_unpack = nullptr;
  plan->s_x[0] = plan->s_x[1] = nullptr;
  if (plan->s_down) cudaStreamDestroy(plan->s_down);
  plan->s_down = nullptr;
  for (auto* evs : {plan->ev_up, plan->ev_group_done})
    for (int g = 0; g < xc::kMaxGroups; ++g)
      if (evs[g]) cudaEventDestroy(evs[g]);
  if (plan->ev_down) cudaEventDestroy(plan->ev_down);
  plan->ev_down = nullptr;
  if (plan->host_stage) cudaFree(plan->host_stage);
  plan->host_stage = nullptr;
  if (plan->acc) cudaFree(plan->acc);
  if (plan->planes) cudaFree(plan->planes);
  if (plan->exps) cudaFree(plan->exps);
  plan->exps = nullptr;
  if (plan->status) cudaFree(plan->status);
  if (plan->status_host) cudaFreeHost(plan->status_host);
  plan->acc = nullptr;
  plan->planes = nullptr;
  plan->status = nullptr;
  plan->status_host = nullptr;
}

xcorr_status check_execute(xcorr_plan plan, const void* d_in, int n_time) {
  xcorr_status st = plan_ok(plan);
  if (st != XCORR_OK) return st;
  if (!d_in) return fail(XCORR_ERR_INVALID_ARG, "d_in is NULL");
  if (plan->cfg.fmt == XCORR_IN_CF32 && reinterpret_cast<uintptr_t>(d_in) % 4)
    return fail(XCORR_ERR_INVALID_ARG, "float input must be 4-byte aligned");
  if (n_time < 1 || n_time > plan->cfg.max_time_per_exec)
    return fail(XCORR_ERR_INVALID_ARG, "n_time must be in [1, max_time_per_exec]");
  if (plan->samples + n_time > plan->max_integration)
    return fail(XCORR_ERR_OVERFLOW, "the integration would exceed " + std::to_string(plan->max_integration) +
                                        " samples (the exact range of one dump); dump with reset first");
  return XCORR_OK;
}

// Channel groups of the tensor path: the tuned count, else enough tile pairs
// per group for about four waves of the persistent X kernel.
int tensor_groups(xcorr_plan plan) {
  int64_t g;
  if (plan->tune_groups > 0) {
    g = plan->tune_groups;
  } else {
    const int nb = (plan->n_inputs + 127) / 128;
    const int64_t items = (int64_t)plan->cfg.n_channels * nb * (nb + 1) / 2;
    g = items / (4LL * plan->num_sms);
  }
  if (g > xc::kMaxGroups) g = xc::kMaxGroups;
  if (g > plan->cfg.n_channels) g = plan->cfg.n_channels;
  return g < 1 ? 1 : static_cast<int>(g);
}

// The 4-bit tensor path can unpack on chip: inputs a multiple of 16 and a
// 16-byte aligned pointer (the decoders read whole 16-sample chunks).
bool fused_applies(xcorr_plan plan, const void* d_in) {
  return plan->cfg.fmt == XCORR_IN_CI4 && !plan->tune_unfused && plan->n_inputs % 16 == 0 &&
         reinterpret_cast<uintptr_t>(d_in) % 16 == 0;
}

// Unpack channels [c0, c0 + nc) of the input into the plan's planes.
cudaError_t unpack_group(xcorr_plan plan, const void* d_in, int n_time, int c0, int nc, cudaStream_t s) {
  const int C = plan->cfg.n_channels, N = plan->n_inputs, T = plan->cfg.max_time_per_exec;
  switch (plan->cfg.fmt) {
    case XCORR_IN_CI4:
      return xc::launch_unpack_ci4_e4m3_channels(static_cast<const uint8_t*>(d_in), static_cast<uint8_t*>(plan->planes),
                                                 n_time, C, c0, nc, N, plan->ni_pad, T, plan->num_sms, s);
    case XCORR_IN_CI8:
      return xc::launch_unpack_ci8_bf16(static_cast<const int8_t*>(d_in), static_cast<uint16_t*>(plan->planes), n_time,
                                        C, c0, nc, N, plan->ni_pad, T, plan->num_sms, s);
    default:
      return xc::launch_unpack_cf32_digits(static_cast<const float*>(d_in), static_cast<uint16_t*>(plan->planes),
                                           plan->exps, n_time, C, c0, nc, N, plan->ni_pad, T, plan->window_samples,
                                           plan->exp_windows, s);
  }
}

// Correlate n_time samples into target (the plan's accumulator, or the
// caller's buffer for a fused dump).  target_fresh: store instead of add.
xcorr_status run_execute(xcorr_plan plan, const void* d_in, int n_time, void* target, bool target_fresh,
                         cudaStream_t s) {
  const int C = plan->cfg.n_channels, N = plan->n_inputs;
  cudaError_t e;
  cudaEvent_t* ev = nullptr;
  if (plan->prof_cap) {
    const int64_t slot = plan->prof_count % plan->prof_cap;
    ev = plan->prof_events + xc::kProfileEvents * slot;
    if ((e = cudaEventRecord(ev[0], s)) != cudaSuccess) return cuda_fail(e, "profile event");
  }
  if (plan->engine == XCORR_ENGINE_TENSOR && fused_applies(plan, d_in)) {
    // 4-bit input with the unpack on chip: one launch per exact block, on the caller's stream
    if (ev && ((e = cudaEventRecord(ev[1], s)) != cudaSuccess || (e = cudaEventRecord(ev[2], s)) != cudaSuccess))
      return cuda_fail(e, "profile event");
    e = xc::launch_xcorr_tc_fused_ci4(static_cast<const uint8_t*>(d_in), C, plan->tune_variant, n_time, C, N,
                                      static_cast<int2*>(target), !target_fresh, plan->status, plan->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "fused X kernel launch");
    if (ev && (e = cudaEventRecord(ev[3], s)) != cudaSuccess) return cuda_fail(e, "profile event");
    if (ev) plan->prof_ngroups[plan->prof_count % plan->prof_cap] = 1;
  } else if (plan->engine == XCORR_ENGINE_TENSOR) {
    const int variant = xc::planes_variant(plan->tune_variant);
    if (plan->tmap_ntime != n_time || plan->tmap_variant != variant) {
      std::string err;
      if (!xc::encode_plane_tmap(&plan->tmap, plan->planes, plan->elem_bytes, N, plan->ni_pad, n_time,
                                 plan->cfg.max_time_per_exec, C * plan->planes_per_chan,
                                 xc::tc_stage_samples(plan->elem_bytes, variant), &err))
        return fail(XCORR_ERR_CUDA, err);
      plan->tmap_ntime = n_time;
      plan->tmap_variant = variant;
    }
    xc::TcLaunch L;
    L.elem_bytes = plan->elem_bytes;
    L.variant = variant;
    L.float_out = plan->cfg.fmt == XCORR_IN_CF32;
    L.n_time = n_time;
    L.n_inputs = N;
    L.planes_per_chan = plan->planes_per_chan;
    if (plan->cfg.fmt == XCORR_IN_CF32) {
      // the six digit products d_p d_q with p + q <= 2
      L.exps = plan->exps;
      L.exp_windows = plan->exp_windows;
      L.ni_pad = plan->ni_pad;
      const int pp[6] = {0, 0, 1, 0, 2, 1}, pq[6] = {0, 1, 0, 2, 0, 1};
      L.n_pairs_k = 6;
      for (int k = 0; k < 6; ++k) {
        L.pair_p[k] = pp[k];
        L.pair_q[k] = pq[k];
      }
    }
    L.window_samples = plan->window_samples;
    L.accumulate = !target_fresh;
    L.out = target;
    L.status = plan->status;
    L.num_sms = plan->num_sms;
    const int G = tensor_groups(plan);
    const int per = (C + G - 1) / G;
    const int nxs = plan->tune_x_streams == 1 ? 1 : 2;
    // fork: the internal streams start after everything queued on s so far
    if ((e = cudaEventRecord(plan->ev_fork, s)) != cudaSuccess) return cuda_fail(e, "fork event");
    if ((e = cudaStreamWaitEvent(plan->s_unpack, plan->ev_fork, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(plan->s_x[0], plan->ev_fork, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(plan->s_x[1], plan->ev_fork, 0)) != cudaSuccess)
      return cuda_fail(e, "fork wait");
    int used = 0;
    for (int g = 0, c0 = 0; c0 < C; ++g, c0 += per) {
      const int nc = (C - c0 < per) ? C - c0 : per;
      if ((e = unpack_group(plan, d_in, n_time, c0, nc, plan->s_unpack)) != cudaSuccess)
        return cuda_fail(e, "unpack launch");
      if ((e = cudaEventRecord(plan->ev_unpacked[g], plan->s_unpack)) != cudaSuccess) return cuda_fail(e, "event");
      cudaStream_t sx = plan->s_x[g % nxs];
      if ((e = cudaStreamWaitEvent(sx, plan->ev_unpacked[g], 0)) != cudaSuccess) return cuda_fail(e, "wait");
      if (ev && (e = cudaEventRecord(ev[2 + 2 * g], sx)) != cudaSuccess) return cuda_fail(e, "profile event");
      L.chan0 = c0;
      L.n_chan = nc;
      if ((e = xc::launch_xcorr_tc(&plan->tmap, L, sx)) != cudaSuccess)
        return cuda_fail(e, "tensor-core X kernel launch");
      if (ev && (e = cudaEventRecord(ev[3 + 2 * g], sx)) != cudaSuccess) return cuda_fail(e, "profile event");
      used = g + 1;
    }
    if (ev && (e = cudaEventRecord(ev[1], plan->s_unpack)) != cudaSuccess) return cuda_fail(e, "profile event");
    // join: s continues after both X streams (which waited for every unpack)
    for (int k = 0; k < 2; ++k) {
      if ((e = cudaEventRecord(plan->ev_x_done[k], plan->s_x[k])) != cudaSuccess ||
          (e = cudaStreamWaitEvent(s, plan->ev_x_done[k], 0)) != cudaSuccess)
        return cuda_fail(e, "join");
    }
    if (ev) plan->prof_ngroups[plan->prof_count % plan->prof_cap] = used;
  } else {
    const int ks = xc::cuda_core_ksplit(n_time, C, N, plan->num_sms);
    int mode = target_fresh ? xc::MODE_STORE : xc::MODE_ADD;
    if (ks > 1) {
      if (target_fresh) {
        e = cudaMemsetAsync(target, 0, (size_t)C * plan->n_pairs * sizeof(int2), s);
        if (e != cudaSuccess) return cuda_fail(e, "accumulator clear");
      }
      mode = xc::MODE_ATOMIC;
    }
    if (ev && ((e = cudaEventRecord(ev[1], s)) != cudaSuccess || (e = cudaEventRecord(ev[2], s)) != cudaSuccess))
      return cuda_fail(e, "profile event");
    e = xc::launch_xcorr_cuda_core(plan->cfg.fmt, d_in, n_time, C, N, static_cast<int2*>(target), mode, ks, s);
    if (e != cudaSuccess) return cuda_fail(e, "CUDA-core X kernel launch");
    if (ev && (e = cudaEventRecord(ev[3], s)) != cudaSuccess) return cuda_fail(e, "profile event");
    if (ev) plan->prof_ngroups[plan->prof_count % plan->prof_cap] = 1;
  }
  if (ev) ++plan->prof_count;
  return XCORR_OK;
}

}  // namespace

namespace xc {
xcorr_status set_error(xcorr_status st, const std::string& msg) { return fail(st, msg); }
xcorr_status plan_check(xcorr_plan plan) { return plan_ok(plan); }
xcorr_status execute_into(xcorr_plan plan, const void* d_in, int n_time, void* target, bool target_fresh,
                          cudaStream_t s) {
  return run_execute(plan, d_in, n_time, target, target_fresh, s);
}
xcorr_status read_device_status(xcorr_plan plan) {
  int code = 0;
  cudaError_t e = cudaMemcpy(&code, plan->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (code) plan->sticky = code;
  return plan_ok(plan);
}
}  // namespace xc

extern "C" {

const char* xcorr_last_error(void) { return g_last_error.c_str(); }

xcorr_status xcorr_plan_create(xcorr_plan* out, const xcorr_config* cfg) {
  if (!out) return fail(XCORR_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(XCORR_ERR_INVALID_ARG, "cfg is NULL");
  const xcorr_config c = *cfg;
  if (c.n_pols != 2) return fail(XCORR_ERR_INVALID_ARG, "n_pols must be 2");
  if (c.n_stations < 1 || c.n_stations > (1 << 20))
    return fail(XCORR_ERR_INVALID_ARG, "n_stations must be in [1, 2^20]");
  if (c.n_channels < 1) return fail(XCORR_ERR_INVALID_ARG, "n_channels must be >= 1");
  if (c.max_time_per_exec < 1) return fail(XCORR_ERR_INVALID_ARG, "max_time_per_exec must be >= 1");
  if (c.fmt != XCORR_IN_CI4 && c.fmt != XCORR_IN_CI8 && c.fmt != XCORR_IN_CF32)
    return fail(XCORR_ERR_INVALID_ARG, "unknown input format");
  if (c.engine != XCORR_ENGINE_AUTO && c.engine != XCORR_ENGINE_TENSOR && c.engine != XCORR_ENGINE_CUDA_CORE)
    return fail(XCORR_ERR_INVALID_ARG, "unknown engine");

  // AUTO: the engine the per-call device times favour (graph-replayed execute_dump; 4-bit input
  // over inputs 2-256, channels 16-256, K 256-2048; int8 over inputs 2-256, channels 16-64,
  // K 256-1024).  The CUDA-core kernel wins only at most 16 channels: for 4-bit input below 16
  // inputs (the tensor path then unpacks to planes first: two launches), for int8 input up to 64
  // inputs (its tensor path always unpacks to BF16 planes first); the tensor cores everywhere else.
  const int cc_inputs = c.fmt == XCORR_IN_CI4 ? 15 : c.fmt == XCORR_IN_CI8 ? 64 : 0;
  const int engine = c.engine != XCORR_ENGINE_AUTO ? c.engine
                     : (c.n_stations <= cc_inputs / 2 && c.n_channels <= 16) ? XCORR_ENGINE_CUDA_CORE
                                                                            : XCORR_ENGINE_TENSOR;
  if (engine == XCORR_ENGINE_CUDA_CORE && c.fmt == XCORR_IN_CF32)
    return fail(XCORR_ERR_UNSUPPORTED, "the CUDA-core engine takes integer input only");

  const int64_t max_int = c.fmt == XCORR_IN_CI4   ? xc::kMaxIntegrationCI4
                          : c.fmt == XCORR_IN_CI8 ? xc::kMaxIntegrationCI8
                                                  : xc::kMaxIntegrationCF32;
  if (c.max_time_per_exec > max_int)
    return fail(XCORR_ERR_OVERFLOW, "max_time_per_exec exceeds the range of one integration, " +
                                        std::to_string(max_int) + " samples");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (prop.major != 10 || prop.minor != 3)
    return fail(XCORR_ERR_UNSUPPORTED, std::string("this library is built for sm_103a (GB300); device is ") +
                                           prop.name + " sm_" + std::to_string(prop.major * 10 + prop.minor));

  const int n_inputs = 2 * c.n_stations;
  const int ni_pad = (n_inputs + 15) / 16 * 16;
  const int64_t n_pairs = n_pairs_of(n_inputs);
  const int elem_bytes = c.fmt == XCORR_IN_CI4 ? 1 : 2;
  const int ppc = c.fmt == XCORR_IN_CF32 ? 6 : 2;
  const size_t acc_bytes = (size_t)c.n_channels * (size_t)n_pairs * 8;
  const size_t planes_bytes = engine == XCORR_ENGINE_TENSOR ? (size_t)c.n_channels * ppc *
                                                                  (size_t)c.max_time_per_exec * ni_pad * elem_bytes
                                                            : 0;
  const int exp_windows = (c.max_time_per_exec + xc::kTcWindowBF16 - 1) / xc::kTcWindowBF16;
  const size_t exps_bytes =
      (engine == XCORR_ENGINE_TENSOR && c.fmt == XCORR_IN_CF32) ? (size_t)c.n_channels * exp_windows * ni_pad * 2 : 0;
  const size_t dev_bytes = acc_bytes + planes_bytes + exps_bytes + 256;
  if (c.hbm_budget_bytes && dev_bytes > c.hbm_budget_bytes)
    return fail(XCORR_ERR_BUDGET, "plan needs " + std::to_string(dev_bytes) + " device bytes, budget is " +
                                      std::to_string(c.hbm_budget_bytes));

  xcorr_plan plan = new (std::nothrow) xcorr_plan_s();
  if (!plan) return fail(XCORR_ERR_OOM, "host allocation failed");
  plan->cfg = c;
  plan->cfg.engine = static_cast<xcorr_engine>(engine);
  plan->device = dev;
  plan->num_sms = prop.multiProcessorCount;
  plan->n_inputs = n_inputs;
  plan->ni_pad = ni_pad;
  plan->n_pairs = n_pairs;
  plan->engine = engine;
  plan->max_integration = max_int;
  plan->planes_bytes = planes_bytes;
  plan->device_bytes = dev_bytes;
  plan->elem_bytes = elem_bytes;
  plan->planes_per_chan = ppc;
  plan->window_samples = c.fmt == XCORR_IN_CI4 ? xc::kTcWindowCI4 : xc::kTcWindowBF16;
  plan->exp_windows = exp_windows;
  // 4-bit input starts on the fused kernel with the A operand in tensor memory (the fastest
  // shape measured), in its small-problem layout where that measured faster: at most 64 inputs
  // (channels packed per tile) with 1024 or more samples per execute or 256 or more channels;
  // the planes path reads the same tuning as its 4 x 48 KB ring
  plan->tune_variant = c.fmt != XCORR_IN_CI4 ? 0
                       : (n_inputs <= 64 && (c.max_time_per_exec >= 1024 || c.n_channels >= 256)) ? xc::kSmallFusedVariant
                                                                                                   : xc::kDefaultFusedVariant;

  if ((e = cudaMalloc(&plan->acc, acc_bytes)) != cudaSuccess ||
      (planes_bytes && (e = cudaMalloc(&plan->planes, planes_bytes)) != cudaSuccess) ||
      (exps_bytes && (e = cudaMalloc(&plan->exps, exps_bytes)) != cudaSuccess) ||
      (e = cudaMalloc(&plan->status, 256)) != cudaSuccess ||
      (e = cudaMallocHost(&plan->status_host, sizeof(int))) != cudaSuccess) {
    release(plan);
    delete plan;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? XCORR_ERR_OOM : XCORR_ERR_CUDA,
                std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  *plan->status_host = 0;
  if (engine == XCORR_ENGINE_TENSOR) {
    e = cudaStreamCreateWithFlags(&plan->s_unpack, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&plan->s_x[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_fork, cudaEventDisableTiming);
    for (int k = 0; k < xc::kMaxGroups && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&plan->ev_unpacked[k], cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&plan->ev_x_done[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      release(plan);
      delete plan;
      return cuda_fail(e, "stream or event creation");
    }
  }
  if (plan->exps && (e = cudaMemset(plan->exps, 0, exps_bytes)) != cudaSuccess) {
    release(plan);
    delete plan;
    return cuda_fail(e, "exponent clear");
  }
  if ((e = cudaMemset(plan->status, 0, 256)) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
    release(plan);
    delete plan;
    return cuda_fail(e, "plan initialisation");
  }
  *out = plan;
  return XCORR_OK;
}

xcorr_status xcorr_execute(xcorr_plan plan, const void* d_in, int n_time, void* stream) {
  xc::NvtxRange range("xcorr_execute");
  xcorr_status st = check_execute(plan, d_in, n_time);
  if (st != XCORR_OK) return st;
  st = run_execute(plan, d_in, n_time, plan->acc, plan->fresh, static_cast<cudaStream_t>(stream));
  if (st != XCORR_OK) return st;
  plan->samples += n_time;
  plan->fresh = false;
  return XCORR_OK;
}

xcorr_status xcorr_dump(xcorr_plan plan, void* out, int out_on_device, unsigned flags, void* stream,
                        int64_t* n_samples) {
  xc::NvtxRange range("xcorr_dump");
  xcorr_status st = plan_ok(plan);
  if (st != XCORR_OK) return st;
  if (!out) return fail(XCORR_ERR_INVALID_ARG, "out is NULL");
  if (flags & ~(XCORR_DUMP_RESET | XCORR_DUMP_ADD_WIDE)) return fail(XCORR_ERR_INVALID_ARG, "unknown dump flag");
  const bool wide = (flags & XCORR_DUMP_ADD_WIDE) != 0;
  if (wide && !out_on_device) return fail(XCORR_ERR_INVALID_ARG, "XCORR_DUMP_ADD_WIDE needs device memory");
  if (wide && reinterpret_cast<uintptr_t>(out) % 16)
    return fail(XCORR_ERR_INVALID_ARG, "the wide output must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t total = (int64_t)plan->cfg.n_channels * plan->n_pairs;
  const size_t bytes = (size_t)total * 8;
  cudaError_t e;
  if (plan->fresh) {  // nothing integrated since the last reset: the integration is zero
    e = cudaMemsetAsync(plan->acc, 0, bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "accumulator clear");
    plan->fresh = false;
  }
  if (wide) {
    if (plan->cfg.fmt == XCORR_IN_CF32)
      e = xc::launch_fold_wide_f64(static_cast<const float2*>(plan->acc), static_cast<double*>(out), total, s);
    else
      e = xc::launch_fold_wide_i64(static_cast<const int2*>(plan->acc), static_cast<int64_t*>(out), total, s);
    if (e != cudaSuccess) return cuda_fail(e, "fold launch");
  } else {
    e = cudaMemcpyAsync(out, plan->acc, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "dump copy");
  }
  e = cudaMemcpyAsync(plan->status_host, plan->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  if (n_samples) *n_samples = plan->samples;
  if (flags & XCORR_DUMP_RESET) {
    plan->samples = 0;
    plan->fresh = true;
  }
  return XCORR_OK;
}

xcorr_status xcorr_accum_load(xcorr_plan plan, const void* src, int src_on_device, int64_t n_samples, void* stream) {
  xcorr_status st = plan_ok(plan);
  if (st != XCORR_OK) return st;
  if (!src) return fail(XCORR_ERR_INVALID_ARG, "src is NULL");
  if (n_samples < 0) return fail(XCORR_ERR_INVALID_ARG, "n_samples must be >= 0");
  if (n_samples > plan->max_integration)
    return fail(XCORR_ERR_OVERFLOW, "n_samples exceeds " + std::to_string(plan->max_integration) +
                                        " samples (the exact range of one dump)");
  if (!plan->fresh || plan->samples != 0)
    return fail(XCORR_ERR_INVALID_ARG, "the plan holds an integration: dump it with XCORR_DUMP_RESET first");
  const size_t bytes = (size_t)plan->cfg.n_channels * plan->n_pairs * 8;
  const cudaError_t e = cudaMemcpyAsync(plan->acc, src, bytes,
                                        src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                        static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "accumulator load");
  plan->samples = n_samples;
  plan->fresh = false;
  return XCORR_OK;
}

xcorr_status xcorr_execute_dump(xcorr_plan plan, const void* d_in, int n_time, void* out, int out_on_device,
                                unsigned flags, void* stream, int64_t* n_samples) {
  xc::NvtxRange range("xcorr_execute_dump");
  xcorr_status st = check_execute(plan, d_in, n_time);
  if (st != XCORR_OK) return st;
  if (!out) return fail(XCORR_ERR_INVALID_ARG, "out is NULL");
  if (flags & ~(XCORR_DUMP_RESET | XCORR_DUMP_ADD_WIDE)) return fail(XCORR_ERR_INVALID_ARG, "unknown dump flag");
  const bool direct = plan->fresh && (flags & XCORR_DUMP_RESET) && !(flags & XCORR_DUMP_ADD_WIDE) && out_on_device;
  if (!direct) {
    st = xcorr_execute(plan, d_in, n_time, stream);
    if (st != XCORR_OK) return st;
    return xcorr_dump(plan, out, out_on_device, flags, stream, n_samples);
  }
  // This execute is the whole integration and it is not kept: the X kernel
  // writes it straight into the caller's buffer and the plan stays reset.  (No
  // copy of the status word follows, which would put a copy between every two
  // kernels of back-to-back calls: a kernel failure is reported by xcorr_sync.)
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = run_execute(plan, d_in, n_time, out, true, s);
  if (st != XCORR_OK) return st;
  if (n_samples) *n_samples = n_time;
  return XCORR_OK;
}

xcorr_status xcorr_execute_dump_host(xcorr_plan plan, const void* h_in, int n_time, void* h_out, int n_groups,
                                     void* stream) {
  xc::NvtxRange range("xcorr_execute_dump_host");
  xcorr_status st = check_execute(plan, h_in, n_time);
  if (st != XCORR_OK) return st;
  if (!h_out) return fail(XCORR_ERR_INVALID_ARG, "h_out is NULL");
  if (!plan->fresh || plan->samples != 0)
    return fail(XCORR_ERR_INVALID_ARG, "the plan holds an integration: dump it with XCORR_DUMP_RESET first");
  if (n_groups < 0) return fail(XCORR_ERR_INVALID_ARG, "n_groups must be >= 0");
  const int C = plan->cfg.n_channels, N = plan->n_inputs;
  const size_t in_elem = plan->cfg.fmt == XCORR_IN_CI4 ? 1 : plan->cfg.fmt == XCORR_IN_CI8 ? 2 : 8;
  const size_t chan_bytes = in_elem * N;  // one channel of one sample
  const size_t row_bytes = chan_bytes * C;
  const size_t stage_bytes = row_bytes * plan->cfg.max_time_per_exec;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  // made on first use, each piece on its own so that a failed call leaves nothing half-made
  if (!plan->host_stage) {
    if ((e = cudaMalloc(&plan->host_stage, stage_bytes)) != cudaSuccess) {
      plan->host_stage = nullptr;
      cudaGetLastError();
      return fail(XCORR_ERR_OOM, "host-execute staging buffer: " + std::string(cudaGetErrorString(e)));
    }
    plan->host_stage_bytes = stage_bytes;
    plan->device_bytes += stage_bytes;
  }
  if (!plan->s_down && (e = cudaStreamCreateWithFlags(&plan->s_down, cudaStreamNonBlocking)) != cudaSuccess) {
    plan->s_down = nullptr;
    return cuda_fail(e, "stream create");
  }
  for (cudaEvent_t* ev : {&plan->ev_down}) {
    if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) {
      *ev = nullptr;
      return cuda_fail(e, "event create");
    }
  }
  for (int g = 0; g < xc::kMaxGroups; ++g)
    for (cudaEvent_t* ev : {&plan->ev_up[g], &plan->ev_group_done[g]})
      if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) {
        *ev = nullptr;
        return cuda_fail(e, "event create");
      }
  uint8_t* stage = static_cast<uint8_t*>(plan->host_stage);
  const size_t out_chan_bytes = static_cast<size_t>(plan->n_pairs) * 8;
  if (!(plan->engine == XCORR_ENGINE_TENSOR && fused_applies(plan, stage))) {
    // one piece: up, X-stage, down, in order on the caller's stream
    if ((e = cudaMemcpyAsync(stage, h_in, row_bytes * n_time, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "input copy");
    if ((st = run_execute(plan, stage, n_time, plan->acc, true, s)) != XCORR_OK) return st;
    if ((e = cudaMemcpyAsync(h_out, plan->acc, out_chan_bytes * C, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(e, "output copy");
  } else {
    // channel groups: group g goes up on s_unpack, is correlated on s_x[g % 2] (a
    // launch can start on the SMs the previous one's tail leaves idle) and comes
    // down on s_down while later groups are still moving
    // by default as many groups as keep each 2-D copy row >= 64 KB: narrower rows
    // halve the copy engines' rate (measured: 210 GB/s at 64 KB, 104 GB/s at 32 KB)
    const size_t min_width = size_t(64) << 10;
    int G = n_groups > 0 ? n_groups : static_cast<int>(row_bytes / min_width < 1 ? 1 : row_bytes / min_width);
    G = G > xc::kMaxGroups ? xc::kMaxGroups : G;
    G = G > C ? C : G;
    if ((e = cudaEventRecord(plan->ev_fork, s)) != cudaSuccess) return cuda_fail(e, "fork event");
    for (cudaStream_t t : {plan->s_unpack, plan->s_x[0], plan->s_x[1], plan->s_down})
      if ((e = cudaStreamWaitEvent(t, plan->ev_fork, 0)) != cudaSuccess) return cuda_fail(e, "fork wait");
    for (int g = 0; g < G; ++g) {
      const int c0 = static_cast<int>(static_cast<int64_t>(C) * g / G);
      const int c1 = static_cast<int>(static_cast<int64_t>(C) * (g + 1) / G);
      if (c1 <= c0) continue;
      const size_t off = chan_bytes * c0, width = chan_bytes * (c1 - c0);
      cudaStream_t sx = plan->s_x[g & 1];
      int2* out_g = static_cast<int2*>(plan->acc) + static_cast<int64_t>(c0) * plan->n_pairs;
      if ((e = cudaMemcpy2DAsync(stage + off, row_bytes, static_cast<const uint8_t*>(h_in) + off, row_bytes, width,
                                 n_time, cudaMemcpyHostToDevice, plan->s_unpack)) != cudaSuccess ||
          (e = cudaEventRecord(plan->ev_up[g], plan->s_unpack)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(sx, plan->ev_up[g], 0)) != cudaSuccess)
        return cuda_fail(e, "group input copy");
      if ((e = xc::launch_xcorr_tc_fused_ci4(stage + off, C, plan->tune_variant, n_time, c1 - c0, N, out_g, false,
                                             plan->status, plan->num_sms, sx)) != cudaSuccess)
        return cuda_fail(e, "fused X kernel launch");
      if ((e = cudaEventRecord(plan->ev_group_done[g], sx)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(plan->s_down, plan->ev_group_done[g], 0)) != cudaSuccess ||
          (e = cudaMemcpyAsync(static_cast<uint8_t*>(h_out) + out_chan_bytes * c0, out_g, out_chan_bytes * (c1 - c0),
                               cudaMemcpyDeviceToHost, plan->s_down)) != cudaSuccess)
        return cuda_fail(e, "group output copy");
    }
    // join: every group's copy-out is on s_down, after its X launch and its input copy
    if ((e = cudaEventRecord(plan->ev_down, plan->s_down)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, plan->ev_down, 0)) != cudaSuccess)
      return cuda_fail(e, "join");
  }
  if ((e = cudaMemcpyAsync(plan->status_host, plan->status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "status copy");
  return XCORR_OK;
}

xcorr_status xcorr_sync(xcorr_plan plan, void* stream) {
  xcorr_status st = plan_ok(plan);
  if (st != XCORR_OK) return st;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int code = 0;
  e = cudaMemcpy(&code, plan->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (code) {
    plan->sticky = code;
    return plan_ok(plan);
  }
  return XCORR_OK;
}

xcorr_status xcorr_plan_query(xcorr_plan plan, xcorr_plan_info* info) {
  if (!plan || !info) return fail(XCORR_ERR_INVALID_ARG, "plan or info is NULL");
  info->n_inputs = plan->n_inputs;
  info->n_channels = plan->cfg.n_channels;
  info->n_pairs = plan->n_pairs;
  info->engine = plan->engine;
  info->samples_integrated = plan->samples;
  info->max_integration = plan->max_integration;
  info->device_bytes = plan->device_bytes;
  info->output_bytes = (size_t)plan->cfg.n_channels * plan->n_pairs * 8;
  const bool fused = plan->engine == XCORR_ENGINE_TENSOR && plan->cfg.fmt == XCORR_IN_CI4 && !plan->tune_unfused &&
                     plan->n_inputs % 16 == 0;
  info->kernels_per_execute = fused ? xc::fused_launches(plan->cfg.max_time_per_exec)
                              : plan->engine == XCORR_ENGINE_TENSOR ? 2 * tensor_groups(plan)
                                                                     : 1;
  info->tuning.stage_variant = plan->tune_variant;
  info->tuning.groups = fused ? 1 : tensor_groups(plan);
  info->tuning.x_streams = plan->tune_x_streams;
  info->tuning.unfused = plan->tune_unfused;
  return XCORR_OK;
}

xcorr_status xcorr_plan_set_tuning(xcorr_plan plan, const xcorr_tuning* t) {
  xcorr_status st = plan_ok(plan);
  if (st != XCORR_OK) return st;
  if (!t) return fail(XCORR_ERR_INVALID_ARG, "tuning is NULL");
  if (t->stage_variant < 0 || t->stage_variant >= xc::kFusedVariants)
    return fail(XCORR_ERR_INVALID_ARG, "stage_variant must be in [0, " + std::to_string(xc::kFusedVariants - 1) + "]");
  if (t->groups < 0 || t->groups > xc::kMaxGroups) return fail(XCORR_ERR_INVALID_ARG, "groups must be in [0, 8]");
  if (t->x_streams != 1 && t->x_streams != 2) return fail(XCORR_ERR_INVALID_ARG, "x_streams must be 1 or 2");
  if (t->unfused != 0 && t->unfused != 1) return fail(XCORR_ERR_INVALID_ARG, "unfused must be 0 or 1");
  plan->tune_variant = t->stage_variant;
  plan->tune_groups = t->groups;
  plan->tune_x_streams = t->x_streams;
  plan->tune_unfused = t->unfused;
  return XCORR_OK;
}

xcorr_status xcorr_autotune(xcorr_plan plan, const void* d_in, int n_time, void* stream, xcorr_tuning* best,
                            float* best_ms) {
  xcorr_status st = plan_ok(plan);
  if (st != XCORR_OK) return st;
  if (!d_in || n_time < 1 || n_time > plan->cfg.max_time_per_exec)
    return fail(XCORR_ERR_INVALID_ARG, "d_in must be set and n_time in [1, max_time_per_exec]");
  if (plan->engine != XCORR_ENGINE_TENSOR) {  // nothing to tune
    if (best) *best = xcorr_tuning{plan->tune_variant, plan->tune_groups, plan->tune_x_streams, plan->tune_unfused};
    if (best_ms) *best_ms = 0.f;
    return XCORR_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "cudaEventCreate");
  }
  const int saved_cap = plan->prof_cap;
  plan->prof_cap = 0;  // candidates are not profiled
  const int group_choices[] = {1, 2, 4, 8};
  xcorr_tuning winner{plan->tune_variant, plan->tune_groups, plan->tune_x_streams, plan->tune_unfused};
  float winner_ms = 1e30f;
  // candidates: the fused 4-bit kernel (3 stage shapes) where it applies, then
  // every planes-based shape
  plan->tune_unfused = 0;
  const bool fused_ok = fused_applies(plan, d_in);
  for (int uf = fused_ok ? 0 : 1; uf <= 1 && st == XCORR_OK; ++uf)
  for (int v = 0; v < (uf == 0 ? xc::kFusedVariants : xc::kTcVariants) && st == XCORR_OK; ++v) {
    for (int gi = 0; gi < 4 && st == XCORR_OK; ++gi) {
      for (int xs = 1; xs <= 2 && st == XCORR_OK; ++xs) {
        if (group_choices[gi] == 1 && xs == 2) continue;  // one group has one X launch
        if (uf == 0 && (gi > 0 || xs > 1)) continue;      // the fused kernel is one launch
        plan->tune_variant = v;
        plan->tune_groups = group_choices[gi];
        plan->tune_x_streams = xs;
        plan->tune_unfused = uf;
        float best_rep = 1e30f;
        for (int rep = 0; rep < 3 && st == XCORR_OK; ++rep) {  // the first run warms up
          cudaEventRecord(e0, s);
          st = run_execute(plan, d_in, n_time, plan->acc, true, s);
          cudaEventRecord(e1, s);
          if (st != XCORR_OK) break;
          if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
            st = cuda_fail(e, "autotune timing");
            break;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0 && ms < best_rep) best_rep = ms;
        }
        if (st == XCORR_OK && best_rep < winner_ms) {
          winner_ms = best_rep;
          winner = xcorr_tuning{v, group_choices[gi], xs, uf};
        }
      }
    }
  }
  plan->prof_cap = saved_cap;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the candidates overwrote the accumulator: the plan starts a new integration
  plan->samples = 0;
  plan->fresh = true;
  plan->tune_variant = winner.stage_variant;
  plan->tune_groups = winner.groups;
  plan->tune_x_streams = winner.x_streams;
  plan->tune_unfused = winner.unfused;
  if (st != XCORR_OK) return st;
  if (best) *best = winner;
  if (best_ms) *best_ms = winner_ms;
  return XCORR_OK;
}

xcorr_status xcorr_autotune_cached(xcorr_plan plan, const void* d_in, int n_time, void* stream, xcorr_tuning* best,
                                   float* best_ms, int* from_cache) {
  xcorr_status st = plan_ok(plan);
  if (st != XCORR_OK) return st;
  if (!d_in || n_time < 1 || n_time > plan->cfg.max_time_per_exec)
    return fail(XCORR_ERR_INVALID_ARG, "d_in must be set and n_time in [1, max_time_per_exec]");
  if (from_cache) *from_cache = 0;
  if (plan->engine != XCORR_ENGINE_TENSOR) return xcorr_autotune(plan, d_in, n_time, stream, best, best_ms);
  const xc::TuneKey key = xc::tune_key("plan", plan->cfg.fmt, plan->n_inputs, plan->cfg.n_channels, n_time);
  xcorr_tuning t{};
  float ms = 0.f;
  if (xc::tune_cache_get(key, &t, &ms)) {
    st = xcorr_plan_set_tuning(plan, &t);
    if (st != XCORR_OK) return st;
    plan->samples = 0;  // as the timed path: the plan starts a new integration
    plan->fresh = true;
    if (best) *best = t;
    if (best_ms) *best_ms = ms;
    if (from_cache) *from_cache = 1;
    return XCORR_OK;
  }
  st = xcorr_autotune(plan, d_in, n_time, stream, &t, &ms);
  if (st != XCORR_OK) return st;
  xc::tune_cache_put(key, t, ms);
  if (best) *best = t;
  if (best_ms) *best_ms = ms;
  return XCORR_OK;
}

xcorr_status xcorr_profile_enable(xcorr_plan plan, int capacity) {
  xcorr_status st = plan_ok(plan);
  if (st != XCORR_OK) return st;
  if (capacity < 0 || capacity > (1 << 16)) return fail(XCORR_ERR_INVALID_ARG, "capacity must be in [0, 65536]");
  free_profile(plan);
  if (capacity == 0) return XCORR_OK;
  const int64_t n = (int64_t)xc::kProfileEvents * capacity;
  plan->prof_events = new (std::nothrow) cudaEvent_t[n]();
  plan->prof_ngroups = new (std::nothrow) int[capacity]();
  if (!plan->prof_events || !plan->prof_ngroups) {
    free_profile(plan);
    return fail(XCORR_ERR_OOM, "host allocation failed");
  }
  plan->prof_cap = capacity;
  for (int64_t k = 0; k < n; ++k) {
    cudaError_t e = cudaEventCreate(&plan->prof_events[k]);
    if (e != cudaSuccess) {
      free_profile(plan);
      return cuda_fail(e, "cudaEventCreate");
    }
  }
  return XCORR_OK;
}

xcorr_status xcorr_profile_read(xcorr_plan plan, float* ms, int capacity, int* count) {
  xcorr_status st = plan_ok(plan);
  if (st != XCORR_OK) return st;
  if (!ms || !count || capacity < 0) return fail(XCORR_ERR_INVALID_ARG, "ms or count is NULL");
  *count = 0;
  if (!plan->prof_cap) return XCORR_OK;
  const int64_t have = plan->prof_count < plan->prof_cap ? plan->prof_count : plan->prof_cap;
  const int64_t n = have < capacity ? have : capacity;
  for (int64_t k = 0; k < n; ++k) {
    const int64_t slot = (plan->prof_count - n + k) % plan->prof_cap;
    cudaEvent_t* ev = plan->prof_events + xc::kProfileEvents * slot;
    const int groups = plan->prof_ngroups[slot];
    float unpack = 0.f, x = 0.f;
    cudaError_t e = cudaEventSynchronize(ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&unpack, ev[0], ev[1]);
    for (int g = 0; g < groups && e == cudaSuccess; ++g) {
      float d = 0.f;
      e = cudaEventSynchronize(ev[3 + 2 * g]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&d, ev[2 + 2 * g], ev[3 + 2 * g]);
      x += d;
    }
    if (e != cudaSuccess) return cuda_fail(e, "profile read");
    ms[2 * k] = unpack;
    ms[2 * k + 1] = x;
  }
  *count = static_cast<int>(n);
  return XCORR_OK;
}

xcorr_status xcorr_destroy(xcorr_plan plan) {
  if (!plan) return XCORR_OK;
  cudaSetDevice(plan->device);
  cudaError_t e = cudaDeviceSynchronize();
  release(plan);
  delete plan;
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize at destroy");
  return XCORR_OK;
}

xcorr_status xcorr_baseline_index(int n_stations, int a, int b, int p, int q, int64_t* idx, int* conj) {
  if (!idx || !conj) return fail(XCORR_ERR_INVALID_ARG, "idx or conj is NULL");
  if (n_stations < 1 || a < 0 || a >= n_stations || b < 0 || b > a || p < 0 || p > 1 || q < 0 || q > 1)
    return fail(XCORR_ERR_INVALID_ARG, "need 0 <= b <= a < n_stations and pols in {0, 1}");
  int64_t i = 2LL * a + p, j = 2LL * b + q;
  *conj = 0;
  if (j > i) {  // only for a == b, p < q: the stored pair is (j, i)
    const int64_t t = i;
    i = j;
    j = t;
    *conj = 1;
  }
  *idx = i * (i + 1) / 2 + j;
  return XCORR_OK;
}

}  // extern "C"
