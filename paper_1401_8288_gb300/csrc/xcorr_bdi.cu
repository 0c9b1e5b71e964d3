// xcorr_bdi.cu -- baseline-dependent integration.
//
// Sec. 6 of the paper plans per-baseline integration lengths: short baselines
// rotate their fringes slowly and can be integrated longer without
// decorrelation, and fewer, longer integrations lower the output data rate.
// Here the baselines are grouped by 128 x 128 tile pair of the input-pair
// triangle (the unit the X kernels compute).  Tile pair t integrates over
// cadence[t] base integrations of the plan; after each base integration one
// pass over the triangle folds the plan's sums into the tile pairs' running
// sums and moves the tile pairs that are due out as dense blocks, so the bytes
// that leave the GPU per base integration shrink with the cadences.
#include <new>
#include <vector>

#include "xcorr_internal.h"

namespace xc {
namespace {

constexpr int kTile = 128;

// Row i and column j of packed pair p = i (i + 1) / 2 + j.
__device__ __forceinline__ void pair_rc(int64_t p, int& i, int& j) {
  int r = static_cast<int>((sqrt(8.0 * static_cast<double>(p) + 1.0) - 1.0) * 0.5);
  while (static_cast<int64_t>(r + 1) * (r + 2) / 2 <= p) ++r;
  while (static_cast<int64_t>(r) * (r + 1) / 2 > p) --r;
  i = r;
  j = static_cast<int>(p - static_cast<int64_t>(r) * (r + 1) / 2);
}

// One thread per (channel, pair): v = running sum (+ the plan's base
// integration); a due tile pair's entry goes to its block and its running sum
// restarts at zero, the others keep v.
__global__ void __launch_bounds__(256) bdi_fold_emit_kernel(const int2* __restrict__ base, int2* __restrict__ run,
                                                            const int* __restrict__ slot, int2* __restrict__ out,
                                                            int64_t n_pairs, int n_chan, int add_base) {
  const int64_t total = n_pairs * n_chan;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(q / n_pairs);
    const int64_t p = q - static_cast<int64_t>(c) * n_pairs;
    int2 v = run[q];
    if (add_base) {
      const int2 b = base[q];
      v.x += b.x;
      v.y += b.y;
    }
    int i, j;
    pair_rc(p, i, j);
    const int I = i / kTile, J = j / kTile;
    const int s = slot[I * (I + 1) / 2 + J];
    if (s >= 0) {
      out[((static_cast<int64_t>(s) * n_chan + c) * kTile + (i - I * kTile)) * kTile + (j - J * kTile)] = v;
      run[q] = make_int2(0, 0);
    } else {
      run[q] = v;
    }
  }
}

}  // namespace
}  // namespace xc

struct xcorr_bdi_s {
  xcorr_plan plan = nullptr;
  int nb = 0, n_tp = 0;
  std::vector<int> cadence;
  std::vector<int64_t> samples;  // samples in each tile pair's running sum
  int64_t step = 0;
  int2* run = nullptr;           // [C][P][2] running sums
  int* d_slot = nullptr;         // per tile pair: its block in this step's output, or -1
  void* stage = nullptr;         // output blocks before the copy to the host
  size_t stage_bytes = 0;
};

namespace {

void free_bdi(xcorr_bdi b) {
  if (b->run) cudaFree(b->run);
  if (b->d_slot) cudaFree(b->d_slot);
  if (b->stage) cudaFree(b->stage);
}

}  // namespace

extern "C" {

xcorr_status xcorr_bdi_create(xcorr_bdi* out, xcorr_plan plan, const int* cadence, int n_tile_pairs) {
  if (!out || !cadence) return xc::set_error(XCORR_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  xcorr_status st = xc::plan_check(plan);
  if (st != XCORR_OK) return st;
  if (plan->cfg.fmt == XCORR_IN_CF32)
    return xc::set_error(XCORR_ERR_UNSUPPORTED, "baseline-dependent integration needs integer input");
  const int nb = (plan->n_inputs + xc::kTile - 1) / xc::kTile;
  if (n_tile_pairs != nb * (nb + 1) / 2)
    return xc::set_error(XCORR_ERR_INVALID_ARG, "n_tile_pairs must be nb (nb + 1) / 2 for nb = ceil(N_i / 128) = " +
                                                    std::to_string(nb));
  for (int t = 0; t < n_tile_pairs; ++t)
    if (cadence[t] < 1) return xc::set_error(XCORR_ERR_INVALID_ARG, "every cadence must be >= 1");
  auto* b = new (std::nothrow) xcorr_bdi_s;
  if (!b) return xc::set_error(XCORR_ERR_OOM, "bdi");
  b->plan = plan;
  b->nb = nb;
  b->n_tp = n_tile_pairs;
  b->cadence.assign(cadence, cadence + n_tile_pairs);
  b->samples.assign(n_tile_pairs, 0);
  const size_t run_bytes = static_cast<size_t>(plan->cfg.n_channels) * plan->n_pairs * 8;
  cudaError_t e;
  if ((e = cudaMalloc(&b->run, run_bytes)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_slot, sizeof(int) * n_tile_pairs)) != cudaSuccess ||
      (e = cudaMemset(b->run, 0, run_bytes)) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
    free_bdi(b);
    delete b;
    cudaGetLastError();
    return xc::set_error(XCORR_ERR_OOM, std::string("bdi allocation: ") + cudaGetErrorString(e));
  }
  *out = b;
  return XCORR_OK;
}

xcorr_status xcorr_bdi_step(xcorr_bdi b, void* out, int out_on_device, void* stream, int* n_due, int* due,
                            int64_t* samples) {
  if (!b || !out || !n_due || !due || !samples) return xc::set_error(XCORR_ERR_INVALID_ARG, "null argument");
  xcorr_plan plan = b->plan;
  xcorr_status st = xc::plan_check(plan);
  if (st != XCORR_OK) return st;
  const int64_t base = plan->fresh ? 0 : plan->samples;
  for (int t = 0; t < b->n_tp; ++t)
    if (b->samples[t] + base > plan->max_integration)
      return xc::set_error(XCORR_ERR_OVERFLOW, "tile pair " + std::to_string(t) +
                                                   " would integrate past the exact bound of " +
                                                   std::to_string(plan->max_integration) + " samples");
  std::vector<int> slot(b->n_tp, -1);
  int nd = 0;
  for (int t = 0; t < b->n_tp; ++t)
    if ((b->step + 1) % b->cadence[t] == 0) {
      slot[t] = nd;
      due[nd] = t;
      samples[nd] = b->samples[t] + base;
      ++nd;
    }
  const int C = plan->cfg.n_channels;
  const size_t out_bytes = static_cast<size_t>(nd) * C * xc::kTile * xc::kTile * 8;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  void* dst = out;
  if (!out_on_device && out_bytes > 0) {
    if (b->stage_bytes < out_bytes) {
      if (b->stage) cudaFree(b->stage);
      b->stage = nullptr;
      b->stage_bytes = 0;
      if ((e = cudaMalloc(&b->stage, out_bytes)) != cudaSuccess) {
        cudaGetLastError();
        return xc::set_error(XCORR_ERR_OOM, std::string("bdi staging: ") + cudaGetErrorString(e));
      }
      b->stage_bytes = out_bytes;
    }
    dst = b->stage;
  }
  // the slot table from pageable memory: the copy has read it when the call returns
  if ((e = cudaMemcpyAsync(b->d_slot, slot.data(), sizeof(int) * b->n_tp, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (out_bytes > 0 && (e = cudaMemsetAsync(dst, 0, out_bytes, s)) != cudaSuccess))
    return xc::set_error(XCORR_ERR_CUDA, std::string("bdi setup: ") + cudaGetErrorString(e));
  const int64_t total = static_cast<int64_t>(C) * plan->n_pairs;
  const int64_t want = (total + 255) / 256;
  const int grid = static_cast<int>(want < plan->num_sms * 8LL ? want : plan->num_sms * 8LL);
  xc::bdi_fold_emit_kernel<<<grid < 1 ? 1 : grid, 256, 0, s>>>(static_cast<const int2*>(plan->acc), b->run,
                                                               b->d_slot, static_cast<int2*>(dst), plan->n_pairs,
                                                               C, base > 0 ? 1 : 0);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return xc::set_error(XCORR_ERR_CUDA, std::string("bdi kernel: ") + cudaGetErrorString(e));
  if (dst != out && (e = cudaMemcpyAsync(out, dst, out_bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return xc::set_error(XCORR_ERR_CUDA, std::string("bdi copy: ") + cudaGetErrorString(e));
  // the plan's base integration now lives in the running sums
  plan->samples = 0;
  plan->fresh = true;
  for (int t = 0; t < b->n_tp; ++t) b->samples[t] = slot[t] >= 0 ? 0 : b->samples[t] + base;
  b->step += 1;
  *n_due = nd;
  return XCORR_OK;
}

xcorr_status xcorr_bdi_destroy(xcorr_bdi b) {
  if (!b) return XCORR_OK;
  cudaSetDevice(b->plan->device);
  cudaDeviceSynchronize();
  free_bdi(b);
  delete b;
  return XCORR_OK;
}

}  // extern "C"
