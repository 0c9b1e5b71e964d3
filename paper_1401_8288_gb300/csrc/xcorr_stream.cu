// xcorr_stream.cu -- the streaming X-stage: packets -> device ring -> X -> dumps.
//
// The paper's receiving server (Sec. 2.3, Sec. 2.4, Fig. 4) runs capture,
// unpack-and-reorder and GPU threads over ring buffers of four sub-blocks.
// Here the host only tracks headers (PacketTracker); the bytes go straight
// to the GPU, where a scatter kernel does the placement and corner turn into a
// device ring of blocks in the [t][c][i] order the X kernels read.  CUDA
// streams overlap the stages the way the paper's threads do:
//   h2d x2  -- copies of landing chunks, alternating (two copy engines)
//   copy    -- scatter of each landed chunk, zero-fill of lost packets
//   compute -- the X-stage of each closed block, into a device dump buffer
//   d2h     -- the copy of each finished dump to pinned host memory
// Events order them: a block's X waits for its last scatter and zero-fill, a
// reused ring slot waits for the X of its previous block, and a dump buffer
// is written again only after its previous copy to the host.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "xcorr_internal.h"
#include "xcorr_stream.h"
#include "xcorr_nvtx.h"

namespace xc {
namespace {

// Device copy of the packet geometry.
struct DevGeometry {
  int nt, nch, na, n_inputs, n_channels, n_groups, n_feng;
  int64_t block_bytes, packet_bytes, packets_per_block, words_per_slot;
};

// Byte offset, within its ring block, of the first payload run of packet
// `pidx` (time block tl, channel group grp, F-engine f).
__device__ __forceinline__ int64_t packet_base(const DevGeometry& g, int64_t pidx) {
  const int f = static_cast<int>(pidx % g.n_feng);
  const int64_t q = pidx / g.n_feng;
  const int grp = static_cast<int>(q % g.n_groups);
  const int64_t tl = q / g.n_groups;
  return (tl * g.nt * g.n_channels + static_cast<int64_t>(grp) * g.nch) * g.n_inputs + static_cast<int64_t>(f) * g.na;
}

// One warp per packet: its N_t x N_ch runs of N_a bytes go to rows (t, c) of
// the ring block at input offset f N_a (16-byte vectors), then the packet's
// arrival bit is set.  At most 32 registers a thread (8 blocks of 256 per SM):
// a block then fits beside the persistent X kernel of the previous block,
// which leaves 8192 registers of an SM free, so placement keeps up while the
// X-stage runs.
__global__ void __launch_bounds__(256, 8) scatter_packets_kernel(const uint8_t* __restrict__ landing,
                                                              const int64_t* __restrict__ codes, int64_t p0,
                                                              int64_t p1, uint8_t* __restrict__ ring,
                                                              uint32_t* __restrict__ bits, DevGeometry g) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const int vec_per_run = g.na >> 4;
  const int n_vec = g.nt * g.nch * vec_per_run;
  for (int64_t k = p0 + w0; k < p1; k += nw) {
    const int64_t code = codes[k];
    if (code < 0) continue;
    const int slot = static_cast<int>(code >> kSlotShift);
    const int64_t pidx = code & ((INT64_C(1) << kSlotShift) - 1);
    uint8_t* base = ring + slot * g.block_bytes + packet_base(g, pidx);
    const uint4* src = reinterpret_cast<const uint4*>(landing + k * g.packet_bytes + XCORR_PACKET_HEADER_BYTES);
    for (int v = lane; v < n_vec; v += 32) {
      const int run = v / vec_per_run, w = v - run * vec_per_run;
      const int tt = run / g.nch, cc = run - tt * g.nch;
      *reinterpret_cast<uint4*>(base + (static_cast<int64_t>(tt) * g.n_channels + cc) * g.n_inputs + w * 16) =
          src[v];
    }
    if (lane == 0) atomicOr(&bits[slot * g.words_per_slot + (pidx >> 5)], 1u << (pidx & 31));
  }
}

// Closing a block: every packet whose bit is clear is zero-filled (a CI4 zero
// is 0 + 0i), and the slot's bits are cleared for its next block.  One warp
// per 32 packets (one bitmap word); at most 32 registers, as for the scatter.
__global__ void __launch_bounds__(256, 8) close_block_kernel(uint8_t* __restrict__ ring, uint32_t* __restrict__ bits,
                                                          int slot, DevGeometry g) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const int vec_per_run = g.na >> 4;
  const int n_vec = g.nt * g.nch * vec_per_run;
  uint32_t* slot_bits = bits + slot * g.words_per_slot;
  uint8_t* block = ring + slot * g.block_bytes;
  for (int64_t wi = w0; wi < g.words_per_slot; wi += nw) {
    const int64_t p0 = wi * 32;
    const int64_t n_here = g.packets_per_block - p0 < 32 ? g.packets_per_block - p0 : 32;
    const uint32_t valid = n_here >= 32 ? 0xFFFFFFFFu : ((1u << n_here) - 1u);
    uint32_t missing = ~slot_bits[wi] & valid;
    while (missing) {
      const int b = __ffs(missing) - 1;
      missing &= missing - 1;
      uint8_t* base = block + packet_base(g, p0 + b);
      for (int v = lane; v < n_vec; v += 32) {
        const int run = v / vec_per_run, w = v - run * vec_per_run;
        const int tt = run / g.nch, cc = run - tt * g.nch;
        *reinterpret_cast<uint4*>(base + (static_cast<int64_t>(tt) * g.n_channels + cc) * g.n_inputs + w * 16) =
            make_uint4(0, 0, 0, 0);
      }
    }
    __syncwarp();
    if (lane == 0) slot_bits[wi] = 0;
  }
}

int grid_for(int64_t warps, int num_sms) {
  const int64_t blocks = (warps + 7) / 8;  // 8 warps per 256-thread block
  const int64_t cap = static_cast<int64_t>(num_sms) * 8;
  return static_cast<int>(blocks < 1 ? 1 : blocks < cap ? blocks : cap);
}

using Clock = std::chrono::steady_clock;

}  // namespace
}  // namespace xc

struct DumpRec {
  xcorr_stream_s* owner = nullptr;
  int64_t index = 0, n_samples = 0, lost = 0;
  int host_buf = -1;
  std::chrono::steady_clock::time_point t_close;
  double latency_ms = 0.0;
  bool done = false;
};

struct xcorr_stream_s {
  xcorr_plan plan = nullptr;
  xcorr_stream_config cfg{};
  xc::StreamGeometry g;
  xc::DevGeometry dg{};
  std::unique_ptr<xc::PacketTracker> tracker;
  int64_t out_bytes = 0, chunk_bytes = 0;
  // device
  uint8_t* ring = nullptr;
  uint32_t* bits = nullptr;
  uint8_t* d_landing = nullptr;
  int64_t* d_codes = nullptr;
  void* d_out[2] = {nullptr, nullptr};
  // pinned host
  uint8_t* h_landing = nullptr;
  int64_t* h_codes = nullptr;
  std::vector<void*> h_out;
  cudaStream_t s_copy = nullptr, s_comp = nullptr, s_d2h = nullptr;
  cudaStream_t s_h2d[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> chunk_done, chunk_landed, slot_free, block_ready;
  cudaEvent_t comp_done[2] = {nullptr, nullptr}, out_free[2] = {nullptr, nullptr};
  std::vector<xcorr_block_event> events, chunk_events;
  int64_t next_chunk = 0;
  int acquired = -1;
  // the dump being integrated
  bool period_open = false;
  int64_t period = 0, period_samples = 0, period_lost = 0;
  bool period_fresh = true;
  int out_j = 0;
  // finished dumps
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::unique_ptr<DumpRec>> dumps;
  std::vector<int64_t> host_owner;  // dump whose copy each host buffer holds (or is receiving)
  int64_t dumps_with_data = 0;
  xcorr_status sticky = XCORR_OK;
};

namespace {

using xc::Clock;

void CUDART_CB dump_copied(void* p) {
  auto* r = static_cast<DumpRec*>(p);
  std::lock_guard<std::mutex> lk(r->owner->mu);
  r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_close).count();
  r->done = true;
  r->owner->cv.notify_all();
}

xcorr_status cuda_err(xcorr_stream s, cudaError_t e, const char* what) {
  s->sticky = XCORR_ERR_CUDA;
  return xc::set_error(XCORR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Copy the finished dump to the host (or record an empty one) and start the next.
xcorr_status issue_dump(xcorr_stream s) {
  auto rec = std::make_unique<DumpRec>();
  rec->owner = s;
  rec->index = s->period;
  rec->n_samples = s->period_samples;
  rec->lost = s->period_lost;
  rec->t_close = Clock::now();
  cudaError_t e;
  if (s->period_samples > 0) {
    rec->host_buf = static_cast<int>(s->dumps_with_data++ % s->cfg.n_host_dumps);
    const int j = s->out_j;
    if ((e = cudaEventRecord(s->comp_done[j], s->s_comp)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s->s_d2h, s->comp_done[j], 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->h_out[rec->host_buf], s->d_out[j], s->out_bytes, cudaMemcpyDeviceToHost,
                             s->s_d2h)) != cudaSuccess ||
        (e = cudaLaunchHostFunc(s->s_d2h, dump_copied, rec.get())) != cudaSuccess ||
        (e = cudaEventRecord(s->out_free[j], s->s_d2h)) != cudaSuccess)
      return cuda_err(s, e, "dump copy");
    s->out_j ^= 1;
  } else {
    rec->done = true;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (rec->host_buf >= 0) s->host_owner[rec->host_buf] = static_cast<int64_t>(s->dumps.size());
    s->dumps.push_back(std::move(rec));
  }
  s->period += 1;
  s->period_samples = 0;
  s->period_lost = 0;
  s->period_fresh = true;
  return XCORR_OK;
}

xcorr_status handle_event(xcorr_stream s, const xcorr_block_event& ev) {
  cudaError_t e;
  if (ev.kind == XCORR_EVENT_OPEN) {
    // the slot's previous block must be correlated before its bytes are overwritten
    if ((e = cudaStreamWaitEvent(s->s_copy, s->slot_free[ev.slot], 0)) != cudaSuccess)
      return cuda_err(s, e, "slot wait");
    return XCORR_OK;
  }
  const int64_t bpd = s->cfg.blocks_per_dump;
  if (!s->period_open) {
    s->period_open = true;
    s->period = ev.block / bpd;
  }
  s->period_lost += ev.lost;
  if (ev.received > 0) {
    const int grid = xc::grid_for(s->dg.words_per_slot, s->plan->num_sms);
    xc::close_block_kernel<<<grid, 256, 0, s->s_copy>>>(s->ring, s->bits, ev.slot, s->dg);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(s, e, "close kernel");
    if ((e = cudaEventRecord(s->block_ready[ev.slot], s->s_copy)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s->s_comp, s->block_ready[ev.slot], 0)) != cudaSuccess)
      return cuda_err(s, e, "block ready");
    if (s->period_fresh && (e = cudaStreamWaitEvent(s->s_comp, s->out_free[s->out_j], 0)) != cudaSuccess)
      return cuda_err(s, e, "dump buffer wait");
    xcorr_status st = xc::execute_into(s->plan, s->ring + ev.slot * s->g.block_bytes, s->g.block_samples,
                                       s->d_out[s->out_j], s->period_fresh, s->s_comp);
    if (st != XCORR_OK) {
      s->sticky = st;
      return st;
    }
    if ((e = cudaEventRecord(s->slot_free[ev.slot], s->s_comp)) != cudaSuccess)
      return cuda_err(s, e, "slot free");
    s->period_samples += s->g.block_samples;
    s->period_fresh = false;
  }
  if ((ev.block + 1) % bpd == 0) return issue_dump(s);
  return XCORR_OK;
}

xcorr_status scatter(xcorr_stream s, int chunk, int64_t p0, int64_t p1) {
  if (p1 <= p0) return XCORR_OK;
  const int grid = xc::grid_for(p1 - p0, s->plan->num_sms);
  xc::scatter_packets_kernel<<<grid, 256, 0, s->s_copy>>>(
      s->d_landing + chunk * s->chunk_bytes, s->d_codes + static_cast<int64_t>(chunk) * s->cfg.chunk_packets, p0, p1,
      s->ring, s->bits, s->dg);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? XCORR_OK : cuda_err(s, e, "scatter kernel");
}

xcorr_status stream_ok(xcorr_stream s) {
  if (!s) return xc::set_error(XCORR_ERR_INVALID_ARG, "stream is NULL");
  if (s->sticky != XCORR_OK) return xc::set_error(s->sticky, "the stream failed earlier; destroy it");
  return xc::plan_check(s->plan);
}

void free_stream(xcorr_stream s) {
  if (s->s_copy) cudaStreamSynchronize(s->s_copy);
  if (s->s_comp) cudaStreamSynchronize(s->s_comp);
  if (s->s_d2h) cudaStreamSynchronize(s->s_d2h);
  for (cudaStream_t st : s->s_h2d)
    if (st) cudaStreamSynchronize(st);
  for (auto* v : {&s->chunk_done, &s->chunk_landed, &s->slot_free, &s->block_ready})
    for (auto ev : *v)
      if (ev) cudaEventDestroy(ev);
  for (int j = 0; j < 2; ++j) {
    if (s->comp_done[j]) cudaEventDestroy(s->comp_done[j]);
    if (s->out_free[j]) cudaEventDestroy(s->out_free[j]);
    if (s->d_out[j]) cudaFree(s->d_out[j]);
  }
  for (cudaStream_t st : {s->s_copy, s->s_comp, s->s_d2h, s->s_h2d[0], s->s_h2d[1]})
    if (st) cudaStreamDestroy(st);
  if (s->ring) cudaFree(s->ring);
  if (s->bits) cudaFree(s->bits);
  if (s->d_landing) cudaFree(s->d_landing);
  if (s->d_codes) cudaFree(s->d_codes);
  if (s->h_landing) cudaFreeHost(s->h_landing);
  if (s->h_codes) cudaFreeHost(s->h_codes);
  for (void* h : s->h_out)
    if (h) cudaFreeHost(h);
}

}  // namespace

extern "C" {

xcorr_status xcorr_stream_create(xcorr_stream* out, xcorr_plan plan, const xcorr_stream_config* cfg) {
  if (!out || !cfg) return xc::set_error(XCORR_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  xcorr_status st = xc::plan_check(plan);
  if (st != XCORR_OK) return st;
  if (plan->cfg.fmt != XCORR_IN_CI4) return xc::set_error(XCORR_ERR_UNSUPPORTED, "streams carry 4+4-bit packets");
  std::unique_ptr<xcorr_stream_s> s(new (std::nothrow) xcorr_stream_s);
  if (!s) return xc::set_error(XCORR_ERR_OOM, "stream");
  std::string err;
  if (!s->g.init(*cfg, plan->n_inputs, plan->cfg.n_channels, &err)) return xc::set_error(XCORR_ERR_INVALID_ARG, err);
  if (cfg->block_samples > plan->cfg.max_time_per_exec)
    return xc::set_error(XCORR_ERR_INVALID_ARG, "block_samples exceeds the plan's max_time_per_exec");
  if (static_cast<int64_t>(cfg->blocks_per_dump) * cfg->block_samples > plan->max_integration)
    return xc::set_error(XCORR_ERR_OVERFLOW, "a dump would exceed the plan's exact integration bound");
  s->plan = plan;
  s->cfg = *cfg;
  const xc::StreamGeometry& g = s->g;
  s->dg = xc::DevGeometry{g.nt, g.nch, g.na, g.n_inputs, g.n_channels, g.n_groups, g.n_feng, g.block_bytes,
                          g.packet_bytes, g.packets_per_block, (g.packets_per_block + 31) / 32};
  s->out_bytes = static_cast<int64_t>(plan->cfg.n_channels) * plan->n_pairs * 8;
  s->chunk_bytes = cfg->chunk_packets * g.packet_bytes;
  const int64_t ring_bytes = g.block_bytes * g.n_blocks;
  const int64_t bits_bytes = s->dg.words_per_slot * 4 * g.n_blocks;
  const int64_t landing_bytes = s->chunk_bytes * cfg->n_chunks;
  const int64_t codes_bytes = cfg->chunk_packets * 8 * cfg->n_chunks;
  const int64_t dev_bytes = ring_bytes + bits_bytes + landing_bytes + codes_bytes + 2 * s->out_bytes;
  if (plan->cfg.hbm_budget_bytes > 0 &&
      static_cast<int64_t>(plan->device_bytes) + dev_bytes > static_cast<int64_t>(plan->cfg.hbm_budget_bytes))
    return xc::set_error(XCORR_ERR_BUDGET, "plan + stream need " + std::to_string(plan->device_bytes + dev_bytes) +
                                               " device bytes, over the plan's hbm_budget_bytes");
  s->tracker.reset(new (std::nothrow) xc::PacketTracker(g, cfg->stack_threshold));
  if (!s->tracker) return xc::set_error(XCORR_ERR_OOM, "tracker");
  s->events.resize(4096);
  auto oom = [&](const char* what) {
    free_stream(s.get());
    cudaGetLastError();
    return xc::set_error(XCORR_ERR_OOM, std::string("stream allocation failed: ") + what);
  };
  if (cudaMalloc(&s->ring, ring_bytes) != cudaSuccess) return oom("ring");
  if (cudaMalloc(&s->bits, bits_bytes) != cudaSuccess) return oom("bitmaps");
  if (cudaMalloc(&s->d_landing, landing_bytes) != cudaSuccess) return oom("landing chunks");
  if (cudaMalloc(&s->d_codes, codes_bytes) != cudaSuccess) return oom("placement codes");
  for (int j = 0; j < 2; ++j)
    if (cudaMalloc(&s->d_out[j], s->out_bytes) != cudaSuccess) return oom("dump buffers");
  if (cudaHostAlloc(&s->h_landing, landing_bytes, cudaHostAllocDefault) != cudaSuccess) return oom("pinned chunks");
  if (cudaHostAlloc(&s->h_codes, codes_bytes, cudaHostAllocDefault) != cudaSuccess) return oom("pinned codes");
  s->h_out.assign(cfg->n_host_dumps, nullptr);
  s->host_owner.assign(cfg->n_host_dumps, -1);
  for (auto& h : s->h_out)
    if (cudaHostAlloc(&h, s->out_bytes, cudaHostAllocDefault) != cudaSuccess) return oom("pinned dumps");
  cudaError_t e;
  auto fail_cuda = [&](const char* what) {
    free_stream(s.get());
    return xc::set_error(XCORR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  if ((e = cudaMemset(s->bits, 0, bits_bytes)) != cudaSuccess) return fail_cuda("bitmap reset");
  if ((e = cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->s_d2h, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->s_h2d[0], cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->s_h2d[1], cudaStreamNonBlocking)) != cudaSuccess)
    return fail_cuda("stream create");
  auto make_events = [&](std::vector<cudaEvent_t>& v, int n) {
    v.assign(n, nullptr);
    for (auto& ev : v)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return false;
    return true;
  };
  if (!make_events(s->chunk_done, cfg->n_chunks) || !make_events(s->chunk_landed, cfg->n_chunks) ||
      !make_events(s->slot_free, g.n_blocks) ||
      !make_events(s->block_ready, g.n_blocks))
    return fail_cuda("event create");
  for (int j = 0; j < 2; ++j)
    if ((e = cudaEventCreateWithFlags(&s->comp_done[j], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s->out_free[j], cudaEventDisableTiming)) != cudaSuccess)
      return fail_cuda("event create");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail_cuda("stream setup");
  *out = s.release();
  return XCORR_OK;
}

xcorr_status xcorr_stream_acquire(xcorr_stream s, void** chunk, int64_t* capacity_packets) {
  xcorr_status st = stream_ok(s);
  if (st != XCORR_OK) return st;
  if (!chunk || !capacity_packets) return xc::set_error(XCORR_ERR_INVALID_ARG, "null argument");
  if (s->acquired >= 0) return xc::set_error(XCORR_ERR_INVALID_ARG, "a chunk is already acquired; commit it first");
  const int k = static_cast<int>(s->next_chunk % s->cfg.n_chunks);
  cudaError_t e = cudaEventSynchronize(s->chunk_done[k]);
  if (e != cudaSuccess) return cuda_err(s, e, "chunk wait");
  s->acquired = k;
  *chunk = s->h_landing + k * s->chunk_bytes;
  *capacity_packets = s->cfg.chunk_packets;
  return XCORR_OK;
}

xcorr_status xcorr_stream_commit(xcorr_stream s, int64_t n_packets) {
  xc::NvtxRange range("xcorr_stream_commit");
  xcorr_status st = stream_ok(s);
  if (st != XCORR_OK) return st;
  if (s->acquired < 0) return xc::set_error(XCORR_ERR_INVALID_ARG, "no chunk acquired");
  if (n_packets < 0 || n_packets > s->cfg.chunk_packets)
    return xc::set_error(XCORR_ERR_INVALID_ARG, "n_packets outside [0, chunk_packets]");
  const int k = s->acquired;
  s->acquired = -1;
  s->next_chunk += 1;
  const int64_t pb = s->g.packet_bytes;
  uint8_t* hp = s->h_landing + k * s->chunk_bytes;
  int64_t* hc = s->h_codes + static_cast<int64_t>(k) * s->cfg.chunk_packets;
  int64_t* dc = s->d_codes + static_cast<int64_t>(k) * s->cfg.chunk_packets;
  cudaError_t e;
  // 1. track every header on the host: placement codes and block events
  std::vector<xcorr_block_event>& evs = s->chunk_events;
  evs.clear();
  int64_t done = 0;
  for (int guard = 0; done < n_packets || guard == 0; ++guard) {
    int n_ev = 0;
    const int64_t got = s->tracker->feed(hp + done * pb, pb, n_packets - done, hc + done, s->events.data(),
                                         static_cast<int>(s->events.size()), &n_ev);
    for (int q = 0; q < n_ev; ++q) {
      evs.push_back(s->events[q]);
      evs.back().position += done;
    }
    if (got == 0 && n_ev == 0 && done < n_packets) return xc::set_error(XCORR_ERR_INVALID_ARG, "tracker stalled");
    done += got;
  }
  // 2. codes and payloads go up together on one of two copy streams (a copy
  //    queued behind the scatters would wait for later chunks' transfers)
  cudaStream_t h2d = s->s_h2d[(s->next_chunk - 1) & 1];
  if (n_packets > 0 &&
      ((e = cudaMemcpyAsync(dc, hc, n_packets * 8, cudaMemcpyHostToDevice, h2d)) != cudaSuccess ||
       (e = cudaMemcpyAsync(s->d_landing + k * s->chunk_bytes, hp, n_packets * pb, cudaMemcpyHostToDevice, h2d)) !=
           cudaSuccess ||
       (e = cudaEventRecord(s->chunk_landed[k], h2d)) != cudaSuccess ||
       (e = cudaStreamWaitEvent(s->s_copy, s->chunk_landed[k], 0)) != cudaSuccess))
    return cuda_err(s, e, "chunk copy");
  // 3. scatter between the events, in packet order
  int64_t cursor = 0;
  for (const xcorr_block_event& ev : evs) {
    if ((st = scatter(s, k, cursor, ev.position)) != XCORR_OK) return st;
    cursor = ev.position;
    if ((st = handle_event(s, ev)) != XCORR_OK) return st;
  }
  if ((st = scatter(s, k, cursor, n_packets)) != XCORR_OK) return st;
  if ((e = cudaEventRecord(s->chunk_done[k], s->s_copy)) != cudaSuccess) return cuda_err(s, e, "chunk event");
  return XCORR_OK;
}

xcorr_status xcorr_stream_flush(xcorr_stream s) {
  xcorr_status st = stream_ok(s);
  if (st != XCORR_OK) return st;
  if (s->acquired >= 0) return xc::set_error(XCORR_ERR_INVALID_ARG, "commit the acquired chunk first");
  for (;;) {
    const int n_ev = s->tracker->finish(s->events.data(), static_cast<int>(s->events.size()));
    for (int q = 0; q < n_ev; ++q)
      if ((st = handle_event(s, s->events[q])) != XCORR_OK) return st;
    if (n_ev < static_cast<int>(s->events.size())) break;
  }
  if (s->period_open && (s->period_samples > 0 || s->period_lost > 0)) return issue_dump(s);
  return XCORR_OK;
}

xcorr_status xcorr_stream_counters(xcorr_stream s, xcorr_packet_counters* counters, int64_t* dumps_issued) {
  if (!s) return xc::set_error(XCORR_ERR_INVALID_ARG, "stream is NULL");
  if (counters) *counters = s->tracker->counters();
  if (dumps_issued) {
    std::lock_guard<std::mutex> lk(s->mu);
    *dumps_issued = static_cast<int64_t>(s->dumps.size());
  }
  return XCORR_OK;
}

xcorr_status xcorr_stream_wait_dump(xcorr_stream s, int64_t k, int timeout_ms, xcorr_dump_record* rec) {
  if (!s || !rec) return xc::set_error(XCORR_ERR_INVALID_ARG, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  if (k < 0 || k >= static_cast<int64_t>(s->dumps.size()))
    return xc::set_error(XCORR_ERR_INVALID_ARG, "that dump has not been issued");
  DumpRec* r = s->dumps[k].get();
  if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [&] { return r->done; }))
    return xc::set_error(XCORR_ERR_CUDA, "timed out waiting for the dump copy");
  rec->index = r->index;
  rec->first_seq = r->index * s->cfg.blocks_per_dump * (s->cfg.block_samples / s->dg.nt) * s->dg.n_groups;
  rec->n_samples = r->n_samples;
  rec->lost_packets = r->lost;
  rec->latency_ms = r->latency_ms;
  // the copy is gone once its host buffer was given to a later dump
  rec->data = (r->host_buf >= 0 && s->host_owner[r->host_buf] == k) ? s->h_out[r->host_buf] : nullptr;
  lk.unlock();
  return xc::read_device_status(s->plan);
}

xcorr_status xcorr_stream_destroy(xcorr_stream s) {
  if (!s) return XCORR_OK;
  cudaSetDevice(s->plan->device);
  free_stream(s);
  delete s;
  return XCORR_OK;
}

}  // extern "C"
