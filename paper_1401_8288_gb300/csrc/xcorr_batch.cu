// xcorr_batch.cu -- many independent correlations of uneven size in one
// persistent tensor-core launch, optionally replayed as a CUDA graph.
//
// A batch holds n subarrays (each its own station count, channel count and
// integration length, 4+4-bit input).  One execute runs a single launch of an
// X kernel over the union of their work items (subarray, channel, I, J),
// sorted longest first and dealt round-robin to the persistent CTAs, so a
// large subarray's tail is filled with the small ones' items instead of
// leaving SMs idle between per-instance launches.  Sec. 2.1: each sub-band
// (here each subarray) is an independent X-stage.
//
// Stage variants 3-5 (the default when every subarray has a multiple of 16
// inputs and fits one exactly-summed block) run the fused 4-bit kernel with
// the A operand in tensor memory straight on the callers' raw inputs; 0-2
// first unpack every subarray into its own E4M3 planes and run the planes
// kernel.  With the fused kernel each subarray may have its own shape, any of
// a 4-bit plan's fused shapes (set by hand or by xcorr_batch_autotune, one
// shape per size class): subarrays whose shape is one of the tensor-memory-A
// kernel's (plan shapes 4-6) form a class with its own item list and one
// shared launch; a subarray with any other shape (the CTA-pair kernel for the
// largest, the small-problem layout, ...) runs as its own launch.  All of these
// launches run side by side on internal streams forked from the caller's, so
// one launch's tail overlaps the others.
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "xcorr_internal.h"
#include "xcorr_nvtx.h"

constexpr int kBatchClasses = 3;  // the tensor-memory-A kernel's batch shapes (plan shapes 4-6)
constexpr int kSoloStreams = 4;   // streams the subarrays with a shape of their own are dealt over
constexpr int kPlanTaShape0 = 4;  // plan shape of the tensor-memory-A kernel's first batch shape

struct xcorr_batch_s {
  int n = 0;
  int device = 0, num_sms = 0;
  int variant = 0;              // 0-2 planes path, 3-5 fused kernel (its variants 0-2)
  std::vector<int> sub_shape;   // fused: each subarray's 4-bit plan shape, 0-10 (4-6: a shared class)
  bool fusable = false;         // every subarray qualifies for the fused kernel
  xc::TaSubDesc* fdescs_host = nullptr;  // fused descriptors (pinned), n entries
  xc::TaSubDesc* fdescs_dev = nullptr;
  std::vector<const void*> ins;  // the inputs the fused descriptors were built for
  int built_variant = -1;        // the variant the device tables hold
  std::vector<xcorr_config> cfg;
  std::vector<int> n_inputs, ni_pad;
  std::vector<int64_t> n_pairs;
  std::vector<void*> planes;
  xc::SubDescHost* descs_host = nullptr;  // n entries (pinned)
  void* descs_dev = nullptr;
  uint4* items_dev = nullptr;
  int n_items = 0;
  // fused classes: item range and shape of each, in items_dev
  int n_classes = 0;
  int class_variant[kBatchClasses] = {}, class_off[kBatchClasses] = {}, class_n[kBatchClasses] = {};
  cudaStream_t class_stream[kBatchClasses] = {};
  cudaEvent_t ev_fork = nullptr, ev_class_done[kBatchClasses] = {};
  std::vector<int> solo;        // subarrays with a shape of their own, largest first
  cudaStream_t solo_stream[kSoloStreams] = {};
  cudaEvent_t ev_solo_done[kSoloStreams] = {};
  int* status = nullptr;
  // graph replay
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
};

namespace {

xcorr_status bfail(xcorr_status st, const std::string& msg) { return xc::set_error(st, msg); }

void batch_release(xcorr_batch b) {
  for (int k = 0; k < kBatchClasses; ++k) {
    if (b->class_stream[k]) cudaStreamDestroy(b->class_stream[k]);
    if (b->ev_class_done[k]) cudaEventDestroy(b->ev_class_done[k]);
  }
  for (int k = 0; k < kSoloStreams; ++k) {
    if (b->solo_stream[k]) cudaStreamDestroy(b->solo_stream[k]);
    if (b->ev_solo_done[k]) cudaEventDestroy(b->ev_solo_done[k]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (void* p : b->planes)
    if (p) cudaFree(p);
  if (b->fdescs_dev) cudaFree(b->fdescs_dev);
  if (b->fdescs_host) cudaFreeHost(b->fdescs_host);
  if (b->descs_dev) cudaFree(b->descs_dev);
  if (b->items_dev) cudaFree(b->items_dev);
  if (b->descs_host) cudaFreeHost(b->descs_host);
  if (b->status) cudaFree(b->status);
}

constexpr int kFusedBase = xc::kTcVariants;  // batch variants kFusedBase + v run the fused kernel's variant v

bool fused_mode(const xcorr_batch_s* b) { return b->variant >= kFusedBase; }

// A fused subarray's shared class (0-2: the tensor-memory-A kernel's batch shapes), or -1 when its
// shape runs it alone.
int ta_class(int plan_shape) {
  return plan_shape >= kPlanTaShape0 && plan_shape < kPlanTaShape0 + kBatchClasses ? plan_shape - kPlanTaShape0 : -1;
}

// The captured graph holds the old shapes: drop it (and the tables) when a shape changes.
void invalidate(xcorr_batch b) {
  b->built_variant = -1;
  if (b->graph_exec) {
    cudaGraphExecDestroy(b->graph_exec);
    cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
  }
}

// The planes path's staging planes, allocated when a planes variant is first chosen.
xcorr_status ensure_planes(xcorr_batch b) {
  for (int s = 0; s < b->n; ++s) {
    if (b->planes[s]) continue;
    const xcorr_config& c = b->cfg[s];
    cudaError_t e = cudaMalloc(&b->planes[s], (size_t)c.n_channels * 2 * c.max_time_per_exec * b->ni_pad[s]);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(XCORR_ERR_OOM, std::string("batch planes: ") + cudaGetErrorString(e));
    }
  }
  return XCORR_OK;
}

// (Re)build the subarray descriptors and the item list for the batch's variant and the given
// inputs (the fused kernel reads them through its tensor maps) and outputs.
xcorr_status build_tables(xcorr_batch b, const void* const* d_ins, void* const* d_outs) {
  const bool fused = fused_mode(b);
  std::vector<uint4> items;
  std::vector<int> cost, cls;
  // classes: the planes path has one (the batch's shape); the fused path one per tensor-memory-A
  // shape in use, and the subarrays of other shapes run alone, largest first
  int class_of[kBatchClasses] = {-1, -1, -1};
  b->n_classes = 0;
  b->solo.clear();
  if (!fused) {
    b->class_variant[b->n_classes++] = b->variant;
  } else {
    for (int k = 0; k < kBatchClasses; ++k) {
      bool used = false;
      for (int s = 0; s < b->n && !used; ++s) used = ta_class(b->sub_shape[s]) == k;
      if (used) {
        class_of[k] = b->n_classes;
        b->class_variant[b->n_classes++] = kFusedBase + k;
      }
    }
    for (int s = 0; s < b->n; ++s)
      if (ta_class(b->sub_shape[s]) < 0) b->solo.push_back(s);
    auto work = [&](int s) {
      return (double)b->cfg[s].n_channels * b->cfg[s].max_time_per_exec * (double)b->n_pairs[s];
    };
    std::stable_sort(b->solo.begin(), b->solo.end(), [&](int a, int c) { return work(a) > work(c); });
  }
  for (int s = 0; s < b->n; ++s) {
    const int cls_s = fused ? ta_class(b->sub_shape[s]) : 0;
    if (fused && cls_s < 0) {  // runs alone: its launcher reads the buffers it is given
      if (d_ins && reinterpret_cast<uintptr_t>(d_ins[s]) % 16)
        return bfail(XCORR_ERR_INVALID_ARG, "subarray " + std::to_string(s) + ": the fused kernels need a 16-byte "
                                                                            "aligned input");
      b->fdescs_host[s].out = d_outs ? static_cast<int2*>(d_outs[s]) : nullptr;
      b->ins[s] = d_ins ? d_ins[s] : nullptr;
      continue;
    }
    const int kt = fused ? xc::fused_ta_stage_samples(cls_s) : xc::tc_stage_samples(1, b->variant);
    const int n_time = b->cfg[s].max_time_per_exec;
    const int C = b->cfg[s].n_channels;
    const int nb = (b->n_inputs[s] + 127) / 128;
    std::string err;
    int n_kt;
    if (fused) {
      xc::TaSubDesc& d = b->fdescs_host[s];
      if (d_ins && !xc::encode_raw_ci4_tmap(&d.tmap, d_ins[s], b->n_inputs[s], C, C, n_time, kt, &err))
        return bfail(XCORR_ERR_INVALID_ARG, "subarray " + std::to_string(s) + ": " + err);
      d.out = d_outs ? static_cast<int2*>(d_outs[s]) : nullptr;
      d.n_pairs = b->n_pairs[s];
      d.n_inputs = b->n_inputs[s];
      d.n_tile_pairs = nb * (nb + 1) / 2;
      d.n_kt = (n_time + kt - 1) / kt;
      d.accumulate = 0;
      n_kt = d.n_kt;
      b->ins[s] = d_ins ? d_ins[s] : nullptr;
    } else {
      if (!xc::encode_plane_tmap(&b->descs_host[s].tmap, b->planes[s], 1, b->n_inputs[s], b->ni_pad[s], n_time,
                                 n_time, 2 * C, kt, &err))
        return bfail(XCORR_ERR_CUDA, err);
      xc::SubDescHost& d = b->descs_host[s];
      d.out = d_outs ? d_outs[s] : nullptr;
      d.n_pairs = b->n_pairs[s];
      d.n_inputs = b->n_inputs[s];
      d.n_kt = (n_time + kt - 1) / kt;
      d.n_tw = (d.n_kt + xc::kTcWindowCI4 / kt - 1) / (xc::kTcWindowCI4 / kt);
      n_kt = d.n_kt;
    }
    for (int c = 0; c < C; ++c)
      for (int I = 0; I < nb; ++I)
        for (int J = 0; J <= I; ++J) {
          items.push_back(make_uint4((unsigned)s, (unsigned)c, (unsigned)I, (unsigned)J));
          cost.push_back(n_kt);
          cls.push_back(fused ? class_of[cls_s] : 0);
        }
  }
  // by class, then longest first: a stable sort keeps each subarray's items channel-major
  std::vector<int> order(items.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return cls[a] != cls[c] ? cls[a] < cls[c] : cost[a] > cost[c]; });
  std::vector<uint4> sorted(items.size());
  for (int k = 0; k < b->n_classes; ++k) b->class_n[k] = 0;
  for (size_t k = 0; k < order.size(); ++k) {
    sorted[k] = items[order[k]];
    ++b->class_n[cls[order[k]]];
  }
  for (int k = 0, off = 0; k < b->n_classes; off += b->class_n[k], ++k) b->class_off[k] = off;
  if (b->items_dev && (int)sorted.size() != b->n_items) {
    cudaFree(b->items_dev);
    b->items_dev = nullptr;
  }
  cudaError_t e;
  if (!b->items_dev && !sorted.empty() &&
      (e = cudaMalloc(&b->items_dev, sorted.size() * sizeof(uint4))) != cudaSuccess)
    return bfail(XCORR_ERR_OOM, std::string("item list: ") + cudaGetErrorString(e));
  b->n_items = (int)sorted.size();
  if ((!sorted.empty() && (e = cudaMemcpy(b->items_dev, sorted.data(), sorted.size() * sizeof(uint4),
                                          cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (fused ? (e = cudaMemcpy(b->fdescs_dev, b->fdescs_host, sizeof(xc::TaSubDesc) * b->n, cudaMemcpyHostToDevice))
             : (e = cudaMemcpy(b->descs_dev, b->descs_host, sizeof(xc::SubDescHost) * b->n,
                               cudaMemcpyHostToDevice))) != cudaSuccess)
    return bfail(XCORR_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
  b->built_variant = b->variant;
  return XCORR_OK;
}

// Enqueue one batch execute: one fused launch, or every unpack and then one X launch.
xcorr_status enqueue(xcorr_batch b, const void* const* d_ins, cudaStream_t s) {
  cudaError_t e;
  if (fused_mode(b) && b->n_classes == 1 && b->solo.empty()) {
    e = xc::launch_xcorr_tc_fused_ta_batch(b->fdescs_dev, b->items_dev, b->n_items, b->class_variant[0] - kFusedBase,
                                           b->status, b->num_sms, s);
    if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("fused batch launch: ") + cudaGetErrorString(e));
    return XCORR_OK;
  }
  if (fused_mode(b)) {
    // one launch per class and one per subarray with a shape of its own, on internal streams
    // forked from s and joined back: they run side by side (each persistent launch takes the
    // SMs the others leave)
    if ((e = cudaEventRecord(b->ev_fork, s)) != cudaSuccess)
      return bfail(XCORR_ERR_CUDA, std::string("fork: ") + cudaGetErrorString(e));
    const int n_solo_streams = (int)b->solo.size() < kSoloStreams ? (int)b->solo.size() : kSoloStreams;
    for (int k = 0; k < n_solo_streams; ++k)
      if ((e = cudaStreamWaitEvent(b->solo_stream[k], b->ev_fork, 0)) != cudaSuccess)
        return bfail(XCORR_ERR_CUDA, std::string("fork wait: ") + cudaGetErrorString(e));
    for (size_t q = 0; q < b->solo.size(); ++q) {
      const int k = b->solo[q];
      const xcorr_config& c = b->cfg[k];
      e = xc::launch_xcorr_tc_fused_ci4(static_cast<const uint8_t*>(d_ins[k]), c.n_channels, b->sub_shape[k],
                                        c.max_time_per_exec, c.n_channels, b->n_inputs[k], b->fdescs_host[k].out,
                                        false, b->status, b->num_sms, b->solo_stream[q % kSoloStreams]);
      if (e != cudaSuccess)
        return bfail(XCORR_ERR_CUDA, "subarray " + std::to_string(k) + " launch: " + cudaGetErrorString(e));
    }
    for (int k = 0; k < n_solo_streams; ++k)
      if ((e = cudaEventRecord(b->ev_solo_done[k], b->solo_stream[k])) != cudaSuccess ||
          (e = cudaStreamWaitEvent(s, b->ev_solo_done[k], 0)) != cudaSuccess)
        return bfail(XCORR_ERR_CUDA, std::string("join: ") + cudaGetErrorString(e));
    for (int k = 0; k < b->n_classes; ++k) {
      cudaStream_t sk = b->class_stream[k];
      if ((e = cudaStreamWaitEvent(sk, b->ev_fork, 0)) != cudaSuccess ||
          (e = xc::launch_xcorr_tc_fused_ta_batch(b->fdescs_dev, b->items_dev + b->class_off[k], b->class_n[k],
                                                  b->class_variant[k] - kFusedBase, b->status, b->num_sms, sk)) !=
              cudaSuccess ||
          (e = cudaEventRecord(b->ev_class_done[k], sk)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(s, b->ev_class_done[k], 0)) != cudaSuccess)
        return bfail(XCORR_ERR_CUDA, std::string("fused batch class launch: ") + cudaGetErrorString(e));
    }
    return XCORR_OK;
  }
  for (int k = 0; k < b->n; ++k) {
    e = xc::launch_unpack_ci4_e4m3(static_cast<const uint8_t*>(d_ins[k]), static_cast<uint8_t*>(b->planes[k]),
                                   b->cfg[k].max_time_per_exec, b->cfg[k].n_channels, b->n_inputs[k], b->ni_pad[k],
                                   b->cfg[k].max_time_per_exec, b->num_sms, s);
    if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("unpack launch: ") + cudaGetErrorString(e));
  }
  e = xc::launch_xcorr_tc_batch(b->descs_dev, b->items_dev, b->n_items, b->variant, b->status, b->num_sms, s);
  if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("batch X launch: ") + cudaGetErrorString(e));
  return XCORR_OK;
}

}  // namespace

extern "C" {

xcorr_status xcorr_batch_create(xcorr_batch* out, const xcorr_config* cfgs, int n) {
  if (!out || !cfgs || n < 1 || n > 4096) return bfail(XCORR_ERR_INVALID_ARG, "need out, cfgs and 1 <= n <= 4096");
  *out = nullptr;
  for (int s = 0; s < n; ++s) {
    const xcorr_config& c = cfgs[s];
    if (c.n_pols != 2 || c.n_stations < 1 || c.n_stations > (1 << 20) || c.n_channels < 1 ||
        c.max_time_per_exec < 1)
      return bfail(XCORR_ERR_INVALID_ARG, "subarray " + std::to_string(s) + ": invalid sizes");
    if (c.fmt != XCORR_IN_CI4)
      return bfail(XCORR_ERR_UNSUPPORTED, "batches take 4+4-bit subarrays (subarray " + std::to_string(s) + ")");
    if (c.max_time_per_exec > xc::kTcWindowCI4)
      return bfail(XCORR_ERR_UNSUPPORTED, "batch subarrays hold at most 130,944 samples per execute");
  }
  int dev = 0, major = 0, minor = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
  if (major != 10 || minor != 3) return bfail(XCORR_ERR_UNSUPPORTED, "needs an sm_103a (GB300) device");

  xcorr_batch b = new (std::nothrow) xcorr_batch_s();
  if (!b) return bfail(XCORR_ERR_OOM, "host allocation failed");
  b->n = n;
  b->device = dev;
  b->num_sms = sms;
  b->cfg.assign(cfgs, cfgs + n);
  size_t budget = 0, need = 0;
  b->fusable = true;
  for (int s = 0; s < n; ++s) {
    const int ni = 2 * cfgs[s].n_stations;
    b->n_inputs.push_back(ni);
    b->ni_pad.push_back((ni + 15) / 16 * 16);
    b->n_pairs.push_back((int64_t)ni * (ni + 1) / 2);
    need += (size_t)cfgs[s].n_channels * 2 * cfgs[s].max_time_per_exec * b->ni_pad.back();
    if (cfgs[s].hbm_budget_bytes) budget = budget ? std::min(budget, cfgs[s].hbm_budget_bytes) : cfgs[s].hbm_budget_bytes;
    b->fusable = b->fusable && ni % 16 == 0 && cfgs[s].max_time_per_exec <= xc::kFusedWindowCI4;
  }
  // the fused kernel reads the raw inputs directly; the planes path needs its staging planes
  b->variant = b->fusable ? kFusedBase : 0;
  b->sub_shape.assign(n, kPlanTaShape0);
  if (!b->fusable && budget && need > budget) {
    delete b;
    return bfail(XCORR_ERR_BUDGET, "the batch needs " + std::to_string(need) + " device bytes of planes, budget " +
                                       std::to_string(budget));
  }
  b->planes.assign(n, nullptr);
  b->ins.assign(n, nullptr);
  for (int s = 0; s < n && e == cudaSuccess && !b->fusable; ++s)
    e = cudaMalloc(&b->planes[s], (size_t)cfgs[s].n_channels * 2 * cfgs[s].max_time_per_exec * b->ni_pad[s]);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&b->fdescs_host), sizeof(xc::TaSubDesc) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->fdescs_dev, sizeof(xc::TaSubDesc) * n);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&b->descs_host), sizeof(xc::SubDescHost) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->descs_dev, sizeof(xc::SubDescHost) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->status, 256);
  if (e == cudaSuccess) e = cudaMemset(b->status, 0, 256);
  for (int k = 0; k < kBatchClasses && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->class_stream[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_class_done[k], cudaEventDisableTiming);
  }
  for (int k = 0; k < kSoloStreams && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->solo_stream[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_solo_done[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    batch_release(b);
    delete b;
    cudaGetLastError();
    return bfail(e == cudaErrorMemoryAllocation ? XCORR_ERR_OOM : XCORR_ERR_CUDA,
                 std::string("batch allocation: ") + cudaGetErrorString(e));
  }
  *out = b;  // the tables are built by the first execute or capture, which name the buffers
  return XCORR_OK;
}

xcorr_status xcorr_batch_set_variant(xcorr_batch b, int stage_variant) {
  if (!b || stage_variant < 0 || stage_variant >= kFusedBase + 3)
    return bfail(XCORR_ERR_INVALID_ARG, "need a batch and stage_variant in [0, 5]");
  if (stage_variant >= kFusedBase && !b->fusable)
    return bfail(XCORR_ERR_UNSUPPORTED,
                 "the fused variants need every subarray to have a multiple of 16 inputs and at most 37,248 samples");
  if (stage_variant < kFusedBase) {
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    xcorr_status st = ensure_planes(b);
    if (st != XCORR_OK) return st;
  }
  b->variant = stage_variant;
  if (stage_variant >= kFusedBase) b->sub_shape.assign(b->n, kPlanTaShape0 + stage_variant - kFusedBase);
  invalidate(b);
  return XCORR_OK;
}

xcorr_status xcorr_batch_set_subarray_variants(xcorr_batch b, const int* variants) {
  if (!b || !variants) return bfail(XCORR_ERR_INVALID_ARG, "batch and variants must not be NULL");
  if (!b->fusable)
    return bfail(XCORR_ERR_UNSUPPORTED, "per-subarray shapes need the fused kernel (every subarray a multiple of 16 "
                                        "inputs and at most 37,248 samples)");
  for (int s = 0; s < b->n; ++s)
    if (variants[s] < 0 || variants[s] >= xc::kFusedVariants)
      return bfail(XCORR_ERR_INVALID_ARG, "subarray " + std::to_string(s) + ": a shape is a 4-bit plan shape, 0 .. " +
                                              std::to_string(xc::kFusedVariants - 1));
  b->variant = kFusedBase;
  b->sub_shape.assign(variants, variants + b->n);
  invalidate(b);
  return XCORR_OK;
}

xcorr_status xcorr_batch_get_subarray_variants(xcorr_batch b, int* variants) {
  if (!b || !variants) return bfail(XCORR_ERR_INVALID_ARG, "batch and variants must not be NULL");
  for (int s = 0; s < b->n; ++s) variants[s] = fused_mode(b) ? b->sub_shape[s] : b->variant;
  return XCORR_OK;
}

xcorr_status xcorr_batch_autotune(xcorr_batch b, const void* const* d_ins, void* const* d_outs, void* stream,
                                  int* variants) {
  if (!b || !d_ins || !d_outs) return bfail(XCORR_ERR_INVALID_ARG, "batch, d_ins and d_outs must not be NULL");
  for (int s = 0; s < b->n; ++s)
    if (!d_ins[s] || !d_outs[s] || reinterpret_cast<uintptr_t>(d_ins[s]) % 16)
      return bfail(XCORR_ERR_INVALID_ARG, "a subarray buffer is NULL or its input is not 16-byte aligned");
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  if (!b->fusable) {  // the planes path has one shape for the whole batch: nothing per subarray
    if (variants)
      for (int s = 0; s < b->n; ++s) variants[s] = b->variant;
    return XCORR_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return bfail(XCORR_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
  }
  std::vector<int> pick(b->n, kPlanTaShape0);
  xcorr_status rs = XCORR_OK;
  for (int s = 0; s < b->n && rs == XCORR_OK; ++s) {
    const xcorr_config& c = b->cfg[s];
    const xc::TuneKey key = xc::tune_key("batch", XCORR_IN_CI4, b->n_inputs[s], c.n_channels, c.max_time_per_exec);
    xcorr_tuning cached{};
    if (xc::tune_cache_get(key, &cached, nullptr) && cached.stage_variant >= 0 &&
        cached.stage_variant < xc::kFusedVariants) {
      pick[s] = cached.stage_variant;
      continue;
    }
    // the subarray alone, with each fused shape (three runs, the first warms up)
    float best = 1e30f;
    for (int v = 0; v < xc::kFusedVariants && rs == XCORR_OK; ++v) {
      float vbest = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        e = xc::launch_xcorr_tc_fused_ci4(static_cast<const uint8_t*>(d_ins[s]), c.n_channels, v,
                                          c.max_time_per_exec, c.n_channels, b->n_inputs[s],
                                          static_cast<int2*>(d_outs[s]), false, b->status, b->num_sms, st);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
          rs = bfail(XCORR_ERR_CUDA, std::string("batch autotune: ") + cudaGetErrorString(e));
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < vbest) vbest = ms;
      }
      if (rs == XCORR_OK && vbest < best) {
        best = vbest;
        pick[s] = v;
      }
    }
    if (rs == XCORR_OK) xc::tune_cache_put(key, xcorr_tuning{pick[s], 1, 1, 0}, best);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rs != XCORR_OK) return rs;
  int code = 0;
  if ((e = cudaMemcpy(&code, b->status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return bfail(XCORR_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
  if (code) return bfail(XCORR_ERR_DEVICE, "a batch kernel reported failure code " + std::to_string(code));
  rs = xcorr_batch_set_subarray_variants(b, pick.data());
  if (rs == XCORR_OK && variants)
    for (int s = 0; s < b->n; ++s) variants[s] = pick[s];
  return rs;
}

xcorr_status xcorr_batch_execute(xcorr_batch b, const void* const* d_ins, void* const* d_outs, void* stream) {
  xc::NvtxRange range("xcorr_batch_execute");
  if (!b || !d_ins || !d_outs) return bfail(XCORR_ERR_INVALID_ARG, "batch, d_ins and d_outs must not be NULL");
  for (int s = 0; s < b->n; ++s)
    if (!d_ins[s] || !d_outs[s]) return bfail(XCORR_ERR_INVALID_ARG, "a subarray buffer is NULL");
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  // the tables are rewritten only when the variant or the buffers they name changed
  const bool fused = fused_mode(b);
  bool same = b->built_variant == b->variant;
  for (int s = 0; s < b->n && same; ++s)
    same = fused ? (b->fdescs_host[s].out == d_outs[s] && b->ins[s] == d_ins[s]) : (b->descs_host[s].out == d_outs[s]);
  if (!same) {
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));  // earlier launches read the tables
    xcorr_status st = build_tables(b, d_ins, d_outs);
    if (st != XCORR_OK) return st;
  }
  return enqueue(b, d_ins, static_cast<cudaStream_t>(stream));
}

xcorr_status xcorr_batch_capture(xcorr_batch b, const void* const* d_ins, void* const* d_outs, void* stream) {
  if (!b || !d_ins || !d_outs) return bfail(XCORR_ERR_INVALID_ARG, "batch, d_ins and d_outs must not be NULL");
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  // (recording only: the graph runs later on whatever stream replays it)
  cudaStreamSynchronize(static_cast<cudaStream_t>(stream));  // earlier launches may still read the tables
  xcorr_status st = build_tables(b, d_ins, d_outs);
  if (st != XCORR_OK) return st;
  if (b->graph_exec) {
    cudaGraphExecDestroy(b->graph_exec);
    cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
  }
  cudaStream_t cap = nullptr;
  if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess)
    return bfail(XCORR_ERR_CUDA, std::string("capture stream: ") + cudaGetErrorString(e));
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st = enqueue(b, d_ins, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    if (st == XCORR_OK && e == cudaSuccess) {
      e = cudaGraphInstantiate(&b->graph_exec, g, 0);
      b->graph = g;
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(cap);
  if (st != XCORR_OK) return st;
  if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  return XCORR_OK;
}

xcorr_status xcorr_batch_replay(xcorr_batch b, void* stream) {
  xc::NvtxRange range("xcorr_batch_replay");
  if (!b || !b->graph_exec) return bfail(XCORR_ERR_INVALID_ARG, "no captured graph: call xcorr_batch_capture first");
  cudaError_t e = cudaGraphLaunch(b->graph_exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return XCORR_OK;
}

xcorr_status xcorr_batch_sync(xcorr_batch b, void* stream) {
  if (!b) return bfail(XCORR_ERR_INVALID_ARG, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
  int code = 0;
  e = cudaMemcpy(&code, b->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
  if (code) return bfail(XCORR_ERR_DEVICE, "a batch kernel reported failure code " + std::to_string(code));
  return XCORR_OK;
}

xcorr_status xcorr_batch_destroy(xcorr_batch b) {
  if (!b) return XCORR_OK;
  cudaSetDevice(b->device);
  cudaError_t e = cudaDeviceSynchronize();
  batch_release(b);
  delete b;
  if (e != cudaSuccess) return bfail(XCORR_ERR_CUDA, std::string("cudaDeviceSynchronize: ") + cudaGetErrorString(e));
  return XCORR_OK;
}

}  // extern "C"
