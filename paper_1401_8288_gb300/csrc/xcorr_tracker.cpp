// xcorr_tracker.cpp -- host-side packet tracking and the packetizer of the
// streaming X-stage (no GPU code).
//
// Placement (Sec. 2.3, Fig. 3): a packet's sequence number and F-engine id
// fix its place in memory regardless of arrival order.  Buffer completion
// (Sec. 2.4): packets belonging to later buffers are held while the current
// one is incomplete; when the held count reaches a threshold, the missing
// packets of the current buffer are recorded lost and it is marked full.
// Readings of this library: the held packets live in their own ring blocks
// (so nothing is copied twice), a packet for a block past the ring also closes
// the oldest block, a complete oldest block closes at once, and blocks close
// strictly in order.
#include <algorithm>
#include <cstring>
#include <new>

#include "xcorr_internal.h"
#include "xcorr_stream.h"

namespace xc {

namespace {

uint64_t load_le64(const uint8_t* p) {
  uint64_t v = 0;
  for (int k = 7; k >= 0; --k) v = (v << 8) | p[k];
  return v;
}

uint32_t load_le32(const uint8_t* p) {
  return static_cast<uint32_t>(p[0]) | (static_cast<uint32_t>(p[1]) << 8) | (static_cast<uint32_t>(p[2]) << 16) |
         (static_cast<uint32_t>(p[3]) << 24);
}

void store_le64(uint8_t* p, uint64_t v) {
  for (int k = 0; k < 8; ++k) p[k] = static_cast<uint8_t>(v >> (8 * k));
}

void store_le32(uint8_t* p, uint32_t v) {
  for (int k = 0; k < 4; ++k) p[k] = static_cast<uint8_t>(v >> (8 * k));
}

// A packet for a block this far past the oldest open one is taken as corrupt
// rather than closing that many empty blocks.
constexpr int64_t kMaxBlockJump = INT64_C(1) << 20;

}  // namespace

bool StreamGeometry::init(const xcorr_stream_config& c, int n_in, int n_chan, std::string* err) {
  auto bad = [&](const char* m) {
    if (err) *err = m;
    return false;
  };
  if (c.n_time_per_packet < 1 || c.n_chan_per_packet < 1 || c.n_inputs_per_packet < 1)
    return bad("packet sizes must be positive");
  if (n_chan % c.n_chan_per_packet) return bad("n_chan_per_packet must divide n_channels");
  if (c.n_inputs_per_packet % 16 || n_in % c.n_inputs_per_packet)
    return bad("n_inputs_per_packet must be a multiple of 16 that divides n_inputs");
  if (c.block_samples < 1 || c.block_samples % c.n_time_per_packet)
    return bad("block_samples must be a positive multiple of n_time_per_packet");
  if (c.n_blocks < 2 || c.n_blocks > 4096) return bad("n_blocks must be in [2, 4096]");
  if (c.blocks_per_dump < 1) return bad("blocks_per_dump must be >= 1");
  if (c.stack_threshold < 1) return bad("stack_threshold must be >= 1");
  if (c.chunk_packets < 1 || c.n_chunks < 2 || c.n_host_dumps < 1)
    return bad("chunk_packets >= 1, n_chunks >= 2 and n_host_dumps >= 1 are required");
  nt = c.n_time_per_packet;
  nch = c.n_chan_per_packet;
  na = c.n_inputs_per_packet;
  n_inputs = n_in;
  n_channels = n_chan;
  block_samples = c.block_samples;
  n_blocks = c.n_blocks;
  n_groups = n_chan / nch;
  n_feng = n_in / na;
  tblocks_per_block = block_samples / nt;
  packets_per_block = static_cast<int64_t>(tblocks_per_block) * n_groups * n_feng;
  if (packets_per_block >= (INT64_C(1) << kSlotShift)) return bad("too many packets per block");
  payload_bytes = static_cast<int64_t>(nt) * nch * na;
  packet_bytes = XCORR_PACKET_HEADER_BYTES + payload_bytes;
  block_bytes = static_cast<int64_t>(block_samples) * n_chan * n_in;
  return true;
}

PacketTracker::PacketTracker(const StreamGeometry& g, int64_t stack_threshold)
    : g_(g),
      threshold_(stack_threshold),
      slot_block_(g.n_blocks, -1),
      slot_recv_(g.n_blocks, 0),
      slot_bits_(g.n_blocks, std::vector<uint64_t>((g.packets_per_block + 63) / 64, 0)) {}

int64_t PacketTracker::received(int64_t block) const {
  const int s = static_cast<int>(block % g_.n_blocks);
  return slot_block_[s] == block ? slot_recv_[s] : 0;
}

bool PacketTracker::want_close() const {
  if (oldest_ < 0 || oldest_ > newest_) return false;
  return received(oldest_) == g_.packets_per_block || stack_ >= threshold_;
}

void PacketTracker::close_oldest(int64_t position, xcorr_block_event* ev, int* n_ev) {
  const int s = static_cast<int>(oldest_ % g_.n_blocks);
  const int64_t recv = received(oldest_);
  xcorr_block_event& e = ev[(*n_ev)++];
  e.kind = XCORR_EVENT_CLOSE;
  e.slot = s;
  e.block = oldest_;
  e.position = position;
  e.received = recv;
  e.lost = g_.packets_per_block - recv;
  counters_.lost += e.lost;
  counters_.blocks_closed += 1;
  if (slot_block_[s] == oldest_) slot_block_[s] = -1;  // free for block oldest + n_blocks
  ++oldest_;
  stack_ -= received(oldest_);  // the new oldest block's packets are no longer held for later
}

bool PacketTracker::drain_closes(int64_t position, xcorr_block_event* ev, int max_ev, int* n_ev) {
  while (want_close()) {
    if (*n_ev >= max_ev) return false;
    close_oldest(position, ev, n_ev);
  }
  return true;
}

int64_t PacketTracker::feed(const uint8_t* packets, int64_t stride, int64_t n, int64_t* codes,
                            xcorr_block_event* ev, int max_ev, int* n_ev) {
  *n_ev = 0;
  for (int64_t k = 0; k < n; ++k) {
    if (!drain_closes(k, ev, max_ev, n_ev)) return k;
    const uint8_t* h = packets + k * stride;
    const uint64_t seq = load_le64(h);
    const uint32_t fid = load_le32(h + 8);
    const int64_t tblock = static_cast<int64_t>(seq / static_cast<uint64_t>(g_.n_groups));
    const int grp = static_cast<int>(seq % static_cast<uint64_t>(g_.n_groups));
    const int64_t b = tblock / g_.tblocks_per_block;
    const int tl = static_cast<int>(tblock % g_.tblocks_per_block);
    const bool corrupt = fid >= static_cast<uint32_t>(g_.n_feng) || seq > (UINT64_C(1) << 62) ||
                         (oldest_ >= 0 && b - oldest_ > kMaxBlockJump);
    if (corrupt || (oldest_ >= 0 && b < oldest_)) {
      // counted only once the packet is consumed (it may be retried after a full event buffer)
      if (corrupt)
        counters_.bad += 1;
      else
        counters_.late += 1;
      counters_.packets += 1;
      codes[k] = -1;
      continue;
    }
    // events this packet needs: closes to make room in the ring, then an open;
    // when the event buffer fills first, the packet is retried by the next call
    if (oldest_ < 0) oldest_ = b;
    while (b >= oldest_ + g_.n_blocks) {
      if (*n_ev >= max_ev) return k;
      close_oldest(k, ev, n_ev);
    }
    const int s = static_cast<int>(b % g_.n_blocks);
    if (slot_block_[s] != b && *n_ev >= max_ev) return k;
    if (slot_block_[s] != b) {
      slot_block_[s] = b;
      slot_recv_[s] = 0;
      std::fill(slot_bits_[s].begin(), slot_bits_[s].end(), 0);
      xcorr_block_event& e = ev[(*n_ev)++];
      e.kind = XCORR_EVENT_OPEN;
      e.slot = s;
      e.block = b;
      e.position = k;
      e.received = 0;
      e.lost = 0;
    }
    counters_.packets += 1;
    const int64_t pidx = (static_cast<int64_t>(tl) * g_.n_groups + grp) * g_.n_feng + fid;
    uint64_t& word = slot_bits_[s][pidx >> 6];
    const uint64_t bit = UINT64_C(1) << (pidx & 63);
    if (word & bit) {
      counters_.duplicates += 1;
      codes[k] = -1;
      continue;
    }
    word |= bit;
    slot_recv_[s] += 1;
    counters_.placed += 1;
    if (b > oldest_) stack_ += 1;
    if (b > newest_) newest_ = b;
    codes[k] = (static_cast<int64_t>(s) << kSlotShift) | pidx;
  }
  drain_closes(n, ev, max_ev, n_ev);  // what does not fit is emitted at the start of the next call
  return n;
}

int PacketTracker::finish(xcorr_block_event* ev, int max_ev) {
  int n_ev = 0;
  while (oldest_ >= 0 && oldest_ <= newest_ && n_ev < max_ev) close_oldest(0, ev, &n_ev);
  return n_ev;
}

}  // namespace xc

// ------------------------------------------------------------------- C ABI --
struct xcorr_tracker_s {
  xc::StreamGeometry g;
  xc::PacketTracker* t = nullptr;
};

extern "C" {

xcorr_status xcorr_tracker_create(xcorr_tracker* out, const xcorr_stream_config* cfg, int n_inputs, int n_channels) {
  if (!out || !cfg) return xc::set_error(XCORR_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (n_inputs < 1 || n_channels < 1) return xc::set_error(XCORR_ERR_INVALID_ARG, "sizes must be positive");
  auto* tr = new (std::nothrow) xcorr_tracker_s;
  if (!tr) return xc::set_error(XCORR_ERR_OOM, "tracker");
  std::string err;
  if (!tr->g.init(*cfg, n_inputs, n_channels, &err)) {
    delete tr;
    return xc::set_error(XCORR_ERR_INVALID_ARG, err);
  }
  tr->t = new (std::nothrow) xc::PacketTracker(tr->g, cfg->stack_threshold);
  if (!tr->t) {
    delete tr;
    return xc::set_error(XCORR_ERR_OOM, "tracker");
  }
  *out = tr;
  return XCORR_OK;
}

xcorr_status xcorr_tracker_feed(xcorr_tracker tr, const void* packets, int64_t stride, int64_t n, int64_t* codes,
                                xcorr_block_event* events, int max_events, int* n_events, int64_t* n_done) {
  if (!tr || (n > 0 && (!packets || !codes)) || !events || !n_events || !n_done || n < 0 || max_events < 1 ||
      stride < XCORR_PACKET_HEADER_BYTES)
    return xc::set_error(XCORR_ERR_INVALID_ARG, "invalid tracker_feed arguments");
  *n_done = tr->t->feed(static_cast<const uint8_t*>(packets), stride, n, codes, events, max_events, n_events);
  return XCORR_OK;
}

xcorr_status xcorr_tracker_finish(xcorr_tracker tr, xcorr_block_event* events, int max_events, int* n_events) {
  if (!tr || !events || !n_events || max_events < 1)
    return xc::set_error(XCORR_ERR_INVALID_ARG, "invalid tracker_finish arguments");
  *n_events = tr->t->finish(events, max_events);
  return XCORR_OK;
}

xcorr_status xcorr_tracker_counters(xcorr_tracker tr, xcorr_packet_counters* out) {
  if (!tr || !out) return xc::set_error(XCORR_ERR_INVALID_ARG, "null argument");
  *out = tr->t->counters();
  return XCORR_OK;
}

xcorr_status xcorr_tracker_destroy(xcorr_tracker tr) {
  if (tr) {
    delete tr->t;
    delete tr;
  }
  return XCORR_OK;
}

xcorr_status xcorr_packetize(const void* samples, int n_time, int n_channels, int n_inputs,
                             const xcorr_stream_config* cfg, int64_t first_time_block, void* packets,
                             int64_t capacity_packets, int64_t* n_packets) {
  if (!samples || !cfg || !packets || !n_packets || first_time_block < 0)
    return xc::set_error(XCORR_ERR_INVALID_ARG, "invalid packetize arguments");
  xc::StreamGeometry g;
  std::string err;
  if (!g.init(*cfg, n_inputs, n_channels, &err)) return xc::set_error(XCORR_ERR_INVALID_ARG, err);
  if (n_time < 0 || n_time % g.nt) return xc::set_error(XCORR_ERR_INVALID_ARG, "n_time must be a multiple of N_t");
  const int64_t n_tb = n_time / g.nt;
  const int64_t total = n_tb * g.n_groups * g.n_feng;
  if (total > capacity_packets) return xc::set_error(XCORR_ERR_INVALID_ARG, "packet buffer too small");
  const uint8_t* x = static_cast<const uint8_t*>(samples);
  uint8_t* out = static_cast<uint8_t*>(packets);
  const int64_t row = static_cast<int64_t>(n_channels) * n_inputs;  // bytes per time sample
  for (int64_t tb = 0; tb < n_tb; ++tb)
    for (int grp = 0; grp < g.n_groups; ++grp)
      for (int f = 0; f < g.n_feng; ++f) {
        std::memset(out, 0, XCORR_PACKET_HEADER_BYTES);
        xc::store_le64(out, static_cast<uint64_t>(first_time_block + tb) * g.n_groups + grp);
        xc::store_le32(out + 8, static_cast<uint32_t>(f));
        uint8_t* pay = out + XCORR_PACKET_HEADER_BYTES;
        for (int tt = 0; tt < g.nt; ++tt)
          for (int cc = 0; cc < g.nch; ++cc) {
            const uint8_t* src = x + (tb * g.nt + tt) * row + static_cast<int64_t>(grp * g.nch + cc) * n_inputs +
                                 static_cast<int64_t>(f) * g.na;
            std::memcpy(pay, src, g.na);
            pay += g.na;
          }
        out += g.packet_bytes;
      }
  *n_packets = total;
  return XCORR_OK;
}

xcorr_status xcorr_packets_advance(void* packets, int64_t stride, int64_t n, int64_t seq_delta) {
  if ((n > 0 && !packets) || n < 0 || stride < XCORR_PACKET_HEADER_BYTES)
    return xc::set_error(XCORR_ERR_INVALID_ARG, "invalid packets_advance arguments");
  uint8_t* p = static_cast<uint8_t*>(packets);
  for (int64_t k = 0; k < n; ++k, p += stride) xc::store_le64(p, xc::load_le64(p) + static_cast<uint64_t>(seq_delta));
  return XCORR_OK;
}

}  // extern "C"
