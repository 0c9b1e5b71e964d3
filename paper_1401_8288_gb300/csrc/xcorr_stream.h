// xcorr_stream.h -- packet geometry and host-side packet tracking of the
// streaming X-stage (internal).
//
// The paper's receive path (Sec. 2.3, Sec. 2.4, Fig. 3, Fig. 4): F-engine
// packets carry a 64-bit sequence number and an F-engine id that together fix
// where the payload belongs, whatever the arrival order; ring buffers of four
// sub-blocks hold the data; when packets of the next buffer pile up past a
// threshold while the current one is incomplete, its missing packets are
// recorded lost and it is marked full.  PacketTracker is that bookkeeping on
// the host: it turns headers into placement codes and block open / close
// events.  The payload bytes never pass through it.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "xcorr.h"

namespace xc {

struct StreamGeometry {
  int nt = 0, nch = 0, na = 0;           // samples, channels, inputs per packet
  int n_inputs = 0, n_channels = 0;
  int block_samples = 0, n_blocks = 0;
  int n_groups = 0;                      // channel groups (packets per F-engine per time block)
  int n_feng = 0;                        // F-engines (input groups)
  int tblocks_per_block = 0;             // packet time blocks per ring block
  int64_t packets_per_block = 0;
  int64_t payload_bytes = 0, packet_bytes = 0;
  int64_t block_bytes = 0;               // block_samples * n_channels * n_inputs

  // Checks the packet and ring fields of cfg against the plan's sizes.
  bool init(const xcorr_stream_config& cfg, int n_inputs, int n_channels, std::string* err);
};

constexpr int kSlotShift = 40;  // placement code = (slot << 40) | packet index in the block

class PacketTracker {
 public:
  PacketTracker(const StreamGeometry& g, int64_t stack_threshold);

  // Tracks packets [0, n) (header of packet k at packets + k * stride) and
  // returns how many were consumed: fewer than n only when the event buffer
  // filled up.  codes[k] receives the placement code or -1 (dropped).
  int64_t feed(const uint8_t* packets, int64_t stride, int64_t n, int64_t* codes, xcorr_block_event* ev,
               int max_ev, int* n_ev);
  // Closes every block up to the newest one that received a packet; returns
  // the number of events written (call again while it returns max_ev).
  int finish(xcorr_block_event* ev, int max_ev);

  const xcorr_packet_counters& counters() const { return counters_; }

 private:
  int64_t received(int64_t block) const;
  bool want_close() const;
  void close_oldest(int64_t position, xcorr_block_event* ev, int* n_ev);
  bool drain_closes(int64_t position, xcorr_block_event* ev, int max_ev, int* n_ev);

  StreamGeometry g_;
  int64_t threshold_;
  int64_t oldest_ = -1;  // oldest open block (-1 before the first packet)
  int64_t newest_ = -1;  // newest block that received a packet
  int64_t stack_ = 0;    // packets placed in blocks after the oldest
  std::vector<int64_t> slot_block_;  // block held by each ring slot, -1 none
  std::vector<int64_t> slot_recv_;
  std::vector<std::vector<uint64_t>> slot_bits_;
  xcorr_packet_counters counters_{};
};

}  // namespace xc
