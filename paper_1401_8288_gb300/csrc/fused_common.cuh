// fused_common.cuh -- pieces shared by the two fused 4-bit X kernels
// (xcorr_tc_fused.cu: both operands decoded into shared memory;
// xcorr_tc_fused_ta.cu: the A operand decoded into tensor memory).
//
// Both read the caller's raw [t][c][i] CI4 bytes through TMA, 128 inputs x KT
// samples per tile with the 128-byte swizzle, walk the lower-triangle tile
// pairs (c, I >= J) of every channel, and turn each 4-bit two's-complement code
// t into the offset-binary E4M3 code u = t + 8 (Sec. 2.3's 4+4-bit samples; the
// correction back to true products is in the kernels' epilogues).
#pragma once
#include <cstdint>

namespace xc {
namespace fused {

constexpr int kBlk = 128;                        // inputs per tile
constexpr uint32_t kNibbleTop = 0x88888888u;     // t -> t + 8 on every nibble
constexpr uint32_t kLowNibbles = 0x0F0F0F0Fu;
constexpr int kPrefetchSamples = 128;            // L2 prefetch distance along time (one 128-sample stage)

// Tile pair p of the packed lower triangle of tiles: p = I (I + 1) / 2 + J.
__device__ __forceinline__ void tile_pair(int p, int& I, int& J) {
  int i = static_cast<int>((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  I = i;
  J = p - i * (i + 1) / 2;
}

// L2 prefetch of one TMA box (no shared memory, nothing to wait for).
__device__ __forceinline__ void tma_prefetch_3d(const void* tmap, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                   reinterpret_cast<uint64_t>(tmap)),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}

// A tile pair of the CTA's item list (items run channel-major over the tile pairs).
struct Item {
  int c, I, J;
  bool diag, valid;
};

__device__ __forceinline__ Item item_at(int n_tile_pairs, int item, int n_items) {
  Item it{};
  it.valid = item < n_items;
  if (it.valid) {
    it.c = item / n_tile_pairs;
    tile_pair(item - it.c * n_tile_pairs, it.I, it.J);
    it.diag = it.I == it.J;
  }
  return it;
}

// L2 prefetch of stage s (KT samples from t0 + s KT) of an item: one box per tile.
template <int KT>
__device__ __forceinline__ void prefetch_stage(const void* raw_map, int t0, int n_kt, const Item& it, int s) {
  if (!it.valid || s >= n_kt) return;
  const int t = t0 + s * KT;
  tma_prefetch_3d(raw_map, it.I * kBlk, it.c, t);
  if (!it.diag) tma_prefetch_3d(raw_map, it.J * kBlk, it.c, t);
}

// The decoder warps' own barrier (id 1), and its OR-reduction form.
__device__ __forceinline__ void dec_bar_sync(uint32_t n_threads) {
  asm volatile("bar.sync 1, %0;" ::"r"(n_threads) : "memory");
}
__device__ __forceinline__ bool dec_bar_or(bool v, uint32_t n_threads) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.or.pred p, 1, %2, q;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(v)), "r"(n_threads)
      : "memory");
  return r != 0;
}

// a += b as an integer multiply-add by `one` (== 1 at run time).  The decoders'
// byte-lane sums then issue on the FMA pipe instead of the ALU pipe, which the
// decode itself keeps busy.
__device__ __forceinline__ void lane_add(uint32_t& a, uint32_t b, uint32_t one) {
  asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(a) : "r"(b), "r"(one));
}

// Four CI4 bytes -> four offset E4M3 real codes and four imaginary codes.
__device__ __forceinline__ void offset_codes(uint32_t w, uint32_t& re, uint32_t& im) {
  const uint32_t u = w ^ kNibbleTop;
  im = u & kLowNibbles;
  re = (u >> 4) & kLowNibbles;
}

}  // namespace fused
}  // namespace xc
