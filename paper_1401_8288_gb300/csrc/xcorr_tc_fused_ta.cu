// xcorr_tc_fused_ta.cu -- the fused 4-bit X-stage with the A operand decoded
// straight into tensor memory.
//
// Same result as xcorr_tc_fused.cu (per channel, the packed lower triangle of
// V = sum_t x_t x_t^H; Sec. 1, Sec. 2.1, Eq. 1) from the same raw [t][c][i]
// CI4 bytes and the same offset-binary E4M3 operands u = t + 8, but the row
// tile's operand never goes through shared memory.  In the shared-memory
// kernel every MMA re-reads A from shared memory, and the operand reads, the
// decoders' stores and the TMA writes together exhaust the SM's shared-memory
// bandwidth well before the tensor pipe; here A lives in tensor memory:
//
//   * an ldmatrix.trans of a 16-sample x 16-input block of raw bytes gives
//     each thread four consecutive samples of one input, which is exactly the
//     register layout a tcgen05.st of 16 lanes x 128 bits takes (lane = input,
//     column = four samples); after the XOR-and-mask decode the registers go
//     to tensor memory unchanged, one store for the real codes and one for the
//     imaginary codes (the .x2 forms of both move two such blocks at once);
//   * the column tile's real and imaginary planes are decoded into shared
//     memory as before (MN-major, 128-byte swizzle) and are the MMAs' B;
//   * per 32-sample step the MMAs are Re|-Im += A_re [B_re | B_im],
//     Re += A_im B_im, -Im += -A_im B_re, A read from tensor memory.
//
// Tensor memory holds the accumulator [Re | -Im] in columns 0-255, a stash
// for Im in columns 256-383 and DEC A stages (real then imaginary codes,
// KT / 2 columns) from column 384, so the accumulator is single-buffered.  The
// epilogue therefore frees it in one quick pass that only moves bits: Re to a
// shared-memory tile of the whole tile pair, Im to the stash.  While the MMAs
// already run the next tile pair it converts (one FFMA against 1.5 2^23 while
// the block's sums stay below 2^22), applies the offset corrections and
// writes the rows to HBM; the decoders keep filling the rings meanwhile.
//
// The per-input sums S = sum_t u that undo the offset (see xcorr_tc_fused.cu)
// come from the A path for the rows (dp4a over the codes each thread holds)
// and from the B path for the columns (byte lanes, as in the other kernel).
//
// Warp roles (448 threads, one CTA per SM): warps 0-3 drain the accumulator
// and write the output; warps 4-11 decode (warp w writes the A lanes of TMEM
// quarter w % 4, 16 inputs, and a share of B); warp 12 is the TMA producer
// with the L2 prefetch; warp 13 owns tensor memory and issues the MMAs.
// Every wait is bounded (sm103_ptx.cuh).
//
// A batch mode (xcorr_batch.cu) runs the same pipeline over the tile pairs of
// several problems, each item naming its problem's descriptor.
#include "fused_common.cuh"
#include "sm103_ptx.cuh"
#include "xcorr_internal.h"

namespace xc {
namespace {

using namespace fused;

constexpr int kEpiWarps = 4;
constexpr int kDecWarp0 = 4;
constexpr int kDecWarps = 8;  // two per tensor-memory lane quarter
constexpr int kProducerWarp = kDecWarp0 + kDecWarps;
constexpr int kMmaWarp = kProducerWarp + 1;
constexpr int kThreads = (kMmaWarp + 1) * 32;
constexpr int kDecThreads = kDecWarps * 32;
constexpr int kChunk = 16;
constexpr int kPitch = kChunk + 1;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kStashCol = 256;                       // 128 columns of corrected Im after the accumulator
constexpr uint32_t kAcol0 = 384;                          // then the A stages
constexpr int kStagingBytes = kBlk * kBlk * 4;            // Re accumulator bits of a whole tile pair
constexpr int kRowcBytes = kBlk * 8;                      // per-row correction constants
constexpr int kSumsBytes = 2 * 2 * kBlk * 8;              // [item parity][rows I, columns J][input] (8P, 8Q)
// Every partial sum of u_a u_b is n 2^-18 with 0 <= n <= 450 T (and |n| <= 225 T for Im).
// For T <= kMagicSamples, |n| < 2^22 and n + 1.5 2^23 is exact in FP32, so one FFMA
// against that constant turns the accumulator into n (in the low bits of the result).
constexpr int kMagicSamples = 9320;
constexpr float kMagic = 12582912.0f;       // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;
constexpr int kScratchBytes = kDecWarps * 8 * kPitch * 8; // [decoder warp][chunk][input] (P, Q), padded rows
constexpr int kBarrierBytes = 512;

template <int KT, int RAW, int DEC>
struct TGeom {
  static constexpr int kTile = KT * kBlk;      // one 128-input x KT-sample tile of bytes
  static constexpr int kRawStage = 2 * kTile;  // raw I, raw J
  static constexpr int kBStage = 2 * kTile;    // B real codes, B imaginary codes
  static constexpr int kAcols = KT / 2;        // one A stage: KT / 4 columns of real codes, then imaginary
  static constexpr int kRowsB = KT / (kDecThreads / 8);  // B rows per decoder thread and stage
  static constexpr int kSteps = KT / 32;                 // MMA steps (32 samples) per stage
  // byte offsets of the buffers from the 1024-aligned start of shared memory; the kernel takes
  // its pointers from these, and the allocation is their end (plus the alignment slack)
  static constexpr int kOffBpl = RAW * kRawStage;
  static constexpr int kOffStaging = kOffBpl + DEC * kBStage;
  static constexpr int kOffRowc = kOffStaging + kStagingBytes;
  static constexpr int kOffSums = kOffRowc + kRowcBytes;
  static constexpr int kOffScratch = kOffSums + kSumsBytes;
  static constexpr int kOffBarriers = kOffScratch + kScratchBytes;
  static constexpr int kSmem = 1024 + kOffBarriers + kBarrierBytes;
  static_assert(KT % 32 == 0, "stages hold whole MMA steps and whole 32-row B passes");
  static_assert(DEC * kAcols <= static_cast<int>(kTmemCols - kAcol0), "A stages fit beside the accumulator");
  static_assert((2 * RAW + 2 * DEC + 7) * 8 + 8 <= kBarrierBytes, "barrier area");
  static_assert(kSmem <= 232448, "shared memory budget");
};

struct TParams {
  int n_chan, n_inputs, n_tile_pairs;
  int t0;              // first sample of this launch
  int n_kt;            // stages per tile pair
  int64_t n_pairs;
  int accumulate;      // add into out (else store)
  // small-problem layout: pack_g channels of n_inputs each side by side in one tile (PACK), and
  // each tile's stages cut into n_split items of split_kt stages whose results are added with
  // atomics (atomic_out)
  int pack_g, n_split, split_kt, atomic_out;
  int n_items;         // items of a non-batch launch: tiles x n_split
  int2* out;
  int* status;
  uint32_t one;        // 1: a multiplier the compiler cannot fold (see lane_add)
  // batch mode: items (subarray, channel, I, J) and one descriptor per subarray
  const TaSubDesc* subs;
  const uint4* items;
  int n_batch_items;
};

// Everything a role needs of one item: its tile pair and its subarray (the launch's own problem,
// or in batch mode the item's subarray descriptor).
struct TItem {
  const CUtensorMap* map;  // raw input
  int2* out;
  int64_t n_pairs;
  int c, I, J, n_inputs, n_kt, accumulate;
  int t_first;             // first sample of the item
  int ax, ay, bx, by;      // TMA coordinates (input or channel-input column, channel) of the row and column tiles
  bool diag, valid;
};

template <bool BATCH, bool SMALL, bool PACK, int KT>
__device__ __forceinline__ TItem resolve(const TParams& p, const CUtensorMap* map, int item, int n_items) {
  TItem it{};
  it.valid = item < n_items;
  if (!it.valid) return it;
  if (BATCH) {
    const uint4 w = p.items[item];
    const TaSubDesc* s = p.subs + w.x;
    it.map = &s->tmap;
    it.out = s->out;
    it.n_pairs = s->n_pairs;
    it.n_inputs = s->n_inputs;
    it.n_kt = s->n_kt;
    it.accumulate = s->accumulate;
    it.c = static_cast<int>(w.y);
    it.I = static_cast<int>(w.z);
    it.J = static_cast<int>(w.w);
    it.t_first = 0;
  } else {
    it.map = map;
    it.out = p.out;
    it.n_pairs = p.n_pairs;
    it.n_inputs = p.n_inputs;
    it.accumulate = p.accumulate;
    int tile = item;
    it.n_kt = p.n_kt;
    it.t_first = p.t0;
    if (SMALL) {  // the time split of the small-problem layout
      tile = item / p.n_split;
      const int split = item - tile * p.n_split;
      it.n_kt = min(p.split_kt, p.n_kt - split * p.split_kt);
      it.t_first = p.t0 + split * p.split_kt * KT;
    }
    if (PACK) {  // tile = a group of pack_g channels, one diagonal tile pair
      it.c = tile;
      it.I = it.J = 0;
    } else {
      it.c = tile / p.n_tile_pairs;
      tile_pair(tile - it.c * p.n_tile_pairs, it.I, it.J);
    }
  }
  it.diag = it.I == it.J;
  if (PACK) {  // the packed view: x = channel * n_inputs + input over one time row
    it.ax = it.bx = it.c * p.pack_g * p.n_inputs;
    it.ay = it.by = 0;
  } else {
    it.ax = it.I * kBlk;
    it.bx = it.J * kBlk;
    it.ay = it.by = it.c;
  }
  return it;
}

// L2 prefetch of stage s (KT samples from the item's first sample + s KT): one box per tile.
template <int KT>
__device__ __forceinline__ void prefetch_item_stage(const TItem& it, int s) {
  if (!it.valid || s >= it.n_kt) return;
  const int t = it.t_first + s * KT;
  tma_prefetch_3d(it.map, it.ax, it.ay, t);
  if (!it.diag) tma_prefetch_3d(it.map, it.bx, it.by, t);
}

// 16-byte chunk swizzle of the Re staging tile: a bijection of row % 8, so the eight rows of a
// phase-1 quarter-warp store hit eight distinct chunks, and rows 2k, 2k + 1 (the two half-warps
// of a phase-2 load) land in opposite halves of each eight-chunk group.
__device__ __forceinline__ int staging_swizzle(int row) { return ((row & 1) << 2) | ((row >> 1) & 3); }

template <int KT, int RAW, int DEC, bool BATCH, bool SMALL, bool PACK>
__global__ void __launch_bounds__(kThreads, 1)
    xcorr_tc_fused_ta_kernel(const __grid_constant__ CUtensorMap raw_map, const __grid_constant__ TParams p) {
  using G = TGeom<KT, RAW, DEC>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* raw = smem;
  uint8_t* bpl = smem + G::kOffBpl;
  uint32_t* staging = reinterpret_cast<uint32_t*>(smem + G::kOffStaging);  // Re [row][16-byte chunk ^ swz(row)]
  int2* rowc = reinterpret_cast<int2*>(smem + G::kOffRowc);                 // [row]
  int2* sums = reinterpret_cast<int2*>(smem + G::kOffSums);
  int2* scratch = reinterpret_cast<int2*>(smem + G::kOffScratch);
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem + G::kOffBarriers);
  uint64_t* raw_empty = raw_full + RAW;
  uint64_t* dec_full = raw_empty + RAW;
  uint64_t* dec_empty = dec_full + DEC;
  uint64_t* tfull = dec_empty + DEC;  // the accumulator holds an item
  uint64_t* tempty = tfull + 1;       // the epilogue has the item in registers
  uint64_t* sfull = tempty + 1;       // [2] an item's input sums are written
  uint64_t* sempty = sfull + 2;       // [2] the epilogue is done with them
  uint64_t* mma_done = sempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < RAW; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], kDecWarps);
    }
    for (int s = 0; s < DEC; ++s) {
      mbar_init(&dec_full[s], kDecWarps);
      mbar_init(&dec_empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, kEpiWarps);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sfull[b], 1);
      mbar_init(&sempty[b], kEpiWarps);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) tmem_alloc(tslot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int n_items = BATCH ? p.n_batch_items : p.n_items;

  if (warp == kProducerWarp) {
    if (lane == 0) {
      constexpr int kAhead = kPrefetchSamples / KT;  // L2 prefetch runs this many stages ahead of the loads
      if (!BATCH) prefetch_tmap(&raw_map);
      TItem next = resolve<BATCH, SMALL, PACK, KT>(p, &raw_map, blockIdx.x, n_items);
      if (BATCH && next.valid) prefetch_tmap(next.map);
      for (int s = 0; s < kAhead; ++s) prefetch_item_stage<KT>(next, s);
      int r = 0;
      uint32_t ph = 0, filled = 0, fill_parity[RAW] = {};
      bool ok = true;
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
        const TItem it = next;
        next = resolve<BATCH, SMALL, PACK, KT>(p, &raw_map, item + gridDim.x, n_items);
        if (BATCH && next.valid) prefetch_tmap(next.map);
        for (int tb = 0; tb < it.n_kt; ++tb) {
          if (tb + kAhead < it.n_kt)
            prefetch_item_stage<KT>(it, tb + kAhead);
          else
            prefetch_item_stage<KT>(next, tb + kAhead - it.n_kt);
          if (!mbar_wait(&raw_empty[r], ph ^ 1u, abort_flag, p.status, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          uint8_t* st = raw + r * G::kRawStage;
          const int t = it.t_first + tb * KT;
          mbar_expect_tx(&raw_full[r], (it.diag ? 1 : 2) * G::kTile);
          tma_load_3d(st, it.map, &raw_full[r], it.ax, it.ay, t);
          if (!it.diag) tma_load_3d(st + G::kTile, it.map, &raw_full[r], it.bx, it.by, t);
          fill_parity[r] = ph;
          filled |= 1u << r;
          if (++r == RAW) {
            r = 0;
            ph ^= 1u;
          }
        }
      }
      // Let every copy this CTA issued land before the CTA can exit.
      volatile int never = 0;
      for (int q = 0; q < RAW; ++q)
        if (filled & (1u << q)) mbar_wait(&raw_full[q], fill_parity[q], &never, p.status, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp >= kDecWarp0 && warp < kDecWarp0 + kDecWarps) {
    const int dw = warp - kDecWarp0, tid = dw * 32 + lane;
    // A: this warp's 16 inputs are TMEM lanes 16 ib .. 16 ib + 15, inside its lane quarter warp % 4
    const int ib = 2 * (warp & 3) + (dw >> 2);
    const uint32_t a_lanes = static_cast<uint32_t>(16 * ib) << 16;
    const int apos = (ib ^ (lane & 7)) << 4;     // chunk ib of row 16 sb + lane under the 128-byte swizzle
    // B: a fixed 16-input chunk L of the column tile, rows phase, phase + 32, ...
    const int L = tid & 7, phase = tid >> 3;
    const int bpos = (L ^ (phase & 7)) << 4;
    int r = 0, d = 0, g = 0;
    uint32_t rph = 0, dph = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++g) {
      const TItem cur = resolve<BATCH, SMALL, PACK, KT>(p, &raw_map, item, n_items);
      // A sums: inputs 16 ib + lane / 4 (0) and + 8 (1), over samples 4 (lane % 4) .. + 3 of every 16
      uint32_t sar0 = 0u, sai0 = 0u, sar1 = 0u, sai1 = 0u;
      // B sums in 16-bit lanes: word e / 2, half e % 2 holds input e of chunk L
      uint32_t s_re[8], s_im[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) s_re[q] = s_im[q] = 0u;
      bool ok = true;
      for (int tb = 0; tb < cur.n_kt; ++tb) {
        if (!mbar_wait_warp(&raw_full[r], rph, abort_flag, p.status, DEV_TIMEOUT_FULL) ||
            !mbar_wait_warp(&dec_empty[d], dph ^ 1u, abort_flag, p.status, DEV_TIMEOUT_EMPTY)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint8_t* raw_a = raw + r * G::kRawStage;
        const uint8_t* raw_b = raw_a + (cur.diag ? 0 : G::kTile);
        // A operand: two blocks of 16 samples x 16 inputs per ldmatrix (thread t addresses row
        // 16 sb + t, both blocks under the same swizzle since 16 sb = 0 mod 8), decoded in
        // registers, stored to TMEM eight columns at a time
        const uint32_t ta = tmem + a_lanes + kAcol0 + static_cast<uint32_t>(d * G::kAcols);
        static_assert(KT % 32 == 0, "whole pairs of 16-sample blocks");
        // four blocks per pair of stores (sixteen columns), then a pair of blocks if KT / 16 is
        // not a multiple of four
#pragma unroll
        for (int sb = 0; sb < KT / 16; sb += 4) {
          const int nb = KT / 16 - sb >= 4 ? 2 : 1;  // ldmatrix pairs of blocks in this group
          uint32_t re[8], im[8];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (h >= nb) break;
            uint32_t x0, x1, x2, x3;
            ldmatrix_t_b8_x2(smem_u32(raw_a + (16 * (sb + 2 * h) + lane) * 128 + apos), x0, x1, x2, x3);
            offset_codes(x0, re[4 * h], im[4 * h]);
            offset_codes(x1, re[4 * h + 1], im[4 * h + 1]);
            offset_codes(x2, re[4 * h + 2], im[4 * h + 2]);
            offset_codes(x3, re[4 * h + 3], im[4 * h + 3]);
            // the two blocks' codes of one input add per byte (<= 30) before the dp4a
            sar0 = __dp4a(re[4 * h] + re[4 * h + 2], 0x01010101u, sar0);
            sai0 = __dp4a(im[4 * h] + im[4 * h + 2], 0x01010101u, sai0);
            sar1 = __dp4a(re[4 * h + 1] + re[4 * h + 3], 0x01010101u, sar1);
            sai1 = __dp4a(im[4 * h + 1] + im[4 * h + 3], 0x01010101u, sai1);
          }
          if (nb == 2) {
            tmem_st_16x128b_x4(ta + 4 * sb, re);
            tmem_st_16x128b_x4(ta + KT / 4 + 4 * sb, im);
          } else {
            tmem_st_16x128b_x2(ta + 4 * sb, re[0], re[1], re[2], re[3]);
            tmem_st_16x128b_x2(ta + KT / 4 + 4 * sb, im[0], im[1], im[2], im[3]);
          }
        }
        // B operand: real and imaginary planes in shared memory at the raw chunk's swizzled offset
        {
          constexpr int R = G::kRowsB;
          const uint8_t* src = raw_b + bpos;
          uint8_t* re_t = bpl + d * G::kBStage + bpos;
          uint8_t* im_t = re_t + G::kTile;
          uint4 v[R];
#pragma unroll
          for (int k = 0; k < R; ++k) v[k] = *reinterpret_cast<const uint4*>(src + (phase + 32 * k) * 128);
          uint32_t a_re[4] = {0u, 0u, 0u, 0u}, a_im[4] = {0u, 0u, 0u, 0u};  // byte lanes: <= 15 R <= 60
#pragma unroll
          for (int k = 0; k < R; ++k) {
            uint4 re, im;
            offset_codes(v[k].x, re.x, im.x);
            offset_codes(v[k].y, re.y, im.y);
            offset_codes(v[k].z, re.z, im.z);
            offset_codes(v[k].w, re.w, im.w);
            lane_add(a_re[0], re.x, p.one), lane_add(a_re[1], re.y, p.one);
            lane_add(a_re[2], re.z, p.one), lane_add(a_re[3], re.w, p.one);
            lane_add(a_im[0], im.x, p.one), lane_add(a_im[1], im.y, p.one);
            lane_add(a_im[2], im.z, p.one), lane_add(a_im[3], im.w, p.one);
            const int off = (phase + 32 * k) * 128;
            *reinterpret_cast<uint4*>(re_t + off) = re;
            *reinterpret_cast<uint4*>(im_t + off) = im;
          }
          // widen to 16-bit lanes: inputs (4q, 4q+1) -> word 2q, (4q+2, 4q+3) -> word 2q+1
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            lane_add(s_re[2 * q], __byte_perm(a_re[q], 0u, 0x4140), p.one);
            lane_add(s_re[2 * q + 1], __byte_perm(a_re[q], 0u, 0x4342), p.one);
            lane_add(s_im[2 * q], __byte_perm(a_im[q], 0u, 0x4140), p.one);
            lane_add(s_im[2 * q + 1], __byte_perm(a_im[q], 0u, 0x4342), p.one);
          }
        }
        // the MMA reads A through tensor memory and B through the async proxy
        tmem_st_wait();
        tc_fence_before();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&raw_empty[r]);
          mbar_arrive(&dec_full[d]);
        }
        if (++r == RAW) {
          r = 0;
          rph ^= 1u;
        }
        if (++d == DEC) {
          d = 0;
          dph ^= 1u;
        }
      }
      // row sums: the four lanes holding one input's samples are lanes 4k .. 4k + 3
#pragma unroll
      for (int m = 1; m <= 2; m <<= 1) {
        sar0 += __shfl_xor_sync(0xFFFFFFFFu, sar0, m);
        sai0 += __shfl_xor_sync(0xFFFFFFFFu, sai0, m);
        sar1 += __shfl_xor_sync(0xFFFFFFFFu, sar1, m);
        sai1 += __shfl_xor_sync(0xFFFFFFFFu, sai1, m);
      }
      // column sums of this warp: lanes L, L + 8, L + 16, L + 24 hold chunk L
      int2 pq[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int sr = static_cast<int>((s_re[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
        const int si = static_cast<int>((s_im[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
        pq[e] = make_int2(sr + si, si - sr);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        pq[e].x += __shfl_xor_sync(0xFFFFFFFFu, pq[e].x, 8);
        pq[e].y += __shfl_xor_sync(0xFFFFFFFFu, pq[e].y, 8);
        pq[e].x += __shfl_xor_sync(0xFFFFFFFFu, pq[e].x, 16);
        pq[e].y += __shfl_xor_sync(0xFFFFFFFFu, pq[e].y, 16);
      }
      if (lane < 8) {
#pragma unroll
        for (int e = 0; e < 16; ++e) scratch[(dw * 8 + lane) * kPitch + e] = pq[e];
      }
      dec_bar_sync(kDecThreads);
      const int buf = g & 1;
      if (ok) ok = mbar_wait_warp(&sempty[buf], ((g >> 1) & 1) ^ 1, abort_flag, p.status, DEV_TIMEOUT_TMEM_EMPTY);
      if (ok) {
        int2* rows = sums + (buf * 2) * kBlk;
        if ((lane & 3) == 0) {
          const int e = 16 * ib + (lane >> 2);
          rows[e] = make_int2(8 * static_cast<int>(sar0 + sai0), 8 * (static_cast<int>(sai0) - static_cast<int>(sar0)));
          rows[e + 8] =
              make_int2(8 * static_cast<int>(sar1 + sai1), 8 * (static_cast<int>(sai1) - static_cast<int>(sar1)));
        }
        if (tid < kBlk) {
          const int e = tid;
          int2 s = make_int2(0, 0);
#pragma unroll
          for (int w = 0; w < kDecWarps; ++w) {
            const int2 x = scratch[(w * 8 + (e >> 4)) * kPitch + (e & 15)];
            s.x += x.x;
            s.y += x.y;
          }
          sums[(buf * 2 + 1) * kBlk + e] = make_int2(8 * s.x, 8 * s.y);
        }
      }
      if (dec_bar_or(!ok || *abort_flag, kDecThreads)) break;
      if (tid == 0) mbar_arrive(&sfull[buf]);
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      const uint32_t id256 = instr_desc_ta(kTypeE4M3, 128, 256, false);
      const uint32_t id128 = instr_desc_ta(kTypeE4M3, 128, 128, false);
      const uint32_t id128n = instr_desc_ta(kTypeE4M3, 128, 128, true);
      constexpr uint32_t kLbo = G::kTile;  // B real and imaginary planes are adjacent 128-byte-wide chunks
      int d = 0, g = 0;
      uint32_t dph = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x, ++g) {
        if (!mbar_wait(tempty, (g & 1) ^ 1, abort_flag, p.status, DEV_TIMEOUT_TMEM_EMPTY)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int n_kt = resolve<BATCH, SMALL, PACK, KT>(p, &raw_map, item, n_items).n_kt;
        for (int tb = 0; tb < n_kt; ++tb) {
          if (!mbar_wait(&dec_full[d], dph, abort_flag, p.status, DEV_TIMEOUT_FULL)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_r = tmem + kAcol0 + static_cast<uint32_t>(d * G::kAcols);
          const uint32_t a_i = a_r + KT / 4;
          const uint32_t b_r = smem_u32(bpl + d * G::kBStage);
          const uint32_t b_i = b_r + G::kTile;
#pragma unroll
          for (int k = 0; k < G::kSteps; ++k) {
            const uint32_t off = static_cast<uint32_t>(k * 32 * 128);  // 32 rows of 128 B
            const uint32_t first = (tb == 0 && k == 0) ? 1u : 0u;
            mma_f8f6f4_ta(tmem, a_r + 8 * k, smem_desc_sw128(b_r + off, kLbo, 1024), id256, first ^ 1u);
            mma_f8f6f4_ta(tmem, a_i + 8 * k, smem_desc_sw128(b_i + off, kLbo, 1024), id128, 1u);
            mma_f8f6f4_ta(tmem + 128, a_i + 8 * k, smem_desc_sw128(b_r + off, kLbo, 1024), id128n, 1u);
          }
          mma_commit(&dec_empty[d]);
          if (++d == DEC) {
            d = 0;
            dph ^= 1u;
          }
        }
        if (ok) mma_commit(tfull);
      }
      volatile int never = 0;
      mma_commit(mma_done);
      mbar_wait(mma_done, 0, &never, p.status, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp < kEpiWarps) {
    // Epilogue, warp w = tile rows 32w .. 32w + 31 (TMEM lanes of quarter w).  Phase 1 only moves
    // the accumulator out, so that it is free as soon as possible: Re bits to the shared-memory
    // staging tile, Im bits to the TMEM stash.  Phase 2, while the MMAs run the next tile pair,
    // converts, applies the offset corrections and writes the rows.  It reads the stash with
    // 16-lane x 256-bit loads, which give thread t columns 2 (t % 4), + 1 (and 8 on) of rows
    // t / 4 and t / 4 + 8, and phase 1 stages each row's Re in that column order, so four threads
    // write 16 consecutive pairs of a row straight from registers.
    const int r_own = warp * 32 + lane;  // this thread's tile row in phase 1
    const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    int g = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++g) {
      const TItem it = resolve<BATCH, SMALL, PACK, KT>(p, &raw_map, item, n_items);
      const int c = it.c, I = it.I, J = it.J, n_inputs = it.n_inputs;
      const int t128 = 128 * it.n_kt * KT;  // 128 T over the padded block (padding decodes to u = 8 + 8i)
      const bool magic = t128 <= 128 * kMagicSamples;
      int2* out_c = it.out + (int64_t)c * it.n_pairs;
      const int row0 = I * kBlk + warp * 32;
      const int buf = g & 1;
      if (!SMALL && it.accumulate) {
        // the sums this tile pair adds to, pulled into L2 while its MMAs run: each thread
        // prefetches the 128-byte lines of its own row's segment (pairs J*128 .. min(J*128 + 127, i))
        const int i = I * kBlk + r_own;
        if (i < n_inputs) {
          const char* a = reinterpret_cast<const char*>(out_c + (int64_t)i * (i + 1) / 2 + J * kBlk);
          const char* e = a + 8 * ((I == J ? r_own : kBlk - 1) + 1);
          for (const char* l = reinterpret_cast<const char*>(reinterpret_cast<uintptr_t>(a) & ~uintptr_t(127)); l < e;
               l += 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(l < a ? a : l));
        }
      }
      if (!mbar_wait_warp(tfull, g & 1, abort_flag, p.status, DEV_TIMEOUT_TMEM_FULL) ||
          !mbar_wait_warp(&sfull[buf], (g >> 1) & 1, abort_flag, p.status, DEV_TIMEOUT_TMEM_FULL))
        break;
      tc_fence_after();
      // 16-pair chunks this warp keeps: none past the inputs (the packed channels), none wholly
      // above the diagonal
      const int n_ch = (PACK ? (warp * 32 >= p.pack_g * n_inputs || c * p.pack_g + (warp * 32) / n_inputs >= p.n_chan)
                             : row0 >= n_inputs)
                           ? 0
                       : I == J ? (warp * 32 + 31) / kChunk + 1
                                : kBlk / kChunk;
      {
        uint4* srow = reinterpret_cast<uint4*>(staging + r_own * kBlk);
        const int sw = staging_swizzle(r_own);
        for (int ch = 0; ch < n_ch; ++ch) {
          uint32_t re[16], nim[16];
          tmem_ld16(taddr + kChunk * ch, re);
          tmem_ld16(taddr + 128 + kChunk * ch, nim);
          tmem_ld_wait();
          tmem_st16(taddr + kStashCol + kChunk * ch, nim);
          // 16-byte piece q of the chunk holds columns 2q, 2q + 1, 8 + 2q, 9 + 2q (phase 2's order)
#pragma unroll
          for (int q = 0; q < kChunk / 4; ++q)
            srow[((kChunk * ch) / 4 + q) ^ sw] = make_uint4(re[2 * q], re[2 * q + 1], re[8 + 2 * q], re[9 + 2 * q]);
        }
        // Re = n_re - 8 P_a - 8 P_b + 128 T,  Im = -n_im - 8 Q_a + 8 Q_b: the row's part
        const int2 rs = sums[(buf * 2) * kBlk + r_own];  // (8P, 8Q) of this row's input
        rowc[r_own] = make_int2(t128 - rs.x - (magic ? kMagicBits : 0), -rs.y + (magic ? kMagicBits : 0));
      }
      // the accumulator (columns 0-255) is free once its loads have landed; the stash stores
      // (columns 256-383) need only land before phase 2 reads them
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);
      // phase 2 reads stash lanes that other threads of the warp stored
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      tc_fence_after();
      // phase 2: thread (rg, q) = (lane / 4, lane % 4) owns rows 32 warp + rg + 8m (m = 0..3) and,
      // in each 16-column chunk, columns 2q, 2q + 1, 8 + 2q, 9 + 2q
      const int2* cs = sums + (buf * 2 + (I == J ? 0 : 1)) * kBlk;  // (8P, 8Q) of the columns
      const int q4 = lane & 3, rg = lane >> 2;
      int2* row_out[4];  // the row's pairs (j = first .. last of the tile), or null
      int firstm[4], lastm[4];
      int2 rcm[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int rr = warp * 32 + rg + 8 * m;
        row_out[m] = nullptr;
        firstm[m] = 0;
        lastm[m] = I == J ? rr : kBlk - 1;  // last column of the row in the tile
        rcm[m] = rowc[rr];
        if (PACK) {
          const int blk = rr / n_inputs, cr = c * p.pack_g + blk;
          if (blk < p.pack_g && cr < p.n_chan) {
            firstm[m] = blk * n_inputs;
            const int i = rr - firstm[m];
            row_out[m] = it.out + (int64_t)cr * it.n_pairs + (int64_t)i * (i + 1) / 2;
          }
        } else {
          const int i = I * kBlk + rr;
          if (i < n_inputs) row_out[m] = out_c + (int64_t)i * (i + 1) / 2 + J * kBlk;
        }
      }
      for (int ch = 0; ch < n_ch; ++ch) {
        uint32_t im[2][8];  // [rows 0-15 | 16-31 of the warp][2j + h .. : column 8j + 2q + e of row rg + 8h]
        tmem_ld_16x256b_x2(taddr + kStashCol + kChunk * ch, im[0]);
        tmem_ld_16x256b_x2(taddr + (16u << 16) + kStashCol + kChunk * ch, im[1]);
        const int jc = kChunk * ch + 2 * q4;  // this thread's first column in the tile
        const int4 s0 = *reinterpret_cast<const int4*>(cs + jc);  // (8P, 8Q) of columns jc, jc + 1
        const int4 s1 = *reinterpret_cast<const int4*>(cs + jc + 8);
        const int sp[4] = {s0.x, s0.z, s1.x, s1.z}, sq[4] = {s0.y, s0.w, s1.y, s1.w};
        tmem_ld_wait();
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          if (row_out[m] == nullptr) continue;
          const int rr = warp * 32 + rg + 8 * m;
          const int first = firstm[m], last = lastm[m];
          if (jc > last || jc + 9 < first) continue;
          const uint4 re4 =
              *reinterpret_cast<const uint4*>(staging + rr * kBlk + ((((kChunk * ch) >> 2) + q4) ^ staging_swizzle(rr)) * 4);
          const uint32_t vr[4] = {re4.x, re4.y, re4.z, re4.w};
          const uint32_t* vi = im[m >> 1];
          const int h = m & 1;
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {  // columns jc + 8 jj, + 1
            const int j0 = jc + 8 * jj;
            int2 v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const uint32_t xr = vr[2 * jj + e], xi = vi[4 * jj + 2 * h + e];
              int nr, ni;
              if (magic) {
                nr = __float_as_int(fmaf(__uint_as_float(xr), 262144.0f, kMagic));
                ni = __float_as_int(fmaf(__uint_as_float(xi), 262144.0f, kMagic));
              } else {
                nr = __float2int_rn(__uint_as_float(xr) * 262144.0f);
                ni = __float2int_rn(__uint_as_float(xi) * 262144.0f);
              }
              v[e] = make_int2(nr + rcm[m].x - sp[2 * jj + e], -ni + rcm[m].y + sq[2 * jj + e]);
            }
            // (first is a multiple of 16 and j0 even: a pair of columns starts inside the row or before it)
            if (j0 > last || j0 < first) continue;
            int2* dst = row_out[m] + (j0 - first);
            const int nv = j0 + 1 <= last ? 2 : 1;
            if (SMALL && p.atomic_out) {  // time-split items of one tile add into the same pairs
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                if (e < nv) {
                  atomicAdd(&dst[e].x, v[e].x);
                  atomicAdd(&dst[e].y, v[e].y);
                }
              }
            } else if (nv == 2 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
              int4 w = make_int4(v[0].x, v[0].y, v[1].x, v[1].y);
              if (it.accumulate) {
                const int4 o = *reinterpret_cast<const int4*>(dst);
                w = make_int4(w.x + o.x, w.y + o.y, w.z + o.z, w.w + o.w);
              }
              *reinterpret_cast<int4*>(dst) = w;
            } else {
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                if (e < nv) {
                  int2 w = v[e];
                  if (it.accumulate) {
                    const int2 o = dst[e];
                    w.x += o.x;
                    w.y += o.y;
                  }
                  dst[e] = w;
                }
              }
            }
          }
        }
      }
      // the input sums are free
      __syncwarp();
      if (lane == 0) mbar_arrive(&sempty[buf]);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

template <int KT, int RAW, int DEC, bool BATCH = false, bool SMALL = false, bool PACK = false>
cudaError_t launch_ta(const CUtensorMap& raw_map, const TParams& p, int grid, cudaStream_t stream) {
  using G = TGeom<KT, RAW, DEC>;
  auto kern = xcorr_tc_fused_ta_kernel<KT, RAW, DEC, BATCH, SMALL, PACK>;
  static int attr_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_device != dev) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmem);
    if (e != cudaSuccess) return e;
    attr_device = dev;
  }
  kern<<<grid, kThreads, G::kSmem, stream>>>(raw_map, p);
  return cudaGetLastError();
}

}  // namespace

// The tensor-memory-A shapes: 128 samples with 2 raw + 2 decoded stages, 96 with 3 + 2, 64 with 4 + 4,
// and (3) the small-problem layout on 128 x (2 + 2).
int fused_ta_stage_samples(int variant) { return variant == 0 || variant == 3 ? 128 : variant == 1 ? 96 : 64; }

// The small-problem layout of a launch: channels packed per tile and the time split.
void small_layout(int n_chan, int n_inputs, int n_kt, int num_sms, int& pack_g, int& tiles, int& n_split,
                  int& split_kt) {
  const int nb = (n_inputs + kBlk - 1) / kBlk;
  pack_g = n_inputs <= kBlk / 2 ? kBlk / n_inputs : 1;
  tiles = pack_g > 1 ? (n_chan + pack_g - 1) / pack_g : n_chan * (nb * (nb + 1) / 2);
  // as many splits as keep the items within one wave of the SMs, each at least one stage long
  n_split = tiles >= num_sms ? 1 : num_sms / tiles;
  if (n_split > n_kt) n_split = n_kt;
  split_kt = (n_kt + n_split - 1) / n_split;
  n_split = (n_kt + split_kt - 1) / split_kt;
}

cudaError_t launch_xcorr_tc_fused_ta_ci4(const uint8_t* in, int row_chans, int variant, int n_time, int n_chan,
                                         int n_inputs, int2* out, bool accumulate, int* status, int num_sms,
                                         cudaStream_t stream) {
  const int nb = (n_inputs + kBlk - 1) / kBlk;
  const int kt = fused_ta_stage_samples(variant);
  if (n_time <= 0 || n_inputs % 16 != 0 || reinterpret_cast<uintptr_t>(in) % 16 != 0 ||
      kFusedWindowCI4 % kt != 0)
    return cudaErrorInvalidValue;
  TParams p{};
  p.n_chan = n_chan;
  p.n_inputs = n_inputs;
  p.n_tile_pairs = nb * (nb + 1) / 2;
  p.n_pairs = (int64_t)n_inputs * (n_inputs + 1) / 2;
  p.out = out;
  p.status = status;
  p.one = 1u;
  const bool small = variant == 3;
  CUtensorMap raw_map;
  if (row_chans < n_chan) return cudaErrorInvalidValue;
  int pack_g = 1;
  if (small) pack_g = n_inputs <= kBlk / 2 ? kBlk / n_inputs : 1;
  if (pack_g > 1) {
    // the packed view: one time row is n_chan * n_inputs bytes (channel-major), read in boxes of 128
    // (pack_g channels side by side) x 1 x kt; the middle dimension has extent 1
    if (!encode_raw_ci4_packed_tmap(&raw_map, in, n_inputs, n_chan, row_chans, n_time, kt, nullptr))
      return cudaErrorInvalidValue;
  } else if (!encode_raw_ci4_tmap(&raw_map, in, n_inputs, n_chan, row_chans, n_time, kt, nullptr)) {
    return cudaErrorInvalidValue;
  }
  p.pack_g = pack_g;
  // one exactly-summed block per launch; later blocks add into the first
  for (int t0 = 0; t0 < n_time; t0 += kFusedWindowCI4) {
    const int len = n_time - t0 < kFusedWindowCI4 ? n_time - t0 : kFusedWindowCI4;
    p.t0 = t0;
    p.n_kt = (len + kt - 1) / kt;
    p.accumulate = (accumulate || t0 > 0) ? 1 : 0;
    int tiles = n_chan * p.n_tile_pairs;
    p.n_split = 1;
    p.split_kt = p.n_kt;
    if (small) small_layout(n_chan, n_inputs, p.n_kt, num_sms, pack_g, tiles, p.n_split, p.split_kt);
    p.atomic_out = p.n_split > 1 ? 1 : 0;
    p.n_items = tiles * p.n_split;
    if (p.atomic_out && !p.accumulate) {  // the split items add into a cleared output
      cudaError_t e = cudaMemsetAsync(out, 0, (size_t)n_chan * p.n_pairs * sizeof(int2), stream);
      if (e != cudaSuccess) return e;
      p.accumulate = 1;
    }
    const int grid = p.n_items < num_sms ? p.n_items : num_sms;
    cudaError_t e;
    switch (variant) {
      case 0: e = launch_ta<128, 2, 2>(raw_map, p, grid, stream); break;
      case 1: e = launch_ta<96, 3, 2>(raw_map, p, grid, stream); break;
      case 2: e = launch_ta<64, 4, 4>(raw_map, p, grid, stream); break;
      default:  // the small-problem layout; with neither packing nor a split it is shape 0's launch
        e = pack_g > 1         ? launch_ta<128, 2, 2, false, true, true>(raw_map, p, grid, stream)
            : p.n_split > 1    ? launch_ta<128, 2, 2, false, true, false>(raw_map, p, grid, stream)
                               : launch_ta<128, 2, 2>(raw_map, p, grid, stream);
        break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace xc

namespace xc {

// The batch form: one launch over items (subarray, channel, I, J) of several 4-bit problems, each
// with its own descriptor (raw tensor map with box_t = the variant's stage height, output, sizes;
// one exactly-summed block each: n_kt * KT <= kFusedWindowCI4).
cudaError_t launch_xcorr_tc_fused_ta_batch(const TaSubDesc* subs, const uint4* items, int n_items, int variant,
                                           int* status, int num_sms, cudaStream_t stream) {
  if (n_items <= 0) return cudaSuccess;
  TParams p{};
  p.status = status;
  p.one = 1u;
  p.n_split = 1;
  p.subs = subs;
  p.items = items;
  p.n_batch_items = n_items;
  CUtensorMap unused{};
  const int grid = n_items < num_sms ? n_items : num_sms;
  switch (variant) {
    case 0: return launch_ta<128, 2, 2, true>(unused, p, grid, stream);
    case 1: return launch_ta<96, 3, 2, true>(unused, p, grid, stream);
    default: return launch_ta<64, 4, 4, true>(unused, p, grid, stream);
  }
}

}  // namespace xc
