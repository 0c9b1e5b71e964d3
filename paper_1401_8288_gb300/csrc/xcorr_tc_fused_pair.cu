// xcorr_tc_fused_pair.cu -- the fused 4-bit X-stage on CTA pairs: two SMs
// share one column tile through a cta_group::2 tcgen05 MMA.
//
// Same result as xcorr_tc_fused_ta.cu (per channel, the packed lower triangle
// of V = sum_t x_t x_t^H; Sec. 1, Sec. 2.1, Eq. 1) from the same raw [t][c][i]
// CI4 bytes and the same offset-binary E4M3 operands u = t + 8, with the row
// tile's operand decoded into tensor memory as there.  Two CTAs of a 2-CTA
// cluster, on two SMs, work on two tile pairs (c, R0, S) and (c, R1, S) that
// share the column tile S:
//
//   * each CTA decodes its own row tile R into its tensor memory (A) and only
//     HALF of S, inputs 64 rank .. 64 rank + 63, into its shared memory as three
//     64-byte-wide planes with the 64-byte swizzle: real codes, imaginary codes,
//     negated real codes (the E4M3 sign bit);
//   * the even CTA issues the MMAs for both, M = 256 (rows 0-127 the even CTA's
//     A, rows 128-255 the odd CTA's) and N = 256 (columns 0-127 from the even
//     CTA's planes, 128-255 from the odd CTA's): per 32-sample step
//     [Re | Im] += A_re [B_re | B_im] and [Re | Im] += A_im [B_im | -B_re], with
//     Im = A_re B_im - A_im B_re (the accumulated -Im of the correction below),
//     so the accumulator of each CTA holds [Re | Im] of the even CTA's 64
//     columns, then of the odd CTA's.  An N = 256 MMA keeps the tensor pipe fed
//     while decoder warps share the issuing warp's SMSP; a stream of N = 128
//     MMAs lost 20-40 % there.
//
// Per SM and stage this halves the column tile's TMA bytes, decode work and
// the tensor core's operand reads against the single-SM kernel.
//
// A channel's tile pairs are grouped by their column tile (fused_pairing.h).
// Column tile S has the row tiles S .. nb - 1; where that count is odd, the
// columns are matched two by two (u, u + 2) and the tile pair (u + 2, u) is
// computed TRANSPOSED, as rows u against columns u + 2: its epilogue writes
// V[b][a] = conj(W[a][b]), where each warp holds 32 consecutive a of one output
// row, so those stores are coalesced as they come out of tensor memory.  Only
// when the channel has an odd number of tile pairs does one entry keep a single
// tile pair (the odd CTA's rows are then computed and dropped).
//
// Eight decoder warps form two groups of four (one warp per tensor-memory lane
// quarter) that take alternate stages; a warp pulls its raw stage into
// registers and returns the slot to the producer before decoding.  Across the
// pair, the odd CTA signals the even one with small bulk copies that complete
// bytes on the even CTA's barriers (a cluster-scope release-arrive stalls the
// arriving thread for over a thousand cycles), the MMAs' commits multicast to
// both CTAs, and each CTA's half of the column sums that undo the offset
// crosses to the other CTA as a bulk copy.  The row sums come from each CTA's
// own A decoders.  Every wait is bounded (sm103_ptx.cuh); the CTAs meet at a
// cluster barrier before their tensor memory is released.
#include "fused_common.cuh"
#include "fused_pairing.h"
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
constexpr int kDecGroups = 2;                    // decoder groups taking alternate stages
constexpr int kGroupWarps = kDecWarps / kDecGroups;  // one warp per tensor-memory lane quarter
constexpr int kChunk = 16;
constexpr int kPitch = kChunk + 1;
constexpr int kHalf = 64;                                 // column-tile inputs each CTA decodes
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kStashCol = 256;                       // Im of the first STASH column chunks after the accumulator
constexpr int kStagingBytes = kBlk * kBlk * 4;            // Re accumulator bits of a whole tile pair
constexpr int kSumsBytes = 2 * 2 * kBlk * 8;              // [item parity][rows R, columns S][input] (8P, 8Q)
// Every partial sum of u_a u_b is n 2^-18 with 0 <= n <= 450 T (and |n| <= 225 T for Im).
// For T <= kMagicSamples, |n| < 2^22 and n + 1.5 2^23 is exact in FP32, so one FFMA
// against that constant turns the accumulator into n (in the low bits of the result).
constexpr int kMagicSamples = 9320;
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;
constexpr int kScratchBytes = kDecWarps * 4 * kPitch * 8;  // [decoder warp][chunk][input] (P, Q), padded rows
constexpr int kRscratchBytes = kBlk * 8;                   // the second decoder group's row sums
constexpr int kBarrierBytes = 512;
// The odd CTA signals the even one with 16-byte copies of a token into per-warp sink slots:
// one per decoder warp and stage, one per epilogue warp and item.
constexpr int kSinkSlots = kDecWarps + kEpiWarps;
constexpr uint32_t kSignalBytes = 16;

// STASH: 16-column chunks of Im kept in tensor memory after the accumulator (the rest of Im goes to
// shared memory); the A stages follow the stash.
template <int KT, int RAW, int DEC, int STASH>
struct PGeom {
  static constexpr uint32_t kAcol0 = kStashCol + 16 * STASH;
  static constexpr int kImHiCols = kBlk - 16 * STASH;       // Im columns staged in shared memory
  static constexpr int kImHiBytes = kBlk * kImHiCols * 4;
  static constexpr int kTileA = KT * kBlk;   // raw row tile: KT rows of 128 bytes, 128-byte swizzle
  static constexpr int kTileB = KT * kHalf;  // raw half column tile: KT rows of 64 bytes, 64-byte swizzle
  static constexpr int kRawStage = kTileA + kTileB;
  static constexpr int kPlane = KT * kHalf;  // one decoded B plane (same layout as the raw half)
  static constexpr int kBStage = 3 * kPlane;  // real codes, imaginary codes, negated real codes
  static constexpr int kAcols = KT / 2;      // one A stage: KT / 4 columns of real codes, then imaginary
  static constexpr int kRowsB = KT / (kGroupWarps * 32 / 4);  // B rows per decoder thread and stage
  static constexpr int kSteps = KT / 32;                 // MMA steps (32 samples) per stage
  // byte offsets of the buffers from the 1024-aligned start of shared memory; the kernel takes
  // its pointers from these, and the allocation is their end (plus the alignment slack)
  static constexpr int kOffBpl = RAW * kRawStage;
  static constexpr int kOffStaging = kOffBpl + DEC * kBStage;
  static constexpr int kOffImHi = kOffStaging + kStagingBytes;
  static constexpr int kOffSums = kOffImHi + kImHiBytes;
  static constexpr int kOffScratch = kOffSums + kSumsBytes;
  static constexpr int kOffRscratch = kOffScratch + kScratchBytes;
  static constexpr int kOffBarriers = kOffRscratch + kRscratchBytes;
  static constexpr int kSmem = 1024 + kOffBarriers + kBarrierBytes;
  static_assert(KT % 32 == 0, "stages hold whole MMA steps and whole 32-row B passes");
  // each decoder group waits only on its own raw slots (stage s uses slot s % RAW, decoded by group
  // s % 2), so no group can test a raw barrier a phase ahead of another group's fill
  static_assert(RAW % kDecGroups == 0, "raw slots belong to one decoder group each");
  static_assert(kRawStage % 1024 == 0 && kTileA % 1024 == 0, "swizzle atoms stay aligned");
  static_assert(DEC * kAcols <= static_cast<int>(kTmemCols - kAcol0), "A stages fit beside the accumulator");
  static_assert(STASH >= 0 && STASH <= 8, "stash chunks");
  static_assert((2 * RAW + 2 * DEC + 7) * 8 + 8 + 16 + 16 * kSinkSlots <= kBarrierBytes, "barrier area");
  static_assert(kSmem <= 232448, "shared memory budget");
};

struct PParams {
  int n_chan, n_inputs;
  int nb;              // row / column tiles
  int n_entries;       // pair entries per channel
  int t0;              // first sample of this launch
  int n_kt;            // stages per tile pair
  int64_t n_pairs;
  int accumulate;      // add into out (else store)
  int2* out;
  int* status;
  uint32_t one;        // 1: a multiplier the compiler cannot fold (see lane_add)
};

// One CTA's share of a pair entry.
struct PItem {
  int c, S, R;  // channel, column tile, this CTA's row tile (-1: none)
  bool valid, has_row, transposed;
};

__device__ __forceinline__ PItem pair_item(const PParams& p, int q, int n_items, uint32_t rank) {
  PItem it{};
  it.valid = q < n_items;
  if (!it.valid) return it;
  it.c = q / p.n_entries;
  int r0, r1;
  pair_entry(p.nb, q - it.c * p.n_entries, it.S, r0, r1);
  it.R = rank == 0 ? r0 : r1;
  it.has_row = it.R >= 0;
  it.transposed = it.has_row && it.R < it.S;
  return it;
}

// L2 prefetch of stage s of an item: this CTA's row tile and its half of the column tile.
template <int KT>
__device__ __forceinline__ void prefetch_pair_stage(const CUtensorMap* map_a, const CUtensorMap* map_b,
                                                    const PItem& it, uint32_t rank, const PParams& p, int s) {
  if (!it.valid || s >= p.n_kt) return;
  const int t = p.t0 + s * KT;
  if (it.has_row) tma_prefetch_3d(map_a, it.R * kBlk, it.c, t);
  if (it.S * kBlk + kHalf * static_cast<int>(rank) < p.n_inputs)
    tma_prefetch_3d(map_b, it.S * kBlk + kHalf * static_cast<int>(rank), it.c, t);
}

// 16-byte chunk swizzle of the Re staging tile (as in the single-SM kernel).
__device__ __forceinline__ int staging_swizzle(int row) { return ((row & 1) << 2) | ((row >> 1) & 3); }

template <int KT, int RAW, int DEC, int STASH>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    xcorr_tc_fused_pair_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                               const __grid_constant__ PParams p) {
  using G = PGeom<KT, RAW, DEC, STASH>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* raw = smem;                      // [stage][row tile | half column tile]
  uint8_t* bpl = smem + G::kOffBpl;  // [stage][real plane | imaginary plane | negated real plane]
  uint32_t* staging = reinterpret_cast<uint32_t*>(smem + G::kOffStaging);  // Re [row][16-byte chunk ^ swz(row)]
  uint32_t* im_hi = reinterpret_cast<uint32_t*>(smem + G::kOffImHi);  // Im past the stash, same layout
  int2* sums = reinterpret_cast<int2*>(smem + G::kOffSums);
  int2* scratch = reinterpret_cast<int2*>(smem + G::kOffScratch);
  int2* rscratch = reinterpret_cast<int2*>(smem + G::kOffRscratch);
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem + G::kOffBarriers);
  uint64_t* raw_empty = raw_full + RAW;
  uint64_t* dec_full = raw_empty + RAW;  // even CTA: both CTAs' decoders filled the stage
  uint64_t* dec_empty = dec_full + DEC;  // both CTAs: the pair's MMAs are done with the stage
  uint64_t* tfull = dec_empty + DEC;     // both CTAs: the accumulator holds an item
  uint64_t* tempty = tfull + 1;          // even CTA: both epilogues have the item out of it
  uint64_t* sfull = tempty + 1;          // [2] both CTAs' sums of an item are written
  uint64_t* sempty = sfull + 2;          // [2] both epilogues are done with them
  uint64_t* mma_done = sempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  uint8_t* token = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tslot + 2) + 15) & ~uintptr_t(15));
  uint8_t* sink = token + kSignalBytes;  // [kSinkSlots][16], written by the odd CTA's signals

  const uint32_t rank = cluster_ctarank(), peer = rank ^ 1u;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < RAW; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], kGroupWarps);
    }
    // dec_full, tempty: the even CTA's own warps arrive (one of them expecting the odd CTA's
    // signal bytes); sfull: the local decoders arrive expecting the other CTA's column sums
    for (int s = 0; s < DEC; ++s) {
      mbar_init(&dec_full[s], kGroupWarps);
      mbar_init(&dec_empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, kEpiWarps);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sfull[b], 1);
      mbar_init(&sempty[b], 2 * kEpiWarps);
    }
    for (int k = 0; k < 4; ++k) reinterpret_cast<uint32_t*>(token)[k] = 0u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the token is read by the async proxy
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) tmem_alloc_pair(tslot, kTmemCols);
  tc_fence_before();
  cluster_sync();  // both CTAs' barriers and tensor memory exist before either touches the other's
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int n_items = p.n_chan * p.n_entries;
  const int cl = static_cast<int>(blockIdx.x >> 1), n_cl = static_cast<int>(gridDim.x >> 1);

  if (warp == kProducerWarp) {
    if (lane == 0) {
      constexpr int kAhead = kPrefetchSamples / KT;  // L2 prefetch runs this many stages ahead of the loads
      prefetch_tmap(&map_a);
      prefetch_tmap(&map_b);
      PItem next = pair_item(p, cl, n_items, rank);
      for (int s = 0; s < kAhead; ++s) prefetch_pair_stage<KT>(&map_a, &map_b, next, rank, p, s);
      int r = 0;
      uint32_t ph = 0, filled = 0, fill_parity[RAW] = {};
      bool ok = true;
      for (int q = cl; ok && q < n_items; q += n_cl) {
        const PItem it = next;
        next = pair_item(p, q + n_cl, n_items, rank);
        const int xb = it.S * kBlk + kHalf * static_cast<int>(rank);
        const bool load_b = xb < p.n_inputs;  // a half wholly past the inputs is never written out
        for (int tb = 0; tb < p.n_kt; ++tb) {
          if (tb + kAhead < p.n_kt)
            prefetch_pair_stage<KT>(&map_a, &map_b, it, rank, p, tb + kAhead);
          else
            prefetch_pair_stage<KT>(&map_a, &map_b, next, rank, p, tb + kAhead - p.n_kt);
          if (!mbar_wait(&raw_empty[r], ph ^ 1u, abort_flag, p.status, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          uint8_t* st = raw + r * G::kRawStage;
          const int t = p.t0 + tb * KT;
          mbar_expect_tx(&raw_full[r], (it.has_row ? G::kTileA : 0) + (load_b ? G::kTileB : 0));
          if (it.has_row) tma_load_3d(st, &map_a, &raw_full[r], it.R * kBlk, it.c, t);
          if (load_b) tma_load_3d(st + G::kTileA, &map_b, &raw_full[r], xb, it.c, t);
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
    // Two groups of four decoder warps take alternate stages (group g decodes the CTA's stages
    // s with s % 2 == g, counted over all its items), so each warp has two stage times for one
    // stage's decode and its waits, fences and signal.  Warp q of a group (q = warp % 4) owns
    // tensor-memory lane quarter q (the A codes of inputs 32q .. 32q + 31) and a quarter of the
    // half column tile's B rows.
    const int dw = warp - kDecWarp0, tid = dw * 32 + lane;
    const int grp = dw / kGroupWarps, q = warp & 3, gtid = (dw % kGroupWarps) * 32 + lane;
    const uint32_t a_lanes = static_cast<uint32_t>(32 * q) << 16;
    // input chunks 2q, 2q + 1 of row 16 sb + lane (128-byte swizzle; 16 sb = 0 mod 8)
    const int apos0 = ((2 * q) ^ (lane & 7)) << 4;
    const int apos1 = ((2 * q + 1) ^ (lane & 7)) << 4;
    // B: a fixed 16-input chunk L of the half column tile, rows phase, phase + 32, ...; under the
    // 64-byte swizzle chunk L of row k sits at chunk L ^ ((k >> 1) & 3), the same for every pass
    const int L = gtid & 3, phase = gtid >> 2;
    const int bpos = (L ^ ((phase >> 1) & 3)) << 4;
    const uint32_t dfull_even = smem_cluster(dec_full, 0);  // the even CTA's dec_full[0]
    const uint32_t sink_even = smem_cluster(sink + kSignalBytes * dw, 0);
    uint32_t gs = 0;  // the CTA's stages before the current item
    int g = 0;
    for (int qi = cl; qi < n_items; qi += n_cl, ++g) {
      const PItem cur = pair_item(p, qi, n_items, rank);
      // A sums of chunk 2q + c: input 16 (2q + c) + lane / 4 (h = 0) and + 8 (h = 1), over samples
      // 4 (lane % 4) .. + 3 of every 16
      uint32_t sar[2][2] = {{0u, 0u}, {0u, 0u}}, sai[2][2] = {{0u, 0u}, {0u, 0u}};
      // B sums in 16-bit lanes: word e / 2, half e % 2 holds input e of chunk L
      uint32_t s_re[8], s_im[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) s_re[k] = s_im[k] = 0u;
      bool ok = true;
      for (int tb = (grp ^ static_cast<int>(gs)) & 1; tb < p.n_kt; tb += kDecGroups) {
        const uint32_t st = gs + static_cast<uint32_t>(tb);  // the CTA's stage index
        const int r = static_cast<int>(st % RAW), d = static_cast<int>(st % DEC);
        const uint32_t rph = (st / RAW) & 1u, dph = (st / DEC) & 1u;
        if (!mbar_wait_warp(&raw_full[r], rph, abort_flag, p.status, DEV_TIMEOUT_FULL)) {
          ok = false;
          break;
        }
        // the whole raw stage into registers (A: 16 samples x 16 inputs per ldmatrix; B: this
        // thread's rows), so that the slot goes back to the producer before the decode: its next
        // fill then overlaps the decode instead of following it
        constexpr int R = G::kRowsB;
        const uint8_t* raw_a = raw + r * G::kRawStage;
        uint32_t xa[KT / 16][2][2];  // [16-sample block][input chunk][register]
        if (cur.has_row) {
#pragma unroll
          for (int sb = 0; sb < KT / 16; sb += 2)
#pragma unroll
            for (int c = 0; c < 2; ++c)
              ldmatrix_t_b8_x2(smem_u32(raw_a + (16 * sb + lane) * 128 + (c ? apos1 : apos0)), xa[sb][c][0],
                               xa[sb][c][1], xa[sb + 1][c][0], xa[sb + 1][c][1]);
        }
        uint4 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k)
          v[k] = *reinterpret_cast<const uint4*>(raw_a + G::kTileA + bpos + (phase + 32 * k) * kHalf);
        __syncwarp();
        if (lane == 0) mbar_arrive(&raw_empty[r]);
        if (!mbar_wait_warp(&dec_empty[d], dph ^ 1u, abort_flag, p.status, DEV_TIMEOUT_EMPTY)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // A operand: decoded in registers, stored to TMEM
        if (cur.has_row) {
          const uint32_t ta = tmem + a_lanes + G::kAcol0 + static_cast<uint32_t>(d * G::kAcols);
#pragma unroll
          for (int sb = 0; sb < KT / 16; sb += 2) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              uint32_t re0, im0, re1, im1, re2, im2, re3, im3;
              offset_codes(xa[sb][c][0], re0, im0);
              offset_codes(xa[sb][c][1], re1, im1);
              offset_codes(xa[sb + 1][c][0], re2, im2);
              offset_codes(xa[sb + 1][c][1], re3, im3);
              // the two blocks' codes of one input add per byte (<= 30) before the dp4a
              sar[c][0] = __dp4a(re0 + re2, 0x01010101u, sar[c][0]);
              sai[c][0] = __dp4a(im0 + im2, 0x01010101u, sai[c][0]);
              sar[c][1] = __dp4a(re1 + re3, 0x01010101u, sar[c][1]);
              sai[c][1] = __dp4a(im1 + im3, 0x01010101u, sai[c][1]);
              const uint32_t tc = ta + (static_cast<uint32_t>(16 * c) << 16);
              tmem_st_16x128b_x2(tc + 4 * sb, re0, re1, re2, re3);
              tmem_st_16x128b_x2(tc + KT / 4 + 4 * sb, im0, im1, im2, im3);
            }
          }
        }
        // B operand: this CTA's half of the column tile, real and imaginary planes at the raw
        // chunk's swizzled offset
        {
          uint8_t* re_t = bpl + d * G::kBStage + bpos;
          uint8_t* im_t = re_t + G::kPlane;
          uint8_t* nre_t = im_t + G::kPlane;
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
            const int off = (phase + 32 * k) * kHalf;
            *reinterpret_cast<uint4*>(re_t + off) = re;
            *reinterpret_cast<uint4*>(im_t + off) = im;
            // -u: the E4M3 sign bit (u >= 0)
            *reinterpret_cast<uint4*>(nre_t + off) =
                make_uint4(re.x ^ 0x80808080u, re.y ^ 0x80808080u, re.z ^ 0x80808080u, re.w ^ 0x80808080u);
          }
          // widen to 16-bit lanes: inputs (4k, 4k+1) -> word 2k, (4k+2, 4k+3) -> word 2k+1
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            lane_add(s_re[2 * k], __byte_perm(a_re[k], 0u, 0x4140), p.one);
            lane_add(s_re[2 * k + 1], __byte_perm(a_re[k], 0u, 0x4342), p.one);
            lane_add(s_im[2 * k], __byte_perm(a_im[k], 0u, 0x4140), p.one);
            lane_add(s_im[2 * k + 1], __byte_perm(a_im[k], 0u, 0x4342), p.one);
          }
        }
        // the pair's MMAs read A through tensor memory and B through the async proxy; the even
        // CTA's warps arrive on their own barrier, the odd CTA's send it a signal copy (issued
        // after their plane writes reached the async proxy)
        tmem_st_wait();
        tc_fence_before();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if (rank != 0)
            bulk_copy_to_cluster(sink_even, token, kSignalBytes, dfull_even + 8u * static_cast<uint32_t>(d));
          else if (q == 0)
            mbar_expect_tx(&dec_full[d], kGroupWarps * kSignalBytes);
          else
            mbar_arrive(&dec_full[d]);
        }
      }
      gs += static_cast<uint32_t>(p.n_kt);
      // row sums: the four lanes holding one input's samples are lanes 4k .. 4k + 3
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int m = 1; m <= 2; m <<= 1) {
            sar[c][h] += __shfl_xor_sync(0xFFFFFFFFu, sar[c][h], m);
            sai[c][h] += __shfl_xor_sync(0xFFFFFFFFu, sai[c][h], m);
          }
      // column sums of this warp: lanes L, L + 4, ..., L + 28 hold chunk L
      int2 pq[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int sr = static_cast<int>((s_re[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
        const int si = static_cast<int>((s_im[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
        pq[e] = make_int2(sr + si, si - sr);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) {
#pragma unroll
        for (int m = 4; m <= 16; m <<= 1) {
          pq[e].x += __shfl_xor_sync(0xFFFFFFFFu, pq[e].x, m);
          pq[e].y += __shfl_xor_sync(0xFFFFFFFFu, pq[e].y, m);
        }
      }
      if (lane < 4) {
#pragma unroll
        for (int e = 0; e < 16; ++e) scratch[(dw * 4 + lane) * kPitch + e] = pq[e];
      }
      // the second group's row sums go through shared memory to the first
      if (grp == 1 && (lane & 3) == 0) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int h = 0; h < 2; ++h)
            rscratch[16 * (2 * q + c) + 8 * h + (lane >> 2)] =
                make_int2(static_cast<int>(sar[c][h]), static_cast<int>(sai[c][h]));
      }
      dec_bar_sync(kDecThreads);
      const int buf = g & 1;
      // both CTAs' epilogues must be done with this buffer: the column sums go to both
      if (ok) ok = mbar_wait_warp(&sempty[buf], ((g >> 1) & 1) ^ 1, abort_flag, p.status, DEV_TIMEOUT_TMEM_EMPTY);
      if (ok) {
        int2* rows = sums + (buf * 2) * kBlk;
        if (grp == 0 && cur.has_row && (lane & 3) == 0) {
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int e = 16 * (2 * q + c) + 8 * h + (lane >> 2);
              const int2 o = rscratch[e];
              const int sr = static_cast<int>(sar[c][h]) + o.x, si = static_cast<int>(sai[c][h]) + o.y;
              rows[e] = make_int2(8 * (sr + si), 8 * (si - sr));
            }
        }
        if (tid < kHalf) {
          int2 sm = make_int2(0, 0);
#pragma unroll
          for (int w = 0; w < kDecWarps; ++w) {
            const int2 x = scratch[(w * 4 + (tid >> 4)) * kPitch + (tid & 15)];
            sm.x += x.x;
            sm.y += x.y;
          }
          sums[(buf * 2 + 1) * kBlk + kHalf * static_cast<int>(rank) + tid] = make_int2(8 * sm.x, 8 * sm.y);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // read by the copy below
        }
      }
      if (dec_bar_or(!ok || *abort_flag, kDecThreads)) break;
      if (tid == 0) {
        // this CTA's half of the column sums goes to the other CTA's copy of the buffer; the local
        // barrier expects the other half
        const int2* half = sums + (buf * 2 + 1) * kBlk + kHalf * static_cast<int>(rank);
        mbar_expect_tx(&sfull[buf], kHalf * 8);
        bulk_copy_to_cluster(smem_cluster(half, peer), half, kHalf * 8, smem_cluster(&sfull[buf], peer));
      }
    }
  } else if (warp == kMmaWarp) {
    if (rank == 0 && lane == 0) {
      // two M = 256, N = 256 MMAs per 32-sample step; each CTA's 128 B columns are two 64-byte-wide
      // atoms one plane apart: [re | im] for the real codes of A, [im | -re] for the imaginary ones,
      // so D holds [Re | Im] of the even CTA's 64 columns, then of the odd CTA's
      const uint32_t idesc = instr_desc_ta(kTypeE4M3, 256, 256, false);
      constexpr uint32_t kLbo = G::kPlane;  // between the two atoms of a CTA's 128 columns
      constexpr uint32_t kSbo = 8 * kHalf;  // eight K rows of 64 bytes
      int d = 0, g = 0;
      uint32_t dph = 0;
      bool ok = true;
      for (int qi = cl; ok && qi < n_items; qi += n_cl, ++g) {
        if (!mbar_wait(tempty, (g & 1) ^ 1, abort_flag, p.status, DEV_TIMEOUT_TMEM_EMPTY)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int tb = 0; tb < p.n_kt; ++tb) {
          if (!mbar_wait(&dec_full[d], dph, abort_flag, p.status, DEV_TIMEOUT_FULL)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_r = tmem + G::kAcol0 + static_cast<uint32_t>(d * G::kAcols);
          const uint32_t a_i = a_r + KT / 4;
          const uint64_t b_r = smem_desc_sw64(smem_u32(bpl + d * G::kBStage), kLbo, kSbo);
          const uint64_t b_i = b_r + (G::kPlane >> 4);  // the start address field counts 16 bytes
#pragma unroll
          for (int k = 0; k < G::kSteps; ++k) {
            const uint64_t off = static_cast<uint64_t>((k * 32 * kHalf) >> 4);  // 32 rows of 64 B
            mma_pair_f8f6f4_ta(tmem, a_r + 8 * k, b_r + off, idesc, (tb == 0 && k == 0) ? 0u : 1u);
            mma_pair_f8f6f4_ta(tmem, a_i + 8 * k, b_i + off, idesc, 1u);
          }
          mma_pair_commit_both(&dec_empty[d]);
          if (++d == DEC) {
            d = 0;
            dph ^= 1u;
          }
        }
        if (ok) mma_pair_commit_both(tfull);
      }
      // the odd CTA's last signals land here once both epilogues have drained the last item
      if (ok) mbar_wait(tempty, (g & 1) ^ 1, abort_flag, p.status, DEV_TIMEOUT_TMEM_EMPTY);
      // the pair's MMAs write both CTAs' tensor memory: let them finish before the cluster barrier
      volatile int never = 0;
      mma_pair_commit_both(mma_done);
      mbar_wait(mma_done, 0, &never, p.status, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp < kEpiWarps) {
    // Epilogue, warp w = tile rows 32w .. 32w + 31 (TMEM lanes of quarter w).  Phase 1 moves the
    // accumulator out (Re bits to the shared-memory staging tile, Im bits to the TMEM stash) so that
    // it is free as soon as possible; phase 2, while the MMAs run the next item, converts, applies
    // the offset corrections and writes.  A transposed item writes V[b][a], b in the column tile:
    // lane a of warp w holds a's row of W, so the warp's 32 values of output row b are consecutive.
    // Otherwise phase 2 reads the Im stash with 16-lane x 256-bit loads, which give thread t
    // columns 2 (t % 4), + 1 (and 8 on) of rows t / 4 and t / 4 + 8; phase 1 stages each row's Re
    // and the rest of its Im in that column order, so four threads write 16 consecutive pairs of a
    // row straight from registers.
    const int r_own = warp * 32 + lane;  // this thread's tile row in phase 1
    const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    const uint32_t tempty_even = smem_cluster(tempty, 0);
    const uint32_t sink_even = smem_cluster(sink + kSignalBytes * (kDecWarps + warp), 0);
    const uint32_t sempty_peer = smem_cluster(sempty, peer);
    const int t128 = 128 * p.n_kt * KT;  // 128 T over the padded block (padding decodes to u = 8 + 8i)
    const bool magic = t128 <= 128 * kMagicSamples;
    const int n_inputs = p.n_inputs;
    int g = 0;
    for (int q = cl; q < n_items; q += n_cl, ++g) {
      const PItem it = pair_item(p, q, n_items, rank);
      const int R = it.R, S = it.S;
      int2* out_c = p.out + (int64_t)it.c * p.n_pairs;
      const int buf = g & 1;
      if (p.accumulate && it.has_row) {
        // the sums this item adds to, pulled into L2 while its MMAs run: each thread prefetches
        // the 128-byte lines of one output row's segment
        int i, j0, len;
        if (it.transposed) {  // row S*128 + r_own, columns R*128 .. R*128 + 127
          i = S * kBlk + r_own;
          j0 = R * kBlk;
          len = kBlk;
        } else {              // row R*128 + r_own, columns S*128 .. min(S*128 + 127, i)
          i = R * kBlk + r_own;
          j0 = S * kBlk;
          len = R == S ? r_own + 1 : kBlk;
        }
        if (i < n_inputs) {
          const char* a = reinterpret_cast<const char*>(out_c + (int64_t)i * (i + 1) / 2 + j0);
          const char* e = a + 8 * len;
          for (const char* l = reinterpret_cast<const char*>(reinterpret_cast<uintptr_t>(a) & ~uintptr_t(127)); l < e;
               l += 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(l < a ? a : l));
        }
      }
      if (!mbar_wait_warp(tfull, g & 1, abort_flag, p.status, DEV_TIMEOUT_TMEM_FULL) ||
          !mbar_wait_warp(&sfull[buf], (g >> 1) & 1, abort_flag, p.status, DEV_TIMEOUT_TMEM_FULL))
        break;
      tc_fence_after();
      // 16-column chunks this warp keeps: none past the inputs, none wholly above the diagonal
      int n_ch = 0;
      if (it.has_row) {
        if (it.transposed) {
          const int cols = n_inputs - S * kBlk;  // output rows b of the column tile (a multiple of 16)
          n_ch = cols >= kBlk ? kBlk / kChunk : cols / kChunk;
        } else {
          const int row0 = R * kBlk + warp * 32;
          n_ch = row0 >= n_inputs ? 0 : R == S ? (warp * 32 + 31) / kChunk + 1 : kBlk / kChunk;
        }
      }
      {
        uint4* srow = reinterpret_cast<uint4*>(staging + r_own * kBlk);
        const int sw = staging_swizzle(r_own);
        uint4* hrow = reinterpret_cast<uint4*>(im_hi + r_own * G::kImHiCols);
        for (int ch = 0; ch < n_ch; ++ch) {
          // D = [Re | Im] of tile columns 0-63, then of 64-127
          const uint32_t re_col = static_cast<uint32_t>(kChunk * ch + (ch >= kBlk / (2 * kChunk) ? kHalf : 0));
          uint32_t re[16], nim[16];
          tmem_ld16(taddr + re_col, re);
          tmem_ld16(taddr + re_col + kHalf, nim);
          tmem_ld_wait();
          // 16-byte piece q of a chunk holds columns 2q, 2q + 1, 8 + 2q, 9 + 2q (phase 2's order)
          if (ch < STASH) {
            tmem_st16(taddr + kStashCol + kChunk * ch, nim);
          } else {
#pragma unroll
            for (int q = 0; q < kChunk / 4; ++q)
              hrow[((kChunk * (ch - STASH)) / 4 + q) ^ sw] =
                  make_uint4(nim[2 * q], nim[2 * q + 1], nim[8 + 2 * q], nim[9 + 2 * q]);
          }
#pragma unroll
          for (int q = 0; q < kChunk / 4; ++q)
            srow[((kChunk * ch) / 4 + q) ^ sw] = make_uint4(re[2 * q], re[2 * q + 1], re[8 + 2 * q], re[9 + 2 * q]);
        }
      }
      // W = n_re - 8 P_a - 8 P_b + 128 T  +  i (-n_im - 8 Q_a + 8 Q_b): the row's part
      const int2 rs = sums[(buf * 2) * kBlk + r_own];  // (8P, 8Q) of this row's input
      const int2 rc_own = make_int2(t128 - rs.x - (magic ? kMagicBits : 0), -rs.y + (magic ? kMagicBits : 0));
      // the accumulator (columns 0-255) is free once its loads have landed; the stash stores
      // (columns 256 .. 256 + 16 STASH - 1) need only land before phase 2 reads them
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (rank != 0)
          bulk_copy_to_cluster(sink_even, token, kSignalBytes, tempty_even);
        else if (warp == 0)
          mbar_expect_tx(tempty, kEpiWarps * kSignalBytes);
        else
          mbar_arrive(tempty);
      }
      // phase 2 reads stash lanes that other threads of the warp stored
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      tc_fence_after();
      const int2* cs = sums + (buf * 2 + 1) * kBlk;  // (8P, 8Q) of the columns, both halves
      if (it.transposed) {
        // V[S*128 + b][R*128 + a] = conj(W[a][b]) = (W.re, -W.im)
        const int2 rc = rc_own;
        const int a_col = R * kBlk + r_own;
        const int sw = staging_swizzle(r_own);
        for (int ch = 0; ch < n_ch; ++ch) {
          uint32_t im[16];
          if (ch < STASH) tmem_ld16(taddr + kStashCol + kChunk * ch, im);
          uint32_t re[16];
#pragma unroll
          for (int q = 0; q < kChunk / 4; ++q) {
            const uint4 v = *reinterpret_cast<const uint4*>(staging + r_own * kBlk + ((((kChunk * ch) / 4 + q) ^ sw) << 2));
            re[2 * q] = v.x, re[2 * q + 1] = v.y, re[8 + 2 * q] = v.z, re[9 + 2 * q] = v.w;
          }
          if (ch < STASH) {
            tmem_ld_wait();
          } else {
#pragma unroll
            for (int q = 0; q < kChunk / 4; ++q) {
              const uint4 v = *reinterpret_cast<const uint4*>(im_hi + r_own * G::kImHiCols +
                                                              ((((kChunk * (ch - STASH)) / 4 + q) ^ sw) << 2));
              im[2 * q] = v.x, im[2 * q + 1] = v.y, im[8 + 2 * q] = v.z, im[9 + 2 * q] = v.w;
            }
          }
#pragma unroll
          for (int k = 0; k < kChunk; ++k) {
            const int b = kChunk * ch + k, i = S * kBlk + b;
            const int2 s = cs[b];
            int nr, ni;
            if (magic) {
              nr = __float_as_int(fmaf(__uint_as_float(re[k]), 262144.0f, kMagic));
              ni = __float_as_int(fmaf(__uint_as_float(im[k]), 262144.0f, kMagic));
            } else {
              nr = __float2int_rn(__uint_as_float(re[k]) * 262144.0f);
              ni = __float2int_rn(__uint_as_float(im[k]) * 262144.0f);
            }
            int2 v = make_int2(nr + rc.x - s.x, ni - rc.y - s.y);
            int2* dst = out_c + (int64_t)i * (i + 1) / 2 + a_col;
            if (p.accumulate) {
              const int2 o = *dst;
              v.x += o.x;
              v.y += o.y;
            }
            *dst = v;
          }
        }
      } else {
        // thread (rg, q) = (lane / 4, lane % 4) owns rows 32 warp + rg + 8m (m = 0..3) and, in each
        // 16-column chunk, columns 2q, 2q + 1, 8 + 2q, 9 + 2q
        const int q4 = lane & 3, rg = lane >> 2;
        for (int ch = 0; ch < n_ch; ++ch) {
          const bool stashed = ch < STASH;  // Im of this chunk in tensor memory (else shared memory)
          const int jc = kChunk * ch + 2 * q4;  // this thread's first column in the tile
          const int4 s0 = *reinterpret_cast<const int4*>(cs + jc);  // (8P, 8Q) of columns jc, jc + 1
          const int4 s1 = *reinterpret_cast<const int4*>(cs + jc + 8);
          const int sp[4] = {s0.x, s0.z, s1.x, s1.z}, sq[4] = {s0.y, s0.w, s1.y, s1.w};
#pragma unroll 1
          for (int hh = 0; hh < 2; ++hh) {  // rows 0-15, then 16-31 of the warp
            uint32_t im[8];  // stashed: [4j + 2h + e]: column 8j + 2q + e of row 16 hh + rg + 8h
            if (stashed) {
              tmem_ld_16x256b_x2(taddr + (static_cast<uint32_t>(16 * hh) << 16) + kStashCol + kChunk * ch, im);
              tmem_ld_wait();
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int m = 2 * hh + h;
              const int2 rc = make_int2(__shfl_sync(0xFFFFFFFFu, rc_own.x, rg + 8 * m),
                                        __shfl_sync(0xFFFFFFFFu, rc_own.y, rg + 8 * m));
              const int rr = warp * 32 + rg + 8 * m, i = R * kBlk + rr;
              const int last = R == S ? rr : kBlk - 1;  // last column of the row in the tile
              if (i >= n_inputs || jc > last) continue;
              const int piece = ((kChunk * ch) >> 2) + q4;
              const uint4 re4 = *reinterpret_cast<const uint4*>(staging + rr * kBlk + ((piece ^ staging_swizzle(rr)) << 2));
              uint32_t vi[4];
              if (stashed) {
                vi[0] = im[2 * h], vi[1] = im[2 * h + 1], vi[2] = im[4 + 2 * h], vi[3] = im[5 + 2 * h];
              } else {
                const uint4 im4 = *reinterpret_cast<const uint4*>(
                    im_hi + rr * G::kImHiCols + (((piece - 4 * STASH) ^ staging_swizzle(rr)) << 2));
                vi[0] = im4.x, vi[1] = im4.y, vi[2] = im4.z, vi[3] = im4.w;
              }
              const uint32_t vr[4] = {re4.x, re4.y, re4.z, re4.w};
              int2 v[4];  // columns jc, jc + 1, jc + 8, jc + 9
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                int nr, ni;
                if (magic) {
                  nr = __float_as_int(fmaf(__uint_as_float(vr[k]), 262144.0f, kMagic));
                  ni = __float_as_int(fmaf(__uint_as_float(vi[k]), 262144.0f, kMagic));
                } else {
                  nr = __float2int_rn(__uint_as_float(vr[k]) * 262144.0f);
                  ni = __float2int_rn(__uint_as_float(vi[k]) * 262144.0f);
                }
                v[k] = make_int2(nr + rc.x - sp[k], -ni + rc.y + sq[k]);
              }
              int2* row_out = out_c + (int64_t)i * (i + 1) / 2 + S * kBlk;
#pragma unroll
              for (int jj = 0; jj < 2; ++jj) {
                const int j0 = jc + 8 * jj;
                if (j0 > last) continue;
                int2* dst = row_out + j0;
                const int nv = j0 + 1 <= last ? 2 : 1;
                if (nv == 2 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
                  int4 w = make_int4(v[2 * jj].x, v[2 * jj].y, v[2 * jj + 1].x, v[2 * jj + 1].y);
                  if (p.accumulate) {
                    const int4 o = *reinterpret_cast<const int4*>(dst);
                    w = make_int4(w.x + o.x, w.y + o.y, w.z + o.z, w.w + o.w);
                  }
                  *reinterpret_cast<int4*>(dst) = w;
                } else {
#pragma unroll
                  for (int e = 0; e < 2; ++e) {
                    if (e < nv) {
                      int2 w = v[2 * jj + e];
                      if (p.accumulate) {
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
        }
      }
      // the input sums are free, in this CTA and (for the column sums it receives) in the other
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&sempty[buf]);
        mbar_arrive_cluster(sempty_peer + 8u * static_cast<uint32_t>(buf));
      }
    }
  }

  tc_fence_before();
  cluster_sync();  // no remote arrive, sum or MMA of either CTA is still in flight
  if (*abort_flag) {
    // a pipeline that gave up may leave signal copies between the CTAs in flight: let them land
    const uint64_t t_end = global_ns() + 20000;
    while (global_ns() < t_end) {
    }
  }
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc_pair(tmem, kTmemCols);
  }
}

template <int KT, int RAW, int DEC, int STASH>
cudaError_t launch_pair(const CUtensorMap& map_a, const CUtensorMap& map_b, const PParams& p, int n_items,
                        int num_sms, cudaStream_t stream) {
  using G = PGeom<KT, RAW, DEC, STASH>;
  auto kern = xcorr_tc_fused_pair_kernel<KT, RAW, DEC, STASH>;
  static int attr_device = -1, max_clusters = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_device != dev) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmem);
    if (e != cudaSuccess) return e;
    // pairs of SMs that can hold one CTA each at the same time
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * 1024);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = G::kSmem;
    e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (max_clusters < 1) return cudaErrorLaunchOutOfResources;
    attr_device = dev;
  }
  int n_cl = max_clusters < num_sms / 2 ? max_clusters : num_sms / 2;
  if (n_cl < 1) n_cl = 1;
  if (n_items < n_cl) n_cl = n_items;
  kern<<<2 * n_cl, kThreads, G::kSmem, stream>>>(map_a, map_b, p);
  return cudaGetLastError();
}

}  // namespace

// The pair shapes: 96 samples with 2 raw + 3 decoded stages (Im of half the tile kept in tensor
// memory), 128 with 2 + 2 (all of Im in tensor memory), 128 with 2 + 3 (half).
int fused_pair_stage_samples(int variant) { return variant == 0 ? 96 : 128; }

cudaError_t launch_xcorr_tc_fused_pair_ci4(const uint8_t* in, int row_chans, int variant, int n_time, int n_chan,
                                           int n_inputs, int2* out, bool accumulate, int* status, int num_sms,
                                           cudaStream_t stream) {
  const int nb = (n_inputs + kBlk - 1) / kBlk;
  const int kt = fused_pair_stage_samples(variant);
  if (n_time <= 0 || n_inputs % 16 != 0 || reinterpret_cast<uintptr_t>(in) % 16 != 0 ||
      kFusedWindowCI4 % kt != 0)
    return cudaErrorInvalidValue;
  PParams p{};
  p.n_chan = n_chan;
  p.n_inputs = n_inputs;
  p.nb = nb;
  p.n_entries = pair_entries(nb);
  p.n_pairs = (int64_t)n_inputs * (n_inputs + 1) / 2;
  p.out = out;
  p.status = status;
  p.one = 1u;
  const int64_t items = (int64_t)n_chan * p.n_entries;
  if (items > 0x7FFFFFFF) return cudaErrorInvalidValue;
  CUtensorMap map_a, map_b;
  if (row_chans < n_chan ||
      !encode_raw_ci4_tmap(&map_a, in, n_inputs, n_chan, row_chans, n_time, kt, nullptr, kBlk) ||
      !encode_raw_ci4_tmap(&map_b, in, n_inputs, n_chan, row_chans, n_time, kt, nullptr, kHalf))
    return cudaErrorInvalidValue;
  // one exactly-summed block per launch; later blocks add into the first
  for (int t0 = 0; t0 < n_time; t0 += kFusedWindowCI4) {
    const int len = n_time - t0 < kFusedWindowCI4 ? n_time - t0 : kFusedWindowCI4;
    p.t0 = t0;
    p.n_kt = (len + kt - 1) / kt;
    p.accumulate = (accumulate || t0 > 0) ? 1 : 0;
    cudaError_t e;
    switch (variant) {
      case 0: e = launch_pair<96, 2, 3, 4>(map_a, map_b, p, static_cast<int>(items), num_sms, stream); break;
      case 1: e = launch_pair<128, 2, 2, 8>(map_a, map_b, p, static_cast<int>(items), num_sms, stream); break;
      default: e = launch_pair<128, 2, 3, 4>(map_a, map_b, p, static_cast<int>(items), num_sms, stream); break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace xc
