// xcorr_tc_fused.cu -- the 4-bit X-stage with the unpack fused into the
// tensor-core kernel.
//
// Same result as xcorr_tc.cu for 4+4-bit input (per channel, the packed lower
// triangle of V = sum_t x_t x_t^H; Sec. 1, Sec. 2.1, Eq. 1), but no E4M3
// planes go through HBM: TMA brings the caller's raw [t][c][i] bytes of a
// 128-input x KT-sample tile into a shared-memory ring (box 128 inputs x 1
// channel x KT samples, 128-byte swizzle), and eight decoder warps turn each
// raw byte into its real and imaginary E4M3 codes at the same offset of two
// operand tiles -- the MN-major 128-byte-swizzled layout the MMA reads (Sec.
// 2.4's unpack, done on chip).
//
// Offset-binary operands.  A 4-bit two's-complement code t in [-8, 7] becomes
// u = t + 8 in [0, 15] by flipping its top bit, and the byte u read as E4M3 is
// exactly u * 2^-9 (codes 0..7 are subnormals m * 2^-9, codes 8..15 are
// (8 + m) * 2^-9).  So the decode is one XOR and a mask per four samples, and
// the MMAs produce sums of u_a u_b.  The true products follow from
//   sum (u_a - 8)(u_b - 8) = sum u_a u_b - 8 S_a - 8 S_b + 64 T,
// which needs the per-input sums S = sum_t u over the block: the decoders
// accumulate them in byte lanes as they go, and the epilogue applies
//   Re V_ab = Re' - 8 (P_a + P_b) + 128 T,   P = S_re + S_im,
//   Im V_ab = Im' - 8 Q_a + 8 Q_b,           Q = S_im - S_re.
// Every partial sum of u_a u_b is an integer multiple of 2^-18 below 2^6
// (|Re'| <= 450 T), exact in the FP32 accumulator for T <= 37,282; a launch
// covers at most 37,248 samples and longer integrations add launches.
//
// Warp roles (448 threads, one CTA per SM): warps 0-3 drain TMEM (one tile
// row per thread) through a shared-memory transpose; warps 4-11 decode and
// sum; warp 12 is the TMA producer (and prefetches into L2 further ahead);
// warp 13 allocates TMEM and issues the three MMAs per 32-sample step into
// [Re | -Im] (double-buffered).  Every wait is bounded (sm103_ptx.cuh).
#include "fused_common.cuh"
#include "sm103_ptx.cuh"
#include "xcorr_internal.h"

namespace xc {
namespace {

using namespace fused;

constexpr int kEpiWarps = 4;
constexpr int kDecWarp0 = 4;
constexpr int kChunk = 16;
constexpr int kPitch = kChunk + 1;
constexpr int kAccCols = 256;  // [Re | -Im]
constexpr uint32_t kTmemCols = 512;
constexpr int kStagingBytes = kEpiWarps * 32 * kPitch * 8;
constexpr int kSumsBytes = 2 * 2 * kBlk * 8;            // [TMEM buffer][I, J][input] (8P, 8Q)
// Every partial sum of u_a u_b is n 2^-18 with 0 <= n <= 450 T (and |n| <= 225 T for Im).
// For T <= kMagicSamples, |n| < 2^22 and n + 1.5 2^23 is exact in FP32, so one FFMA
// against that constant turns the accumulator into n (in the low bits of the result).
constexpr int kMagicSamples = 9320;
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;
constexpr int kBarrierBytes = 256;

// Warp roles for DW decoder warps: 0-3 epilogue, 4 .. 3 + DW decoders, then
// the TMA producer and the MMA warp.
template <int DW>
struct Roles {
  static constexpr int kProducerWarp = kDecWarp0 + DW;
  static constexpr int kMmaWarp = kDecWarp0 + DW + 1;
  static constexpr int kThreads = (kDecWarp0 + DW + 2) * 32;
  static constexpr int kDecThreads = DW * 32;
  static constexpr int kTileThreads = DW * 16;                 // off the diagonal: one tile per half
  static constexpr int kScratchBytes = DW * 8 * 16 * 8;        // [decoder warp][chunk][input] (P, Q)
  static_assert(DW % 2 == 0, "two halves of decoder warps");
};

template <int KT, int RAW, int DEC, int DW>
struct FGeom {
  static constexpr int kTile = KT * kBlk;        // one 128-input x KT-sample tile, raw or decoded
  static constexpr int kRawStage = 2 * kTile;    // raw I, raw J
  static constexpr int kDecStage = 4 * kTile;    // Xr_I, Xi_I, Xr_J, Xi_J
  static constexpr int kSmem = 1024 + RAW * kRawStage + DEC * kDecStage + kStagingBytes + kSumsBytes +
                               Roles<DW>::kScratchBytes + kBarrierBytes;
  // rows per thread and stage off / on the diagonal (8 threads per 128-byte row)
  static constexpr int kRowsOff = KT / (Roles<DW>::kTileThreads / 8);
  static constexpr int kRowsDiag = KT / (Roles<DW>::kDecThreads / 8);
  static_assert(KT % (Roles<DW>::kDecThreads / 8) == 0, "whole rows per decoder thread");
  static constexpr int kSteps = KT / 32;         // MMA steps (32 samples) per stage
  static_assert(KT % 32 == 0, "stage must hold whole MMA steps");
  static_assert(kSmem <= 232448, "shared memory budget");
};

struct FParams {
  int n_chan, n_inputs, n_tile_pairs;
  int t0, t_end;       // samples [t0, t_end) of this launch
  int n_kt;            // stages per tile pair
  int64_t n_pairs;
  int accumulate;      // add into out (else store)
  int2* out;
  int* status;
  uint32_t one;        // 1: a multiplier the compiler cannot fold (see lane_add)
};

// One decoder thread's share of one tile pair: a fixed 16-input chunk L of one
// tile and rows phase, phase + KT/R, ...; R rows per stage.  A raw chunk sits
// at the same swizzled offset as its decoded chunks (TMA and the MMA use the
// same 128-byte swizzle), so the thread reads and writes offset `pos` of each
// row.  Returns the chunk's per-input sums in 16-bit lanes (word e/2, half
// e%2 holds input e); false if a wait gave up.
template <int KT, int RAW, int DEC, int DW, int R>
__device__ __forceinline__ bool decode_item(const FParams& p, const uint8_t* raw, uint8_t* dec, uint64_t* raw_full,
                                            uint64_t* raw_empty, uint64_t* dec_full, uint64_t* dec_empty,
                                            volatile int* abort_flag, int& r, uint32_t& rph, int& d, uint32_t& dph,
                                            int slot, int tp, int lane, uint32_t (&s_re)[8], uint32_t (&s_im)[8]) {
  using G = FGeom<KT, RAW, DEC, DW>;
  constexpr int kStep = KT / R;  // a multiple of 8, so every row of the thread has the same swizzle
  static_assert(kStep % 8 == 0, "row step must keep the swizzle phase");
  const int L = tp & 7, phase = tp >> 3;
  const int pos = (L ^ (phase & 7)) << 4;  // 128-byte swizzle: chunk L of row r sits at chunk L ^ (r % 8)
#pragma unroll
  for (int q = 0; q < 8; ++q) s_re[q] = s_im[q] = 0u;
  for (int tb = 0; tb < p.n_kt; ++tb) {
    if (!mbar_wait_warp(&raw_full[r], rph, abort_flag, p.status, DEV_TIMEOUT_FULL) ||
        !mbar_wait_warp(&dec_empty[d], dph ^ 1u, abort_flag, p.status, DEV_TIMEOUT_EMPTY))
      return false;
    const uint8_t* src = raw + r * G::kRawStage + slot * G::kTile + pos;
    uint8_t* re_t = dec + d * G::kDecStage + (2 * slot) * G::kTile + pos;
    uint8_t* im_t = re_t + G::kTile;
    uint4 v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = *reinterpret_cast<const uint4*>(src + (phase + k * kStep) * 128);
    uint32_t a_re[4] = {0u, 0u, 0u, 0u}, a_im[4] = {0u, 0u, 0u, 0u};  // byte lanes: <= 15 * R <= 120
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
      const int off = (phase + k * kStep) * 128;
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
    // the MMA reads the tiles through the async proxy
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
  return true;
}

template <int KT, int RAW, int DEC, int DW>
__global__ void __launch_bounds__(Roles<DW>::kThreads, 1)
    xcorr_tc_fused_kernel(const __grid_constant__ CUtensorMap raw_map, const __grid_constant__ FParams p) {
  using G = FGeom<KT, RAW, DEC, DW>;
  using W = Roles<DW>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* raw = smem;
  uint8_t* dec = raw + RAW * G::kRawStage;
  int2* staging = reinterpret_cast<int2*>(dec + DEC * G::kDecStage);
  int2* sums = reinterpret_cast<int2*>(reinterpret_cast<uint8_t*>(staging) + kStagingBytes);  // [2][2][128]
  int2* scratch = sums + 2 * 2 * kBlk;                                                           // [8][8][16]
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(scratch + DW * 8 * 16);
  uint64_t* raw_empty = raw_full + RAW;
  uint64_t* dec_full = raw_empty + RAW;
  uint64_t* dec_empty = dec_full + DEC;
  uint64_t* tfull = dec_empty + DEC;
  uint64_t* tempty = tfull + 2;
  uint64_t* sfull = tempty + 2;
  uint64_t* mma_done = sfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < RAW; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], DW);
    }
    for (int s = 0; s < DEC; ++s) {
      mbar_init(&dec_full[s], DW);
      mbar_init(&dec_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
      mbar_init(&sfull[b], 1);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == W::kMmaWarp) tmem_alloc(tslot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int n_items = p.n_chan * p.n_tile_pairs;

  if (warp == W::kProducerWarp) {
    if (lane == 0) {
      constexpr int kAhead = kPrefetchSamples / KT;  // L2 prefetch runs this many stages ahead of the loads
      prefetch_tmap(&raw_map);
      {
        const Item first = item_at(p.n_tile_pairs, blockIdx.x, n_items);
        for (int s = 0; s < kAhead; ++s) prefetch_stage<KT>(&raw_map, p.t0, p.n_kt, first, s);
      }
      int r = 0;
      uint32_t ph = 0, filled = 0, fill_parity[RAW] = {};
      bool ok = true;
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
        const Item it = item_at(p.n_tile_pairs, item, n_items);
        for (int tb = 0; tb < p.n_kt; ++tb) {
          if (tb + kAhead < p.n_kt)
            prefetch_stage<KT>(&raw_map, p.t0, p.n_kt, it, tb + kAhead);
          else
            prefetch_stage<KT>(&raw_map, p.t0, p.n_kt, item_at(p.n_tile_pairs, item + gridDim.x, n_items),
                               tb + kAhead - p.n_kt);
          if (!mbar_wait(&raw_empty[r], ph ^ 1u, abort_flag, p.status, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          uint8_t* st = raw + r * G::kRawStage;
          const int t = p.t0 + tb * KT;
          mbar_expect_tx(&raw_full[r], (it.diag ? 1 : 2) * G::kTile);
          tma_load_3d(st, &raw_map, &raw_full[r], it.I * kBlk, it.c, t);
          if (!it.diag) tma_load_3d(st + G::kTile, &raw_map, &raw_full[r], it.J * kBlk, it.c, t);
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
  } else if (warp >= kDecWarp0 && warp < kDecWarp0 + DW) {
    const int tid = (warp - kDecWarp0) * 32 + lane;
    const int dw = warp - kDecWarp0;
    int r = 0, d = 0, g = 0;
    uint32_t rph = 0, dph = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++g) {
      const Item cur = item_at(p.n_tile_pairs, item, n_items);
      const bool diag = cur.diag;
      uint32_t s_re[8], s_im[8];
      // off the diagonal the first half of the threads take tile I and the second half tile J;
      // on it, all take tile I
      const bool ok_dec =
          diag ? decode_item<KT, RAW, DEC, DW, G::kRowsDiag>(p, raw, dec, raw_full, raw_empty, dec_full, dec_empty,
                                                             abort_flag, r, rph, d, dph, 0, tid, lane, s_re, s_im)
               : decode_item<KT, RAW, DEC, DW, G::kRowsOff>(p, raw, dec, raw_full, raw_empty, dec_full, dec_empty,
                                                            abort_flag, r, rph, d, dph, tid / W::kTileThreads,
                                                            tid % W::kTileThreads, lane, s_re, s_im);
      bool ok = ok_dec;
      // per-input sums of this item: within the warp, lanes L, L+8, L+16, L+24 hold chunk L
      int2 pq[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int sr = ok ? static_cast<int>((s_re[e >> 1] >> (16 * (e & 1))) & 0xFFFFu) : 0;
        const int si = ok ? static_cast<int>((s_im[e >> 1] >> (16 * (e & 1))) & 0xFFFFu) : 0;
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
        for (int e = 0; e < 16; ++e) scratch[(dw * 8 + lane) * 16 + e] = pq[e];
      }
      dec_bar_sync(W::kDecThreads);
      const int buf = g & 1;
      const uint32_t use = static_cast<uint32_t>(g >> 1);
      if (ok) ok = mbar_wait_warp(&tempty[buf], (use & 1u) ^ 1u, abort_flag, p.status, DEV_TIMEOUT_TMEM_EMPTY);
      // thread (slot, e) of the first 256 (128 on the diagonal) sums input e of
      // its tile over the decoder warps that covered that tile
      if (ok && tid < (diag ? 128 : 256)) {
        const int slot = diag ? 0 : tid >> 7, e = tid & 127;
        const int w0 = diag ? 0 : slot * (DW / 2), nw = diag ? DW : DW / 2;
        int2 s = make_int2(0, 0);
        for (int w = w0; w < w0 + nw; ++w) {
          const int2 x = scratch[(w * 8 + (e >> 4)) * 16 + (e & 15)];
          s.x += x.x;
          s.y += x.y;
        }
        sums[(buf * 2 + slot) * kBlk + e] = make_int2(8 * s.x, 8 * s.y);
      }
      if (dec_bar_or(!ok || *abort_flag, W::kDecThreads)) break;
      if (tid == 0) mbar_arrive(&sfull[buf]);
    }
  } else if (warp == W::kMmaWarp) {
    if (lane == 0) {
      const uint32_t id256 = instr_desc(kTypeE4M3, true, 128, 256, false);
      const uint32_t id128 = instr_desc(kTypeE4M3, true, 128, 128, false);
      const uint32_t id128n = instr_desc(kTypeE4M3, true, 128, 128, true);
      constexpr uint32_t kLbo = G::kTile;  // Xr_J and Xi_J are adjacent 128-byte-wide chunks
      int d = 0, g = 0;
      uint32_t dph = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x, ++g) {
        const int c = item / p.n_tile_pairs;
        int I, J;
        tile_pair(item - c * p.n_tile_pairs, I, J);
        const bool diag = (I == J);
        const int buf = g & 1;
        const uint32_t use = static_cast<uint32_t>(g >> 1);
        if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, abort_flag, p.status, DEV_TIMEOUT_TMEM_EMPTY)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + static_cast<uint32_t>(buf * kAccCols);
        for (int tb = 0; tb < p.n_kt; ++tb) {
          if (!mbar_wait(&dec_full[d], dph, abort_flag, p.status, DEV_TIMEOUT_FULL)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_r = smem_u32(dec + d * G::kDecStage);
          const uint32_t a_i = a_r + G::kTile;
          const uint32_t b_r = diag ? a_r : a_r + 2 * G::kTile;
          const uint32_t b_i = b_r + G::kTile;
#pragma unroll
          for (int k = 0; k < G::kSteps; ++k) {
            const uint32_t off = static_cast<uint32_t>(k * 32 * 128);  // 32 rows of 128 B
            const uint32_t first = (tb == 0 && k == 0) ? 1u : 0u;
            mma_f8f6f4(acc, smem_desc_sw128(a_r + off, kLbo, 1024), smem_desc_sw128(b_r + off, kLbo, 1024), id256,
                       first ^ 1u);
            mma_f8f6f4(acc, smem_desc_sw128(a_i + off, kLbo, 1024), smem_desc_sw128(b_i + off, kLbo, 1024), id128,
                       1u);
            mma_f8f6f4(acc + 128, smem_desc_sw128(a_i + off, kLbo, 1024), smem_desc_sw128(b_r + off, kLbo, 1024),
                       id128n, 1u);
          }
          mma_commit(&dec_empty[d]);
          if (++d == DEC) {
            d = 0;
            dph ^= 1u;
          }
        }
        if (ok) mma_commit(&tfull[buf]);
      }
      volatile int never = 0;
      mma_commit(mma_done);
      mbar_wait(mma_done, 0, &never, p.status, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp < kEpiWarps) {
    // Epilogue: warp w drains TMEM lanes 32w .. 32w + 31 (tile rows), 16 columns at a time.
    int2* stage_rows = staging + warp * 32 * kPitch;
    const int half = lane >> 4, col = lane & 15;
    const int t128 = 128 * p.n_kt * KT;  // 128 T over the padded block (padding decodes to u = 8 + 8i)
    int g = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++g) {
      const int c = item / p.n_tile_pairs;
      int I, J;
      tile_pair(item - c * p.n_tile_pairs, I, J);
      int2* out_c = p.out + (int64_t)c * p.n_pairs;
      const int row0 = I * kBlk + warp * 32;
      const int buf = g & 1;
      const uint32_t use = static_cast<uint32_t>(g >> 1);
      if (!mbar_wait_warp(&tfull[buf], use & 1u, abort_flag, p.status, DEV_TIMEOUT_TMEM_FULL) ||
          !mbar_wait_warp(&sfull[buf], use & 1u, abort_flag, p.status, DEV_TIMEOUT_TMEM_FULL))
        break;
      tc_fence_after();
      const int2 rs = sums[(buf * 2) * kBlk + warp * 32 + lane];  // (8P, 8Q) of this row's input
      const int4* cs4 = reinterpret_cast<const int4*>(sums + (buf * 2 + (I == J ? 0 : 1)) * kBlk);
      const bool magic = t128 <= 128 * kMagicSamples;
      // Re = n_re - 8 P_a - 8 P_b + 128 T,  Im = -n_im - 8 Q_a + 8 Q_b
      const int row_re = t128 - rs.x - (magic ? kMagicBits : 0);
      const int row_im = -rs.y + (magic ? kMagicBits : 0);
      const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + buf * kAccCols;
      for (int j0 = 0; j0 < kBlk; j0 += kChunk) {
        const int jfirst = J * kBlk + j0;
        if (jfirst > row0 + 31 || row0 >= p.n_inputs) continue;  // wholly above the diagonal or past the inputs
        uint32_t re[16], nim[16];
        tmem_ld16(taddr + j0, re);
        tmem_ld16(taddr + 128 + j0, nim);
        // the column sums first: the staging stores below would otherwise hold back every load
        int4 s[kChunk / 2];
#pragma unroll
        for (int k = 0; k < kChunk / 2; ++k) s[k] = cs4[j0 / 2 + k];  // (8P, 8Q) of columns 2k, 2k + 1
        tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          re[q] = magic ? __float_as_uint(fmaf(__uint_as_float(re[q]), 262144.0f, kMagic))
                        : static_cast<uint32_t>(__float2int_rn(__uint_as_float(re[q]) * 262144.0f));
          nim[q] = magic ? __float_as_uint(fmaf(__uint_as_float(nim[q]), 262144.0f, kMagic))
                         : static_cast<uint32_t>(__float2int_rn(__uint_as_float(nim[q]) * 262144.0f));
        }
#pragma unroll
        for (int k = 0; k < kChunk / 2; ++k) {
          stage_rows[lane * kPitch + 2 * k] =
              make_int2(static_cast<int>(re[2 * k]) + row_re - s[k].x, -static_cast<int>(nim[2 * k]) + row_im + s[k].y);
          stage_rows[lane * kPitch + 2 * k + 1] = make_int2(static_cast<int>(re[2 * k + 1]) + row_re - s[k].z,
                                                            -static_cast<int>(nim[2 * k + 1]) + row_im + s[k].w);
        }
        __syncwarp();
        // a half-warp writes 16 consecutive pairs of one row: the 16 staged values first, then the stores
        const int j = jfirst + col;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int2 v[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) v[r] = stage_rows[(2 * (8 * h + r) + half) * kPitch + col];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int i = row0 + 2 * (8 * h + r) + half;
            if (i < p.n_inputs && j <= i) {
              int2* dst = out_c + (int64_t)i * (i + 1) / 2 + j;
              if (p.accumulate) {
                const int2 o = *dst;
                v[r].x += o.x;
                v[r].y += o.y;
              }
              *dst = v[r];
            }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == W::kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

template <int KT, int RAW, int DEC, int DW>
cudaError_t launch_fused(const CUtensorMap& raw_map, const FParams& p, int grid, cudaStream_t stream) {
  using G = FGeom<KT, RAW, DEC, DW>;
  auto kern = xcorr_tc_fused_kernel<KT, RAW, DEC, DW>;
  static int attr_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_device != dev) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmem);
    if (e != cudaSuccess) return e;
    attr_device = dev;
  }
  kern<<<grid, Roles<DW>::kThreads, G::kSmem, stream>>>(raw_map, p);
  return cudaGetLastError();
}

}  // namespace

// The fused variants: 128 samples (2 raw + 2 decoded stages), 96 (4 + 2), 64 (6 + 3), all with
// 8 decoder warps, and 96 (4 + 2) with 12; variants 4-6 are the kernel of xcorr_tc_fused_ta.cu
// (A operand in tensor memory), variants 7-9 the kernel of xcorr_tc_fused_pair.cu (CTA pairs
// sharing a column tile).  Deeper raw rings hide more TMA latency, deeper decoded rings more
// decoder jitter, more decoder warps more of the decode's latency.
int fused_stage_samples(int variant) {
  if (variant == 10) return fused_ta_stage_samples(3);
  if (variant >= 7) return fused_pair_stage_samples(variant - 7);
  if (variant >= 4) return fused_ta_stage_samples(variant - 4);
  return variant == 0 ? 128 : variant == 2 ? 64 : 96;
}

int fused_launches(int n_time) { return n_time <= 0 ? 0 : (n_time + kFusedWindowCI4 - 1) / kFusedWindowCI4; }

cudaError_t launch_xcorr_tc_fused_ci4(const uint8_t* in, int row_chans, int variant, int n_time, int n_chan,
                                      int n_inputs, int2* out, bool accumulate, int* status, int num_sms,
                                      cudaStream_t stream) {
  if (variant == 10)  // the tensor-memory-A kernel's small-problem layout
    return launch_xcorr_tc_fused_ta_ci4(in, row_chans, 3, n_time, n_chan, n_inputs, out, accumulate, status,
                                        num_sms, stream);
  if (variant >= 7)
    return launch_xcorr_tc_fused_pair_ci4(in, row_chans, variant - 7, n_time, n_chan, n_inputs, out, accumulate,
                                          status, num_sms, stream);
  if (variant >= 4)
    return launch_xcorr_tc_fused_ta_ci4(in, row_chans, variant - 4, n_time, n_chan, n_inputs, out, accumulate, status,
                                        num_sms, stream);
  const int nb = (n_inputs + kBlk - 1) / kBlk;
  const int kt = fused_stage_samples(variant);
  if (n_time <= 0 || n_inputs % 16 != 0 || reinterpret_cast<uintptr_t>(in) % 16 != 0 ||
      kFusedWindowCI4 % kt != 0)
    return cudaErrorInvalidValue;
  FParams p{};
  p.n_chan = n_chan;
  p.n_inputs = n_inputs;
  p.n_tile_pairs = nb * (nb + 1) / 2;
  p.n_pairs = (int64_t)n_inputs * (n_inputs + 1) / 2;
  p.out = out;
  p.status = status;
  p.one = 1u;
  const int64_t items = (int64_t)n_chan * p.n_tile_pairs;
  const int grid = static_cast<int>(items < num_sms ? items : num_sms);
  CUtensorMap raw_map;
  if (row_chans < n_chan || !encode_raw_ci4_tmap(&raw_map, in, n_inputs, n_chan, row_chans, n_time, kt, nullptr))
    return cudaErrorInvalidValue;
  // one exactly-summed block per launch; later blocks add into the first
  for (int t0 = 0; t0 < n_time; t0 += kFusedWindowCI4) {
    const int len = n_time - t0 < kFusedWindowCI4 ? n_time - t0 : kFusedWindowCI4;
    p.t0 = t0;
    p.t_end = t0 + len;
    p.n_kt = (len + kt - 1) / kt;
    p.accumulate = (accumulate || t0 > 0) ? 1 : 0;
    cudaError_t e;
    switch (variant) {
      case 0: e = launch_fused<128, 2, 2, 8>(raw_map, p, grid, stream); break;
      case 1: e = launch_fused<96, 4, 2, 8>(raw_map, p, grid, stream); break;
      case 2: e = launch_fused<64, 6, 3, 8>(raw_map, p, grid, stream); break;
      default: e = launch_fused<96, 4, 2, 12>(raw_map, p, grid, stream); break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace xc
