// xcorr_tc.cu -- the X-stage on the Blackwell tensor cores (tcgen05).
//
// For each channel c the X-stage is the complex rank-K update
//     V = sum_t x_t x_t^H,  x_t = xr_t + j xi_t  (Sec. 1 and Sec. 2.1; Eq. 1
// counts the N_i (N_i + 1) / 2 pairs), which splits into real products:
//     Re V = Xr Xr^T + Xi Xi^T,   Im V = Xi Xr^T - Xr Xi^T
// with X[i][t] the N_i x K matrix of one channel's samples.
//
// The operands are planes of tensor-core numbers, [channel][plane][t][input]:
//   * 4-bit samples: two E4M3 planes (re, im); every code in [-8, 7] is exact;
//   * int8 samples:  two BF16 planes; every int8 value is exact;
//   * float samples: six BF16 planes of integer digits.  Per input and time
//     window of W samples each component is quantised against the window's
//     largest magnitude 2^E to a 23-bit integer M = d0 2^16 + d1 2^8 + d2
//     with balanced digits |d_p| <= 128 (exact BF16 values); a product of two
//     components is the sum of the digit products d_p d_q 2^(-8(p+q)) with
//     p + q <= 2 (the dropped ones are below 2^-23 of the largest product).
// The K axis runs over (time window, plane pair, stage): for 4-bit and int8
// input a single pair (the re/im planes against themselves), for float input
// the six digit pairs (p, q).  Each (window, pair) block is accumulated in
// FP32 tensor memory and drained on its own: every partial sum of a block is
// an integer of magnitude below 2^24 (at most 128, 32768 or 2 * 2^14 per
// sample for 4-bit, int8 and digit products), so it is exact -- which matters
// because the tensor core truncates each accumulation toward zero -- and the
// drain converts it exactly to int32, or scales it by 2^(E_i + E_j - 12 -
// 8(p + q)) and adds it (rounded to nearest) into a float accumulator.
//
// The input triangle is cut into 128 x 128 tile pairs (I >= J); a persistent
// CTA walks a static list of (channel, I, J) items, channel-major, so the
// CTAs in flight share the channels' planes in L2.  Per stage TMA brings the
// four tiles Xr_p(I), Xi_p(I), Xr_q(J), Xi_q(J) (two when I == J and p == q)
// into a shared-memory ring as MN-major operands (the transpose of the corner
// turn happens in the operand fetch), and one thread issues, per MMA step,
// three MMAs into an FP32 accumulator of 256 TMEM columns holding [Re | -Im]:
//     [Re | -Im] += Xr_I [Xr_J | Xi_J]^T       (M = 128, N = 256)
//     Re         += Xi_I Xi_J^T                (N = 128)
//     -Im        += (-Xi_I) Xr_J^T             (N = 128, negate-A bit)
// Two accumulator buffers (512 columns) let the drain of one block overlap the
// MMAs of the next.
//
// Warp roles (320 threads, one CTA per SM): warps 0-7 drain TMEM -- thread =
// accumulator row, warps w and w + 4 take the two 64-column halves of the same
// 32 rows -- adding every block into running sums held in registers, and
// write the finished tile once through a shared-memory transpose that makes
// the global stores row-contiguous; warp 8 is the TMA producer; warp 9
// allocates TMEM and issues the MMAs.  Every wait is bounded (sm103_ptx.cuh).
#include <cstring>
#include <type_traits>

#include "sm103_ptx.cuh"
#include "xcorr_internal.h"

namespace xc {
namespace {

constexpr int kBlk = 128;          // inputs per tile side
constexpr int kEpiWarps = 8;       // two per TMEM lane quarter, 64 columns each
constexpr int kThreads = 320;
constexpr int kProducerWarp = 8;
constexpr int kMmaWarp = 9;
constexpr int kCols = 64;          // tile columns held per epilogue thread (its row)
constexpr int kChunk = 8;          // columns per shared-memory transpose step
constexpr int kPitch = kChunk + 1; // 8-byte words per staged row
constexpr int kAccCols = 256;      // [Re | -Im]
constexpr uint32_t kTmemCols = 512;
constexpr int kStagingBytes = kEpiWarps * 32 * kPitch * 8;
constexpr int kBarrierBytes = 256;

// Stage shape of variant v: stage bytes 64 KB x 3, 48 KB x 4 or 32 KB x 6.
constexpr int stage_rows_of(int v, int esize) { return (v == 0 ? 128 : v == 1 ? 96 : 64) / esize; }
constexpr int stages_of(int v) { return v == 0 ? 3 : v == 1 ? 4 : 6; }

template <int ESIZE, int KT, int STAGES>
struct Geometry {
  static constexpr int kChunksPerTile = kBlk * ESIZE / 128;  // 128-byte MN chunks
  static constexpr int kChunkBytes = KT * 128;               // one chunk: KT rows of 128 B
  static constexpr int kTileBytes = kChunksPerTile * kChunkBytes;
  static constexpr int kStageBytes = 4 * kTileBytes;
  static constexpr int kMmaK = 32 / ESIZE;                   // K of one MMA (rows)
  static constexpr int kSteps = KT / kMmaK;
  static constexpr int kSmemBytes = 1024 + STAGES * kStageBytes + kStagingBytes + kBarrierBytes;
  static_assert(KT % kMmaK == 0, "stage must hold whole MMA steps");
  static_assert(KT % 8 == 0, "swizzle atoms are 8 rows");
  static_assert(kSmemBytes <= 232448, "shared memory budget");
};

struct TcParams {
  int chan0, n_chan, n_inputs, n_tile_pairs;
  int n_kt;           // stages along time
  int n_pairs_k;      // plane pairs on the K axis
  int spw;            // stages per time window
  int n_tw;           // time windows
  int planes_per_chan;
  int64_t n_pairs;
  int accumulate_first;  // the first block adds into out (else it stores)
  void* out;             // int2 or float2 [C][P]
  int* status;
  const int16_t* exps;   // float input: window exponents [C][exp_windows][ni_pad]
  int exp_windows, ni_pad;
  int8_t pair_p[8], pair_q[8];  // digit indices of each plane pair
  // batch mode: items (subarray, channel, I, J), longest first
  const SubDescHost* subs;
  const uint4* items;
  int n_batch_items;
};

// What one work item (a tile pair of one channel) needs.
struct ItemView {
  const CUtensorMap* tmap;
  int zc;          // plane index of the item's channel, first plane
  int chan;        // channel (single mode: within the plan)
  int I, J;        // tile pair
  int n_kt, n_tw;  // stages, windows
  int n_inputs;
  uint2* out_c;    // the channel's packed triangle
};

__device__ __forceinline__ void tile_pair(int p, int& I, int& J) {
  int i = static_cast<int>((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  I = i;
  J = p - i * (i + 1) / 2;
}

template <bool BATCH>
__device__ __forceinline__ void view_item(const TcParams& p, const CUtensorMap* tmap0, int item, ItemView& v) {
  if (BATCH) {
    const uint4 it = p.items[item];
    const SubDescHost& d = p.subs[it.x];
    v.tmap = &d.tmap;
    v.chan = static_cast<int>(it.y);
    v.zc = 2 * v.chan;
    v.I = static_cast<int>(it.z);
    v.J = static_cast<int>(it.w);
    v.n_kt = d.n_kt;
    v.n_tw = d.n_tw;
    v.n_inputs = d.n_inputs;
    v.out_c = static_cast<uint2*>(d.out) + (int64_t)v.chan * d.n_pairs;
  } else {
    const int cl = item / p.n_tile_pairs;
    tile_pair(item - cl * p.n_tile_pairs, v.I, v.J);
    v.tmap = tmap0;
    v.chan = p.chan0 + cl;
    v.zc = v.chan * p.planes_per_chan;
    v.n_kt = p.n_kt;
    v.n_tw = p.n_tw;
    v.n_inputs = p.n_inputs;
    v.out_c = static_cast<uint2*>(p.out) + (int64_t)v.chan * p.n_pairs;
  }
}

template <int ESIZE>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (ESIZE == 1)
    mma_f8f6f4(d, a, b, id, acc);
  else
    mma_f16(d, a, b, id, acc);
}

template <int ESIZE, int KT, int STAGES, bool FLOAT_OUT, bool BATCH>
__global__ void __launch_bounds__(kThreads, 1)
    xcorr_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TcParams p) {
  using G = Geometry<ESIZE, KT, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stages = smem;
  uint2* staging = reinterpret_cast<uint2*>(smem + STAGES * G::kStageBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * G::kStageBytes + kStagingBytes);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* mma_done = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
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

  const int n_items = BATCH ? p.n_batch_items : p.n_chan * p.n_tile_pairs;

  if (warp == kProducerWarp) {
    if (lane == 0) {
      if (!BATCH) prefetch_tmap(&tmap);
      int s = 0;
      uint32_t ph = 0, filled = 0, fill_parity[STAGES] = {};
      bool ok = true;
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
        ItemView v;
        view_item<BATCH>(p, &tmap, item, v);
        const int zc = v.zc, I = v.I, J = v.J;
        const int half = p.planes_per_chan / 2;  // re planes, then im planes
        const int n_blocks = v.n_tw * p.n_pairs_k;  // drained blocks: (window, pair)
        for (int blk = 0; ok && blk < n_blocks; ++blk) {
          const int w = blk / p.n_pairs_k, pk = blk - w * p.n_pairs_k;
          const int pp = p.pair_p[pk], pq = p.pair_q[pk];
          const bool shared = (I == J) && (pp == pq);
          const int tb1 = min(v.n_kt, (w + 1) * p.spw);
        for (int tb = w * p.spw; tb < tb1; ++tb) {
          const int t0 = tb * KT;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, p.status, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          uint8_t* st = stages + s * G::kStageBytes;
          mbar_expect_tx(&full[s], (shared ? 2 : 4) * G::kTileBytes);
#pragma unroll
          for (int ch = 0; ch < G::kChunksPerTile; ++ch) {
            const int xi = I * kBlk + ch * (128 / ESIZE), xj = J * kBlk + ch * (128 / ESIZE);
            tma_load_3d(st + ch * G::kChunkBytes, v.tmap, &full[s], xi, t0, zc + pp);
            tma_load_3d(st + G::kTileBytes + ch * G::kChunkBytes, v.tmap, &full[s], xi, t0, zc + half + pp);
            if (!shared) {
              tma_load_3d(st + 2 * G::kTileBytes + ch * G::kChunkBytes, v.tmap, &full[s], xj, t0, zc + pq);
              tma_load_3d(st + 3 * G::kTileBytes + ch * G::kChunkBytes, v.tmap, &full[s], xj, t0, zc + half + pq);
            }
          }
          fill_parity[s] = ph;
          filled |= 1u << s;
          if (++s == STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
        }
      }
      // Let every copy this CTA issued land before the CTA can exit.
      volatile int never = 0;
      for (int q = 0; q < STAGES; ++q)
        if (filled & (1u << q)) mbar_wait(&full[q], fill_parity[q], &never, p.status, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      const uint32_t type = ESIZE == 1 ? kTypeE4M3 : kTypeBF16;
      const uint32_t id256 = instr_desc(type, true, 128, 256, false);
      const uint32_t id128 = instr_desc(type, true, 128, 128, false);
      const uint32_t id128n = instr_desc(type, true, 128, 128, true);
      constexpr uint32_t kLbo = G::kChunkBytes;  // distance between 128-byte M/N chunks
      int s = 0;
      uint32_t ph = 0;
      int g = 0;  // windows processed by this CTA
      bool ok = true;
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
        ItemView v;
        view_item<BATCH>(p, &tmap, item, v);
        const int I = v.I, J = v.J;
        const int n_blocks = v.n_tw * p.n_pairs_k;
        for (int blk = 0; ok && blk < n_blocks; ++blk, ++g) {
          const int w = blk / p.n_pairs_k, pk = blk - w * p.n_pairs_k;
          const bool shared = (I == J) && (p.pair_p[pk] == p.pair_q[pk]);
          const int buf = g & 1;
          const uint32_t use = static_cast<uint32_t>(g >> 1);
          if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, abort_flag, p.status, DEV_TIMEOUT_TMEM_EMPTY)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + static_cast<uint32_t>(buf * kAccCols);
          const int kb0 = w * p.spw;
          const int kb1 = min(v.n_kt, kb0 + p.spw);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&full[s], ph, abort_flag, p.status, DEV_TIMEOUT_FULL)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_r = smem_u32(stages + s * G::kStageBytes);
            const uint32_t a_i = a_r + G::kTileBytes;
            const uint32_t b_r = shared ? a_r : a_r + 2 * G::kTileBytes;
            const uint32_t b_i = b_r + G::kTileBytes;
#pragma unroll
            for (int k = 0; k < G::kSteps; ++k) {
              const uint32_t off = static_cast<uint32_t>(k * G::kMmaK * 128);  // kMmaK rows of 128 B
              const uint32_t first = (kb == kb0 && k == 0) ? 1u : 0u;
              mma<ESIZE>(d, smem_desc_sw128(a_r + off, kLbo, 1024), smem_desc_sw128(b_r + off, kLbo, 1024),
                         id256, first ^ 1u);
              mma<ESIZE>(d, smem_desc_sw128(a_i + off, kLbo, 1024), smem_desc_sw128(b_i + off, kLbo, 1024),
                         id128, 1u);
              mma<ESIZE>(d + 128, smem_desc_sw128(a_i + off, kLbo, 1024),
                         smem_desc_sw128(b_r + off, kLbo, 1024), id128n, 1u);
            }
            mma_commit(&empty[s]);
            if (++s == STAGES) {
              s = 0;
              ph ^= 1u;
            }
          }
          if (ok) mma_commit(&tfull[buf]);
        }
      }
      // Wait (bounded) until every MMA this thread issued has completed.
      volatile int never = 0;
      mma_commit(mma_done);
      mbar_wait(mma_done, 0, &never, p.status, DEV_TIMEOUT_DRAIN);
    }
  } else {
    // Epilogue: warp w drains TMEM lanes 32 (w % 4) .. + 31 (tile rows),
    // columns 64 (w / 4) .. + 63; each thread keeps its row's running sums.
    using Acc = typename std::conditional<FLOAT_OUT, float, int>::type;
    uint2* stage_rows = staging + warp * 32 * kPitch;
    const int quarter = warp & 3, colh = warp >> 2;
    int g = 0;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
      ItemView v;
      view_item<BATCH>(p, &tmap, item, v);
      const int n_inputs = v.n_inputs;
      const int n_blocks = v.n_tw * p.n_pairs_k;
      uint2* out_c = v.out_c;
      const int row0 = v.I * kBlk + quarter * 32;  // first global input row of this warp
      const int col0 = v.J * kBlk + colh * kCols;  // first global input column of this warp
      const bool live = (row0 < n_inputs) && (col0 <= row0 + 31) && (col0 < n_inputs);
      Acc acc_re[kCols], acc_im[kCols];
#pragma unroll
      for (int q = 0; q < kCols; ++q) acc_re[q] = acc_im[q] = Acc(0);
      for (int blk = 0; blk < n_blocks; ++blk, ++g) {
        const int buf = g & 1;
        const uint32_t use = static_cast<uint32_t>(g >> 1);
        if (!mbar_wait_warp(&tfull[buf], use & 1u, abort_flag, p.status, DEV_TIMEOUT_TMEM_FULL)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // float input: this block's scale 2^k, k = E_i + E_j - 12 - 8(p + q); the row's part here
        const int16_t* exps_w = nullptr;
        int row_k = 0;
        bool row_bad = false;
        if (FLOAT_OUT) {
          const int w = blk / p.n_pairs_k, pk = blk - w * p.n_pairs_k;
          exps_w = p.exps + ((int64_t)v.chan * p.exp_windows + w) * p.ni_pad;
          const int i_row = min(row0 + lane, n_inputs - 1);
          const int e_row = exps_w[i_row];
          row_k = e_row - 12 - 8 * (p.pair_p[pk] + p.pair_q[pk]);
          row_bad = e_row == kExpNonFinite;
        }
        const uint32_t taddr =
            tmem + (static_cast<uint32_t>(quarter * 32) << 16) + buf * kAccCols + colh * kCols;
        if (FLOAT_OUT) {
          // exact integer block sums times an exact power of two 2^k, applied as two factors
          // 2^(k >> 1) and 2^(k - (k >> 1)) so that neither leaves the float range
          // (k <= 242): a sum whose product overflows becomes +-inf, a zero sum stays zero, and
          // a product below the normal range rounds once, as a subnormal.  A window with a
          // non-finite sample makes its blocks NaN.  The column exponents of 8 columns come in
          // one 16-byte load (padding entries are zero).
#pragma unroll
          for (int k = 0; k < kCols / 8; ++k) {
            uint32_t re[8], nim[8];
            tmem_ld8(taddr + 8 * k, re);
            tmem_ld8(taddr + 128 + 8 * k, nim);
            tmem_ld_wait();
            if (live) {
              const uint4 e8 = *reinterpret_cast<const uint4*>(exps_w + col0 + 8 * k);
              const uint32_t ew[4] = {e8.x, e8.y, e8.z, e8.w};
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const int ej = static_cast<int16_t>((ew[q >> 1] >> (16 * (q & 1))) & 0xFFFFu);
                // below -298 a block's contribution rounds to zero either way
                const int kk = max(row_k + ej, -298);
                const float f1 = (row_bad || ej == kExpNonFinite) ? __int_as_float(0x7FC00000) : pow2i(kk >> 1);
                const float f2 = pow2i(kk - (kk >> 1));
                acc_re[8 * k + q] += (__uint_as_float(re[q]) * f1) * f2;
                acc_im[8 * k + q] -= (__uint_as_float(nim[q]) * f1) * f2;
              }
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < kCols / 8; ++k) {
            uint32_t re[8], nim[8];
            tmem_ld8(taddr + 8 * k, re);
            tmem_ld8(taddr + 128 + 8 * k, nim);
            tmem_ld_wait();
            if (live) {
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                acc_re[8 * k + q] += __float2int_rn(__uint_as_float(re[q]));
                acc_im[8 * k + q] -= __float2int_rn(__uint_as_float(nim[q]));
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
      }
      if (!ok || !live) continue;
      // Write the finished tile rows.  Per 8-column step a quarter-warp writes
      // 8 consecutive pairs of one row (64 bytes); when adding into earlier
      // integrations all loads of the lane are issued before its stores.
      const bool add = p.accumulate_first != 0;
      const int sub = lane >> 3, col = lane & 7;
#pragma unroll
      for (int ch = 0; ch < kCols / kChunk; ++ch) {
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
          Acc vr = acc_re[ch * kChunk + q], vi = acc_im[ch * kChunk + q];
          stage_rows[lane * kPitch + q] = FLOAT_OUT ? make_uint2(__float_as_uint(vr), __float_as_uint(vi))
                                                    : make_uint2(static_cast<uint32_t>(vr), static_cast<uint32_t>(vi));
        }
        __syncwarp();
        const int j = col0 + ch * kChunk + col;
        uint32_t valid = 0;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int i = row0 + 4 * r + sub;
          if (i < n_inputs && j <= i) valid |= 1u << r;
        }
        uint2 old[8];
        if (add) {  // (continuing an integration: rarer, kept out of the register budget)
#pragma unroll 1
          for (int r = 0; r < 8; ++r) {
            const int i = row0 + 4 * r + sub;
            old[r] = (valid >> r) & 1u ? out_c[(int64_t)i * (i + 1) / 2 + j] : make_uint2(0u, 0u);
          }
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          if ((valid >> r) & 1u) {
            const int rr = 4 * r + sub;
            const int i = row0 + rr;
            uint2 v = stage_rows[rr * kPitch + col];
            if (add) {
              if (FLOAT_OUT) {
                v.x = __float_as_uint(__uint_as_float(v.x) + __uint_as_float(old[r].x));
                v.y = __float_as_uint(__uint_as_float(v.y) + __uint_as_float(old[r].y));
              } else {
                v.x += old[r].x;
                v.y += old[r].y;
              }
            }
            out_c[(int64_t)i * (i + 1) / 2 + j] = v;
          }
        }
        __syncwarp();
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// One instantiation per (operand type, stage variant, output type) in use.
template <int ESIZE, int V, bool FLOAT_OUT, bool BATCH = false>
cudaError_t launch_variant(const CUtensorMap* tmap, const TcParams& p, int grid, cudaStream_t stream) {
  constexpr int KT = stage_rows_of(V, ESIZE), S = stages_of(V);
  using G = Geometry<ESIZE, KT, S>;
  auto kern = xcorr_tc_kernel<ESIZE, KT, S, FLOAT_OUT, BATCH>;
  static int attr_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_device != dev) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmemBytes);
    if (e != cudaSuccess) return e;
    attr_device = dev;
  }
  kern<<<grid, kThreads, G::kSmemBytes, stream>>>(*tmap, p);
  return cudaGetLastError();
}

}  // namespace

int tc_stage_samples(int elem_bytes, int variant) { return stage_rows_of(variant, elem_bytes); }

cudaError_t launch_xcorr_tc_batch(const void* subs, const uint4* items, int n_items, int variant, int* status,
                                  int num_sms, cudaStream_t stream) {
  const int kt = stage_rows_of(variant, 1);
  TcParams p{};
  p.n_pairs_k = 1;
  p.spw = kTcWindowCI4 / kt;
  p.planes_per_chan = 2;
  p.accumulate_first = 0;
  p.status = status;
  p.subs = static_cast<const SubDescHost*>(subs);
  p.items = items;
  p.n_batch_items = n_items;
  const int grid = n_items < num_sms ? n_items : num_sms;
  if (grid < 1) return cudaSuccess;
  CUtensorMap unused;
  std::memset(&unused, 0, sizeof(unused));
  switch (variant) {
    case 0: return launch_variant<1, 0, false, true>(&unused, p, grid, stream);
    case 1: return launch_variant<1, 1, false, true>(&unused, p, grid, stream);
    default: return launch_variant<1, 2, false, true>(&unused, p, grid, stream);
  }
}

cudaError_t launch_xcorr_tc(const CUtensorMap* tmap, const TcLaunch& L, cudaStream_t stream) {
  const int nb = (L.n_inputs + kBlk - 1) / kBlk;
  const int kt = stage_rows_of(L.variant, L.elem_bytes);
  TcParams p{};
  p.chan0 = L.chan0;
  p.n_chan = L.n_chan;
  p.n_inputs = L.n_inputs;
  p.n_tile_pairs = nb * (nb + 1) / 2;
  p.n_kt = (L.n_time + kt - 1) / kt;
  p.n_pairs_k = L.n_pairs_k;
  p.spw = L.window_samples / kt;
  p.n_tw = (p.n_kt + p.spw - 1) / p.spw;
  p.planes_per_chan = L.planes_per_chan;
  p.exps = L.exps;
  p.exp_windows = L.exp_windows;
  p.ni_pad = L.ni_pad;
  p.n_pairs = (int64_t)L.n_inputs * (L.n_inputs + 1) / 2;
  p.accumulate_first = L.accumulate ? 1 : 0;
  p.out = L.out;
  p.status = L.status;
  for (int k = 0; k < 8; ++k) {
    p.pair_p[k] = static_cast<int8_t>(k < L.n_pairs_k ? L.pair_p[k] : 0);
    p.pair_q[k] = static_cast<int8_t>(k < L.n_pairs_k ? L.pair_q[k] : 0);
  }
  if (p.spw < 1 || L.window_samples % kt || (L.float_out && !L.exps)) return cudaErrorInvalidValue;
  const int64_t items = (int64_t)L.n_chan * p.n_tile_pairs;
  const int grid = static_cast<int>(items < L.num_sms ? items : L.num_sms);
  if (L.elem_bytes == 1) {
    switch (L.variant) {
      case 0: return launch_variant<1, 0, false>(tmap, p, grid, stream);
      case 1: return launch_variant<1, 1, false>(tmap, p, grid, stream);
      default: return launch_variant<1, 2, false>(tmap, p, grid, stream);
    }
  }
  if (L.float_out) {
    switch (L.variant) {
      case 0: return launch_variant<2, 0, true>(tmap, p, grid, stream);
      case 1: return launch_variant<2, 1, true>(tmap, p, grid, stream);
      default: return launch_variant<2, 2, true>(tmap, p, grid, stream);
    }
  }
  switch (L.variant) {
    case 0: return launch_variant<2, 0, false>(tmap, p, grid, stream);
    case 1: return launch_variant<2, 1, false>(tmap, p, grid, stream);
    default: return launch_variant<2, 2, false>(tmap, p, grid, stream);
  }
}

}  // namespace xc
