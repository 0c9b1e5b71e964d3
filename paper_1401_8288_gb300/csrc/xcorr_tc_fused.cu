// xcorr_tc_fused.cu -- the 4-bit X-stage with the unpack fused into the
// tensor-core kernel.
//
// Same computation as xcorr_tc.cu for 4+4-bit input (per channel, the packed
// lower triangle of V = sum_t x_t x_t^H; Sec. 1, Sec. 2.1, Eq. 1), but no
// E4M3 planes are written to or read from HBM: TMA brings the raw CI4 bytes
// of a 128-input x KT-sample tile straight from the caller's [t][c][i] input
// (box: 128 inputs x 1 channel x KT samples), which lands in shared memory in
// exactly the MN-major 128-byte-swizzled layout the MMA reads.  Eight decoder
// warps turn each raw byte into its E4M3 real and imaginary codes at the same
// offset of two operand tiles (Sec. 2.4's unpack, done on chip), and the MMA
// thread issues the same three MMAs per 32-sample step into [Re | -Im].  HBM
// traffic per step falls from input + 2 x planes written + planes read + output
// to input + output.
//
// Warp roles (448 threads, one CTA per SM): warps 0-3 drain TMEM (one tile row
// per thread) through a shared-memory transpose; warps 4-11 decode; warp 12
// is the TMA producer; warp 13 allocates TMEM and issues the MMAs.  Rings:
// RAW stages of raw tiles (I, J) and DEC stages of decoded tiles (Xr_I, Xi_I,
// Xr_J, Xi_J).  One drained block per tile pair: the caller uses this kernel
// only while n_time <= 130,944, where every FP32 partial sum is an exact
// integer below 2^24.  Every wait is bounded (sm103_ptx.cuh).
#include "ci4_decode.cuh"
#include "sm103_ptx.cuh"
#include "xcorr_internal.h"

namespace xc {
namespace {

constexpr int kBlk = 128;
constexpr int kEpiWarps = 4;
constexpr int kDecWarps = 8;
constexpr int kDecWarp0 = 4;
constexpr int kProducerWarp = 12;
constexpr int kMmaWarp = 13;
constexpr int kThreads = 448;
constexpr int kChunk = 16;
constexpr int kPitch = kChunk + 1;
constexpr int kAccCols = 256;  // [Re | -Im]
constexpr uint32_t kTmemCols = 512;
constexpr int kStagingBytes = kEpiWarps * 32 * kPitch * 8;
constexpr int kBarrierBytes = 512;

template <int KT, int RAW, int DEC>
struct FGeom {
  static constexpr int kTile = KT * 128;        // one 128-input tile, raw or decoded
  static constexpr int kRawStage = 2 * kTile;   // raw I, raw J
  static constexpr int kDecStage = 4 * kTile;   // Xr_I, Xi_I, Xr_J, Xi_J
  static constexpr int kSmem = 1024 + RAW * kRawStage + DEC * kDecStage + kStagingBytes + kBarrierBytes;
  static constexpr int kSteps = KT / 32;        // MMA steps (32 samples) per stage
  static_assert(KT % 32 == 0, "stage must hold whole MMA steps");
  static_assert(kSmem <= 232448, "shared memory budget");
};

struct FParams {
  int n_chan, n_inputs, n_tile_pairs, n_kt;
  int64_t n_pairs;
  int accumulate;  // add into out (else store)
  int2* out;
  int* status;
};

__device__ __forceinline__ void tile_pair(int p, int& I, int& J) {
  int i = static_cast<int>((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  I = i;
  J = p - i * (i + 1) / 2;
}

template <int KT, int RAW, int DEC>
__global__ void __launch_bounds__(kThreads, 1)
    xcorr_tc_fused_kernel(const __grid_constant__ CUtensorMap raw_map, const __grid_constant__ FParams p) {
  using G = FGeom<KT, RAW, DEC>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* raw = smem;
  uint8_t* dec = smem + RAW * G::kRawStage;
  int2* staging = reinterpret_cast<int2*>(dec + DEC * G::kDecStage);
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(staging) + kStagingBytes);
  uint64_t* raw_empty = raw_full + RAW;
  uint64_t* dec_full = raw_empty + RAW;
  uint64_t* dec_empty = dec_full + DEC;
  uint64_t* tfull = dec_empty + DEC;
  uint64_t* tempty = tfull + 2;
  uint64_t* mma_done = tempty + 2;
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
  const int n_items = p.n_chan * p.n_tile_pairs;

  if (warp == kProducerWarp) {
    if (lane == 0) {
      prefetch_tmap(&raw_map);
      int r = 0;
      uint32_t ph = 0, filled = 0, fill_parity[RAW] = {};
      bool ok = true;
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
        const int c = item / p.n_tile_pairs;
        int I, J;
        tile_pair(item - c * p.n_tile_pairs, I, J);
        const bool diag = (I == J);
        for (int tb = 0; tb < p.n_kt; ++tb) {
          if (!mbar_wait(&raw_empty[r], ph ^ 1u, abort_flag, p.status, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          uint8_t* st = raw + r * G::kRawStage;
          mbar_expect_tx(&raw_full[r], (diag ? 1 : 2) * G::kTile);
          tma_load_3d(st, &raw_map, &raw_full[r], I * kBlk, c, tb * KT);
          if (!diag) tma_load_3d(st + G::kTile, &raw_map, &raw_full[r], J * kBlk, c, tb * KT);
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
    // Decoders: raw CI4 bytes -> E4M3 real / imaginary codes at the same offsets.
    const int tid = (warp - kDecWarp0) * 32 + lane;
    int r = 0, d = 0;
    uint32_t rph = 0, dph = 0;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
      const int c = item / p.n_tile_pairs;
      int I, J;
      tile_pair(item - c * p.n_tile_pairs, I, J);
      const int total = (I == J ? 1 : 2) * (G::kTile / 16);  // 16-byte chunks this stage
      for (int tb = 0; tb < p.n_kt; ++tb) {
        if (!mbar_wait(&raw_full[r], rph, abort_flag, p.status, DEV_TIMEOUT_FULL) ||
            !mbar_wait(&dec_empty[d], dph ^ 1u, abort_flag, p.status, DEV_TIMEOUT_EMPTY)) {
          ok = false;
          break;
        }
        const uint4* src = reinterpret_cast<const uint4*>(raw + r * G::kRawStage);
        uint8_t* dst = dec + d * G::kDecStage;
#pragma unroll 4
        for (int q = tid; q < total; q += kDecWarps * 32) {
          const int tile = q / (G::kTile / 16);
          const int off = (q - tile * (G::kTile / 16)) * 16;
          const uint4 v = src[q];
          uint4 re, im;
          ci4_to_e4m3(v.x, re.x, im.x);
          ci4_to_e4m3(v.y, re.y, im.y);
          ci4_to_e4m3(v.z, re.z, im.z);
          ci4_to_e4m3(v.w, re.w, im.w);
          *reinterpret_cast<uint4*>(dst + (2 * tile) * G::kTile + off) = re;
          *reinterpret_cast<uint4*>(dst + (2 * tile + 1) * G::kTile + off) = im;
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
    }
  } else if (warp == kMmaWarp) {
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
    int g = 0;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x, ++g) {
      const int c = item / p.n_tile_pairs;
      int I, J;
      tile_pair(item - c * p.n_tile_pairs, I, J);
      int2* out_c = p.out + (int64_t)c * p.n_pairs;
      const int row0 = I * kBlk + warp * 32;
      const int buf = g & 1;
      const uint32_t use = static_cast<uint32_t>(g >> 1);
      if (!mbar_wait(&tfull[buf], use & 1u, abort_flag, p.status, DEV_TIMEOUT_TMEM_FULL)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + buf * kAccCols;
      for (int j0 = 0; j0 < kBlk; j0 += kChunk) {
        uint32_t re[16], nim[16];
        tmem_ld16(taddr + j0, re);
        tmem_ld16(taddr + 128 + j0, nim);
        tmem_ld_wait();
        const int jfirst = J * kBlk + j0;
        if (jfirst > row0 + 31 || row0 >= p.n_inputs) continue;  // wholly above the diagonal or past the inputs
#pragma unroll
        for (int q = 0; q < 16; ++q)
          stage_rows[lane * kPitch + q] = make_int2(__float2int_rn(__uint_as_float(re[q])),
                                                    -__float2int_rn(__uint_as_float(nim[q])));
        __syncwarp();
        // a half-warp writes 16 consecutive pairs of one row
        const int j = jfirst + col;
        uint32_t valid = 0;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int i = row0 + 2 * r + half;
          if (i < p.n_inputs && j <= i) valid |= 1u << r;
        }
        int2 old[16];
        if (p.accumulate) {  // (continuing an integration: loads first, then adds)
#pragma unroll 1
          for (int r = 0; r < 16; ++r) {
            const int i = row0 + 2 * r + half;
            old[r] = (valid >> r) & 1u ? out_c[(int64_t)i * (i + 1) / 2 + j] : make_int2(0, 0);
          }
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          if ((valid >> r) & 1u) {
            const int rr = 2 * r + half;
            const int i = row0 + rr;
            int2 v = stage_rows[rr * kPitch + col];
            if (p.accumulate) {
              v.x += old[r].x;
              v.y += old[r].y;
            }
            out_c[(int64_t)i * (i + 1) / 2 + j] = v;
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
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

template <int KT, int RAW, int DEC>
cudaError_t launch_fused(const CUtensorMap* raw_map, const FParams& p, int grid, cudaStream_t stream) {
  using G = FGeom<KT, RAW, DEC>;
  auto kern = xcorr_tc_fused_kernel<KT, RAW, DEC>;
  static int attr_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_device != dev) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmem);
    if (e != cudaSuccess) return e;
    attr_device = dev;
  }
  kern<<<grid, kThreads, G::kSmem, stream>>>(*raw_map, p);
  return cudaGetLastError();
}

}  // namespace

// Stage heights of the fused variants: 128 samples (2 raw + 2 decoded stages),
// 96 (2 + 3), 64 (4 + 4).
int fused_stage_samples(int variant) { return variant == 0 ? 128 : variant == 1 ? 96 : 64; }

cudaError_t launch_xcorr_tc_fused_ci4(const CUtensorMap* raw_map, int variant, int n_time, int n_chan, int n_inputs,
                                      int2* out, bool accumulate, int* status, int num_sms, cudaStream_t stream) {
  const int nb = (n_inputs + kBlk - 1) / kBlk;
  const int kt = fused_stage_samples(variant);
  FParams p{};
  p.n_chan = n_chan;
  p.n_inputs = n_inputs;
  p.n_tile_pairs = nb * (nb + 1) / 2;
  p.n_kt = (n_time + kt - 1) / kt;
  p.n_pairs = (int64_t)n_inputs * (n_inputs + 1) / 2;
  p.accumulate = accumulate ? 1 : 0;
  p.out = out;
  p.status = status;
  if (n_time > kTcWindowCI4) return cudaErrorInvalidValue;  // one exact block per tile pair
  const int64_t items = (int64_t)n_chan * p.n_tile_pairs;
  const int grid = static_cast<int>(items < num_sms ? items : num_sms);
  switch (variant) {
    case 0: return launch_fused<128, 2, 2>(raw_map, p, grid, stream);
    case 1: return launch_fused<96, 2, 3>(raw_map, p, grid, stream);
    default: return launch_fused<64, 4, 4>(raw_map, p, grid, stream);
  }
}

}  // namespace xc
