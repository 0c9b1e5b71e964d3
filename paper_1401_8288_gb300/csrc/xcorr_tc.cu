// xcorr_tc.cu -- the X-stage on the Blackwell tensor cores (tcgen05).
//
// For each channel c the X-stage is the complex rank-K update
//     V = sum_t x_t x_t^H,  x_t = xr_t + j xi_t  (Sec. 1 and Sec. 2.1; Eq. 1
// counts the N_i (N_i + 1) / 2 pairs), which splits into real products:
//     Re V = Xr Xr^T + Xi Xi^T,   Im V = Xi Xr^T - Xr Xi^T
// with X[i][t] the N_i x K matrix of one channel's samples.
//
// The input triangle is cut into 128 x 128 tile pairs (I >= J); a persistent
// CTA walks a static list of (channel, I, J) items, channel-major, so the
// CTAs in flight share the channels' planes in L2.  Per 64-sample stage, TMA
// brings the four 64 x 128 E4M3 tiles Xr_I, Xi_I, Xr_J, Xi_J (two on the
// diagonal) into a six-deep shared-memory ring as MN-major operands, and one thread issues,
// per 32-sample step, three MMAs into an FP32 accumulator of 256 TMEM columns
// holding [Re | -Im]:
//     [Re | -Im] += Xr_I [Xr_J | Xi_J]^T       (M = 128, N = 256)
//     Re         += Xi_I Xi_J^T                (N = 128)
//     -Im        += (-Xi_I) Xr_J^T             (N = 128, negate-A bit)
// Every product is exact (4-bit integers are E4M3 values), and FP32 sums of
// integers are exact below 2^24, so the K axis is cut into windows of at most
// 130,944 samples (128 * 130,944 < 2^24); each window is drained to int32.  Two
// accumulator buffers (512 columns) let the epilogue of one window overlap the
// MMAs of the next.
//
// Warp roles (192 threads, one CTA per SM): warps 0-3 drain TMEM (thread =
// accumulator row) and add the lower-triangle part of the tile into the packed
// int32 accumulator through a shared-memory transpose that makes the global
// stores row-contiguous; warp 4 is the TMA producer; warp 5 allocates TMEM and
// issues the MMAs.
#include "sm103_ptx.cuh"
#include "xcorr_internal.h"

namespace xc {
namespace {

constexpr int kBlk = 128;                   // inputs per tile side
constexpr int kKT = kTcStageT;              // samples per stage
constexpr int kTileBytes = kBlk * kKT;      // one E4M3 plane tile: 8 KB
constexpr int kStageBytes = 4 * kTileBytes; // Xr_I, Xi_I, Xr_J, Xi_J
constexpr int kStages = 6;
constexpr int kEpiWarps = 4;
constexpr int kThreads = 192;
constexpr int kProducerWarp = 4;
constexpr int kMmaWarp = 5;
constexpr int kChunk = 16;         // accumulator columns per epilogue step
constexpr int kPitch = kChunk + 1; // int2 per staged row
constexpr int kAccCols = 256;      // [Re | -Im]
constexpr uint32_t kTmemCols = 512;
constexpr int kStagingBytes = kEpiWarps * 32 * kPitch * 8;
constexpr int kBarrierBytes = 256;
constexpr int kSmemBytes = 1024 + kStages * kStageBytes + kStagingBytes + kBarrierBytes;
static_assert(kSmemBytes <= 232448, "shared memory budget");

struct TcParams {
  int chan0, n_chan, n_inputs, n_tile_pairs, n_kblocks, kb_per_window;
  int64_t n_pairs;
  int accumulate_first;  // the first window adds into acc (else it stores)
  int2* acc;
  int* status;
};

__device__ __forceinline__ void tile_pair(int p, int& I, int& J) {
  int i = static_cast<int>((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  I = i;
  J = p - i * (i + 1) / 2;
}

__global__ void __launch_bounds__(kThreads, 1)
    xcorr_tc_e4m3_kernel(const __grid_constant__ CUtensorMap tmap, const TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stages = smem;
  int2* staging = reinterpret_cast<int2*>(smem + kStages * kStageBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes + kStagingBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* mma_done = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
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

  const int n_items = p.n_chan * p.n_tile_pairs;
  const int n_windows = (p.n_kblocks + p.kb_per_window - 1) / p.kb_per_window;

  if (warp == kProducerWarp) {
    if (lane == 0) {
      prefetch_tmap(&tmap);
      int s = 0;
      uint32_t ph = 0, filled = 0, fill_parity[kStages] = {};
      bool ok = true;
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
        const int cl = item / p.n_tile_pairs;
        const int c = p.chan0 + cl;
        int I, J;
        tile_pair(item - cl * p.n_tile_pairs, I, J);
        const bool diag = (I == J);
        for (int kb = 0; kb < p.n_kblocks; ++kb) {
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, p.status, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          uint8_t* st = stages + s * kStageBytes;
          mbar_expect_tx(&full[s], (diag ? 2 : 4) * kTileBytes);
          tma_load_3d(st, &tmap, &full[s], I * kBlk, kb * kKT, 2 * c);
          tma_load_3d(st + kTileBytes, &tmap, &full[s], I * kBlk, kb * kKT, 2 * c + 1);
          if (!diag) {
            tma_load_3d(st + 2 * kTileBytes, &tmap, &full[s], J * kBlk, kb * kKT, 2 * c);
            tma_load_3d(st + 3 * kTileBytes, &tmap, &full[s], J * kBlk, kb * kKT, 2 * c + 1);
          }
          fill_parity[s] = ph;
          filled |= 1u << s;
          if (++s == kStages) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      // Let every copy this CTA issued land before the CTA can exit.
      volatile int never = 0;
      for (int q = 0; q < kStages; ++q)
        if (filled & (1u << q)) mbar_wait(&full[q], fill_parity[q], &never, p.status, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      const uint32_t id256 = instr_desc(kTypeE4M3, true, 128, 256, false);
      const uint32_t id128 = instr_desc(kTypeE4M3, true, 128, 128, false);
      const uint32_t id128n = instr_desc(kTypeE4M3, true, 128, 128, true);
      int s = 0;
      uint32_t ph = 0;
      int g = 0;  // windows processed by this CTA
      bool ok = true;
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
        const int c = item / p.n_tile_pairs;
        int I, J;
        tile_pair(item - c * p.n_tile_pairs, I, J);
        const bool diag = (I == J);
        for (int w = 0; ok && w < n_windows; ++w, ++g) {
          const int buf = g & 1;
          const uint32_t use = static_cast<uint32_t>(g >> 1);
          if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, abort_flag, p.status, DEV_TIMEOUT_TMEM_EMPTY)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + static_cast<uint32_t>(buf * kAccCols);
          const int kb0 = w * p.kb_per_window;
          const int kb1 = min(p.n_kblocks, kb0 + p.kb_per_window);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&full[s], ph, abort_flag, p.status, DEV_TIMEOUT_FULL)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_r = smem_u32(stages + s * kStageBytes);
            const uint32_t a_i = a_r + kTileBytes;
            const uint32_t b_r = diag ? a_r : a_r + 2 * kTileBytes;
            const uint32_t b_i = b_r + kTileBytes;
#pragma unroll
            for (int k = 0; k < kKT / 32; ++k) {
              const uint32_t off = static_cast<uint32_t>(k) * 32u * kBlk;  // 32 rows of 128 B
              const uint32_t first = (kb == kb0 && k == 0) ? 1u : 0u;
              mma_f8f6f4(d, smem_desc_sw128(a_r + off, kTileBytes, 1024),
                         smem_desc_sw128(b_r + off, kTileBytes, 1024), id256, first ^ 1u);
              mma_f8f6f4(d, smem_desc_sw128(a_i + off, kTileBytes, 1024),
                         smem_desc_sw128(b_i + off, kTileBytes, 1024), id128, 1u);
              mma_f8f6f4(d + 128, smem_desc_sw128(a_i + off, kTileBytes, 1024),
                         smem_desc_sw128(b_r + off, kTileBytes, 1024), id128n, 1u);
            }
            mma_commit(&empty[s]);
            if (++s == kStages) {
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
    // Epilogue: warp w drains TMEM lanes 32w .. 32w + 31 (tile rows).
    int2* stage_rows = staging + warp * 32 * kPitch;
    const int half = lane >> 4, col = lane & 15;
    int g = 0;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
      const int cl = item / p.n_tile_pairs;
      int I, J;
      tile_pair(item - cl * p.n_tile_pairs, I, J);
      int2* acc_c = p.acc + (int64_t)(p.chan0 + cl) * p.n_pairs;
      const int row0 = I * kBlk + warp * 32;  // first global input row of this warp
      for (int w = 0; w < n_windows; ++w, ++g) {
        const int buf = g & 1;
        const uint32_t use = static_cast<uint32_t>(g >> 1);
        if (!mbar_wait(&tfull[buf], use & 1u, abort_flag, p.status, DEV_TIMEOUT_TMEM_FULL)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const bool add = (w > 0) || p.accumulate_first;
        const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + buf * kAccCols;
        for (int j0 = 0; j0 < kBlk; j0 += kChunk) {
          uint32_t re[16], nim[16];
          tmem_ld16(taddr + j0, re);
          tmem_ld16(taddr + 128 + j0, nim);
          tmem_ld_wait();
          // skip chunks that lie wholly above the diagonal or past the inputs
          const int jfirst = J * kBlk + j0;
          const bool any = (jfirst <= row0 + 31) && (row0 < p.n_inputs);
          if (any) {
#pragma unroll
            for (int q = 0; q < 16; ++q)
              stage_rows[lane * kPitch + q] = make_int2(__float2int_rn(__uint_as_float(re[q])),
                                                        -__float2int_rn(__uint_as_float(nim[q])));
            __syncwarp();
#pragma unroll 4
            for (int r = 0; r < 32; r += 2) {
              const int rr = r + half;
              const int i = row0 + rr;
              const int j = jfirst + col;
              if (i < p.n_inputs && j <= i) {
                int2 v = stage_rows[rr * kPitch + col];
                int2* dst = acc_c + (int64_t)i * (i + 1) / 2 + j;
                if (add) {
                  const int2 o = *dst;
                  v.x += o.x;
                  v.y += o.y;
                }
                *dst = v;
              }
            }
            __syncwarp();
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
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

}  // namespace

cudaError_t launch_xcorr_tc_e4m3(const CUtensorMap* tmap, int n_time, int chan0, int n_chan,
                                 int n_inputs, int2* acc, bool accumulate, int* status,
                                 int num_sms, cudaStream_t stream) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(xcorr_tc_e4m3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int nb = (n_inputs + kBlk - 1) / kBlk;
  TcParams p;
  p.chan0 = chan0;
  p.n_chan = n_chan;
  p.n_inputs = n_inputs;
  p.n_tile_pairs = nb * (nb + 1) / 2;
  p.n_kblocks = (n_time + kKT - 1) / kKT;
  p.kb_per_window = kTcMaxKblocksPerWindow;
  p.n_pairs = (int64_t)n_inputs * (n_inputs + 1) / 2;
  p.accumulate_first = accumulate ? 1 : 0;
  p.acc = acc;
  p.status = status;
  const int64_t items = (int64_t)n_chan * p.n_tile_pairs;
  const int grid = static_cast<int>(items < num_sms ? items : num_sms);
  xcorr_tc_e4m3_kernel<<<grid, kThreads, kSmemBytes, stream>>>(*tmap, p);
  return cudaGetLastError();
}

}  // namespace xc
