// xcorr_cuda_core.cu -- the plain CUDA-core X kernel (the comparison method).
//
// Same computation as the tensor-core kernel (per channel, the packed lower
// triangle of V = sum_t x_t x_t^H, Sec. 1 / Sec. 2.1 / Eq. 1), done with
// 4-way int8 dot products (dp4a) and exact int32 accumulation:
//     Re += dp4a(xr_i, xr_j) + dp4a(xi_i, xi_j)
//     Im += dp4a(xi_i, xr_j) - dp4a(xr_i, xi_j)
// where each 32-bit operand packs four consecutive time samples of one input.
//
// A CTA of 256 threads owns a 64 x 64 tile pair (I >= J) of one channel and a
// range of time.  It reads the packed input itself (4+4-bit or int8 complex),
// widens it to int8 and turns four time rows x four inputs into four
// time-packed words per input with byte permutes (the corner turn of Sec. 2.4
// done in registers), so this engine needs no staging planes.  Each thread
// keeps a 4 x 4 block of (Re, Im_a, Im_b) sums in registers.  When the time
// axis is split over several CTAs, their partial sums meet with atomic adds
// (exact in integers).
#include "xcorr_internal.h"

namespace xc {
namespace {

constexpr int kT = 64;      // inputs per tile side
constexpr int kKT = 32;     // samples per smem chunk (8 words of 4 samples)
constexpr int kW = kKT / 4; // words per row per chunk

// Widen four packed 4-bit codes (one per byte, in the high or low nibble) to
// sign-extended int8 lanes.
__device__ __forceinline__ uint32_t sext_nibbles(uint32_t x) {
  x &= 0x0F0F0F0Fu;
  return x | ((x & 0x08080808u) * 0x1Eu);
}

// 4 x 4 byte transpose: w[q] byte k  ->  v[k] byte q.
__device__ __forceinline__ void transpose4x4(const uint32_t (&w)[4], uint32_t (&v)[4]) {
  const uint32_t x0 = __byte_perm(w[0], w[1], 0x5140), x1 = __byte_perm(w[0], w[1], 0x7362);
  const uint32_t x2 = __byte_perm(w[2], w[3], 0x5140), x3 = __byte_perm(w[2], w[3], 0x7362);
  v[0] = __byte_perm(x0, x2, 0x5410);
  v[1] = __byte_perm(x0, x2, 0x7632);
  v[2] = __byte_perm(x1, x3, 0x5410);
  v[3] = __byte_perm(x1, x3, 0x7632);
}

struct CcParams {
  const uint8_t* in;
  int n_time, n_chan, n_inputs, n_tile_pairs, ksplit, k_per_split;
  int64_t n_pairs;
  int mode;
  int aligned;  // rows of 4 inputs can be read as one 4-byte (CI4) or 8-byte (CI8) word
  int2* acc;
};

__device__ __forceinline__ void tile_pair(int p, int& I, int& J) {
  int i = static_cast<int>((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  I = i;
  J = p - i * (i + 1) / 2;
}

// Load 4 time rows x 4 inputs of one block, widened and time-packed:
// re[k] / im[k] hold samples t0 .. t0 + 3 of input base + k.
template <int FMT>
__device__ __forceinline__ void load_group(const CcParams& p, int c, int t0, int t_end, int base,
                                           bool aligned, uint32_t (&re)[4], uint32_t (&im)[4]) {
  uint32_t wr[4], wi[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int t = t0 + q;
    wr[q] = 0u;
    wi[q] = 0u;
    if (t < t_end && base < p.n_inputs) {
      const int64_t s = ((int64_t)t * p.n_chan + c) * p.n_inputs + base;  // first sample of the group
      if (FMT == XCORR_IN_CI4) {
        uint32_t raw;
        if (aligned && base + 4 <= p.n_inputs) {
          raw = __ldg(reinterpret_cast<const uint32_t*>(p.in + s));
        } else {
          raw = 0u;
          for (int k = 0; k < 4 && base + k < p.n_inputs; ++k) raw |= (uint32_t)p.in[s + k] << (8 * k);
        }
        wr[q] = sext_nibbles(raw >> 4);
        wi[q] = sext_nibbles(raw);
      } else {
        uint32_t lo, hi;
        if (aligned && base + 4 <= p.n_inputs) {
          const uint2 v = __ldg(reinterpret_cast<const uint2*>(p.in + 2 * s));
          lo = v.x;
          hi = v.y;
        } else {
          lo = hi = 0u;
          for (int k = 0; k < 4 && base + k < p.n_inputs; ++k) {
            const uint32_t pair = (uint32_t)p.in[2 * s + 2 * k] | ((uint32_t)p.in[2 * s + 2 * k + 1] << 8);
            if (k < 2) lo |= pair << (16 * k); else hi |= pair << (16 * (k - 2));
          }
        }
        wr[q] = __byte_perm(lo, hi, 0x6420);
        wi[q] = __byte_perm(lo, hi, 0x7531);
      }
    }
  }
  transpose4x4(wr, re);
  transpose4x4(wi, im);
}

template <int FMT>
__global__ void __launch_bounds__(256) xcorr_cc_kernel(const CcParams p) {
  __shared__ __align__(16) uint32_t sm[2][4][kW][kT];  // [buffer][Ar, Ai, Br, Bi][word][row]
  const int tid = threadIdx.x;
  const int split = blockIdx.x % p.ksplit;
  const int rest = blockIdx.x / p.ksplit;
  const int c = rest / p.n_tile_pairs;
  int I, J;
  tile_pair(rest - c * p.n_tile_pairs, I, J);
  const bool diag = (I == J);
  const int t_begin = split * p.k_per_split;
  const int t_end = min(p.n_time, t_begin + p.k_per_split);
  const bool aligned = p.aligned != 0;

  // loader role: threads 0..127 fetch block I, 128..255 block J
  const int side = tid >> 7, u = tid & 127;
  const int g4 = u & 15, t4 = u >> 4;  // input group of 4, time group of 4
  const int blk = side ? J : I;
  const bool loads = !(side && diag);
  const int base = blk * kT + 4 * g4;

  // compute role
  const int ty = tid >> 4, tx = tid & 15;
  int re[4][4], ima[4][4], imb[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) re[a][b] = ima[a][b] = imb[a][b] = 0;

  uint32_t nr[4], ni[4];
  int buf = 0;
  if (loads) {
    load_group<FMT>(p, c, t_begin + 4 * t4, t_end, base, aligned, nr, ni);
    *reinterpret_cast<uint4*>(&sm[0][2 * side][t4][4 * g4]) = make_uint4(nr[0], nr[1], nr[2], nr[3]);
    *reinterpret_cast<uint4*>(&sm[0][2 * side + 1][t4][4 * g4]) = make_uint4(ni[0], ni[1], ni[2], ni[3]);
  }
  __syncthreads();
  const int bsel = diag ? 0 : 2;
  for (int t0 = t_begin; t0 < t_end; t0 += kKT) {
    const bool more = t0 + kKT < t_end;
    if (more && loads) load_group<FMT>(p, c, t0 + kKT + 4 * t4, t_end, base, aligned, nr, ni);
#pragma unroll
    for (int w = 0; w < kW; ++w) {
      int ar[4], ai[4], br[4], bi[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ar[a] = static_cast<int>(sm[buf][0][w][ty + 16 * a]);
        ai[a] = static_cast<int>(sm[buf][1][w][ty + 16 * a]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        br[b] = static_cast<int>(sm[buf][bsel][w][tx + 16 * b]);
        bi[b] = static_cast<int>(sm[buf][bsel + 1][w][tx + 16 * b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          re[a][b] = __dp4a(ar[a], br[b], re[a][b]);
          re[a][b] = __dp4a(ai[a], bi[b], re[a][b]);
          ima[a][b] = __dp4a(ai[a], br[b], ima[a][b]);
          imb[a][b] = __dp4a(ar[a], bi[b], imb[a][b]);
        }
    }
    if (more) {
      buf ^= 1;
      if (loads) {
        *reinterpret_cast<uint4*>(&sm[buf][2 * side][t4][4 * g4]) = make_uint4(nr[0], nr[1], nr[2], nr[3]);
        *reinterpret_cast<uint4*>(&sm[buf][2 * side + 1][t4][4 * g4]) = make_uint4(ni[0], ni[1], ni[2], ni[3]);
      }
      __syncthreads();
    }
  }

  int2* acc_c = p.acc + (int64_t)c * p.n_pairs;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = I * kT + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = J * kT + tx + 16 * b;
      if (i < p.n_inputs && j <= i) {
        int2* dst = acc_c + (int64_t)i * (i + 1) / 2 + j;
        const int vr = re[a][b], vi = ima[a][b] - imb[a][b];
        if (p.mode == MODE_ATOMIC) {
          atomicAdd(&dst->x, vr);
          atomicAdd(&dst->y, vi);
        } else if (p.mode == MODE_ADD) {
          const int2 o = *dst;
          *dst = make_int2(o.x + vr, o.y + vi);
        } else {
          *dst = make_int2(vr, vi);
        }
      }
    }
  }
}

}  // namespace

int cuda_core_ksplit(int n_time, int n_chan, int n_inputs, int num_sms) {
  const int nb = (n_inputs + kT - 1) / kT;
  const int64_t tiles = (int64_t)n_chan * nb * (nb + 1) / 2;
  const int64_t want = 4LL * num_sms;  // CTAs for a full device (several per SM)
  int ks = 1;
  while (tiles * ks < want && (n_time / (ks * 2)) >= 4 * kKT) ks *= 2;
  return ks;
}

cudaError_t launch_xcorr_cuda_core(int fmt, const void* in, int n_time, int n_chan, int n_inputs,
                                   int2* acc, int mode, int ksplit, cudaStream_t stream) {
  const int nb = (n_inputs + kT - 1) / kT;
  CcParams p;
  p.in = static_cast<const uint8_t*>(in);
  p.n_time = n_time;
  p.n_chan = n_chan;
  p.n_inputs = n_inputs;
  p.n_tile_pairs = nb * (nb + 1) / 2;
  p.ksplit = ksplit;
  p.k_per_split = ((n_time + ksplit - 1) / ksplit + kKT - 1) / kKT * kKT;
  p.n_pairs = (int64_t)n_inputs * (n_inputs + 1) / 2;
  p.mode = mode;
  p.aligned = (n_inputs % 4 == 0) &&
              (reinterpret_cast<uintptr_t>(in) % (fmt == XCORR_IN_CI4 ? 4 : 8) == 0);
  p.acc = acc;
  const int64_t blocks = (int64_t)n_chan * p.n_tile_pairs * ksplit;
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
  if (fmt == XCORR_IN_CI4)
    xcorr_cc_kernel<XCORR_IN_CI4><<<(unsigned)blocks, 256, 0, stream>>>(p);
  else
    xcorr_cc_kernel<XCORR_IN_CI8><<<(unsigned)blocks, 256, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace xc
