// ci4_decode.cuh -- 4+4-bit complex samples to E4M3 codes, four at a time.
//
// A CI4 byte holds a 4-bit two's-complement real part in its high nibble and
// the imaginary part in its low nibble (the library's reading of the paper's
// four bits for each of the real and imaginary parts, Sec. 2.3).  Every value in [-8, 7] is an
// exact E4M3 number, so these codes feed kind::f8f6f4 MMAs with the true
// integers.  The lookups are byte permutes over two 8-entry tables.
#pragma once
#include <cstdint>

namespace xc {

// E4M3 codes of 0..7 and of -8..-1, four per word, lowest byte first.
constexpr uint32_t kE4m3Pos0 = 0x44403800u;  // 0, 1, 2, 3
constexpr uint32_t kE4m3Pos1 = 0x4E4C4A48u;  // 4, 5, 6, 7
constexpr uint32_t kE4m3Neg0 = 0xCACCCED0u;  // -8, -7, -6, -5
constexpr uint32_t kE4m3Neg1 = 0xB8C0C4C8u;  // -4, -3, -2, -1

// Byte-wise table lookup: `lo3` holds a 3-bit index in the low bits of each
// byte, `neg` is 0xFF in the bytes whose 4-bit code is negative.
__device__ __forceinline__ uint32_t e4m3_of_nibbles(uint32_t lo3, uint32_t neg) {
  uint32_t sel = lo3 | (lo3 >> 4);  // pack the four indices into 16 bits
  sel = (sel & 0xFFu) | ((sel >> 8) & 0xFF00u);
  const uint32_t pos = __byte_perm(kE4m3Pos0, kE4m3Pos1, sel);
  const uint32_t ngt = __byte_perm(kE4m3Neg0, kE4m3Neg1, sel);
  return (ngt & neg) | (pos & ~neg);
}

// Four CI4 samples (one per byte) -> four E4M3 real parts and four imaginary parts.
__device__ __forceinline__ void ci4_to_e4m3(uint32_t v, uint32_t& re, uint32_t& im) {
  re = e4m3_of_nibbles((v >> 4) & 0x07070707u, ((v >> 7) & 0x01010101u) * 0xFFu);
  im = e4m3_of_nibbles(v & 0x07070707u, ((v >> 3) & 0x01010101u) * 0xFFu);
}

}  // namespace xc
