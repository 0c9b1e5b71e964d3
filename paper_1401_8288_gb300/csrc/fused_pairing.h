// fused_pairing.h -- which tile pairs of a channel the two CTAs of a pair share (the
// CTA-pair fused kernel, xcorr_tc_fused_pair.cu).  Plain integer code, usable on the host
// (tests/test_pairing.py compiles it with g++ and checks every tile count up to 300).
//
// A channel's visibilities (the packed lower triangle of V, Eq. 1) split into tile pairs (I, J),
// I >= J, of 128 x 128 inputs.  The two CTAs of a pair share the column tile S and each computes
// one row tile against it; an entry names S and the two row tiles.  Column tile S holds the row
// tiles S .. nb - 1.  Columns whose count is odd (S = o, o + 2, ..., o = (nb - 1) % 2) are
// matched as (u, u + 2): u gives its row tile u + 2 away, and u + 2 takes the tile pair (u + 2, u)
// as row tile u, computed transposed.  An odd column left without a partner (always nb - 1) keeps
// a single row tile.
#pragma once

#ifdef __CUDACC__
#define XC_PAIR_FN __host__ __device__ inline
#else
#define XC_PAIR_FN inline
#endif

namespace xc {
namespace fused {

enum : int { kColEven = 0, kColGives = 1, kColTakes = 2, kColSingle = 3 };

XC_PAIR_FN int pair_col_kind(int nb, int S) {
  const int o = (nb - 1) & 1;
  if ((S - o) & 1) return kColEven;
  if (((S - o) >> 1) & 1) return kColTakes;
  return S + 2 <= nb - 1 ? kColGives : kColSingle;
}

// Row tiles column S ends up with.
XC_PAIR_FN int pair_col_len(int nb, int S) {
  const int k = pair_col_kind(nb, S);
  return nb - S - (k == kColGives ? 1 : 0) + (k == kColTakes ? 1 : 0);
}

// Entries of the columns before S: half of their original counts, less one half while a column
// that gave a row tile away is not yet balanced by the one that took it.
XC_PAIR_FN int pair_col_prefix(int nb, int S) {
  const int q = S * nb - S * (S - 1) / 2;
  const bool open =
      (S >= 1 && pair_col_kind(nb, S - 1) == kColGives) || (S >= 2 && pair_col_kind(nb, S - 2) == kColGives);
  return (q - (open ? 1 : 0)) >> 1;
}

// Entries per channel: ceil(nb (nb + 1) / 4).
XC_PAIR_FN int pair_entries(int nb) { return pair_col_prefix(nb, nb - 1) + ((pair_col_len(nb, nb - 1) + 1) >> 1); }

// Row tile j of column S's list: the taken tile first, the given one skipped.
XC_PAIR_FN int pair_col_row(int nb, int S, int j) {
  const int k = pair_col_kind(nb, S);
  if (k == kColTakes) return j == 0 ? S - 2 : S + j - 1;
  if (k == kColGives) return S + j + (j >= 2 ? 1 : 0);
  return S + j;
}

// Entry e of a channel: the column tile and the two CTAs' row tiles (-1: none).  A row tile
// below S means the tile pair (S, row) computed transposed.
XC_PAIR_FN void pair_entry(int nb, int e, int& S, int& r0, int& r1) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pair_col_prefix(nb, mid) <= e)
      lo = mid;
    else
      hi = mid - 1;
  }
  S = lo;
  const int k = e - pair_col_prefix(nb, S);
  r0 = pair_col_row(nb, S, 2 * k);
  r1 = 2 * k + 1 < pair_col_len(nb, S) ? pair_col_row(nb, S, 2 * k + 1) : -1;
}

}  // namespace fused
}  // namespace xc
