"""Pins for the oracle: each test ties it to something other than itself.

* the CI4 decode against int8 shift arithmetic and hand-written bytes;
* the whole triangle against a numpy full-matrix brute force (einsum of x x^H)
  on tiny inputs, including every pair of byte codes;
* closed forms: constant inputs, quarter-turn tones (V_ij = K A^2 j^(q_i - q_j));
* invariants: real non-negative autos, additivity over time, permutation
  equivariance with conjugation, the int8 and float formats agreeing with the
  4-bit one on the same values;
* one statistical check: the phase of a plane-wave source.

A plausible slip in the oracle (a dropped term, a sign, a swapped conjugate,
a transposed pair index, the nibble order) fails at least one of these.
"""

import numpy as np
import pytest

import oracle
from oracle import FMT_CF32, FMT_CI4, FMT_CI8
from paper_1401_8288_gb300 import synth


def decode_np(b: np.ndarray) -> np.ndarray:
    """CI4 -> complex128 by arithmetic shifts of the byte read as int8."""
    s = np.asarray(b, dtype=np.uint8).view(np.int8)
    re = (s >> 4).astype(np.int64)
    im = (np.left_shift(s, 4).astype(np.int8) >> 4).astype(np.int64)
    return re + 1j * im


def full_matrix(xc: np.ndarray) -> np.ndarray:
    """Brute force: V[c] = sum_t x_t x_t^H as a full matrix, xc [K][C][N]."""
    return np.einsum("tci,tcj->cij", xc, xc.conj())


def lower(vfull: np.ndarray) -> np.ndarray:
    """Full matrices [C][N][N] -> packed lower triangle [C][P][2]."""
    n = vfull.shape[1]
    ii, jj = np.tril_indices(n)
    order = np.argsort(ii * (ii + 1) // 2 + jj)
    v = vfull[:, ii[order], jj[order]]
    return np.stack([v.real, v.imag], axis=-1)


def ci4_to_ci8(x: np.ndarray) -> np.ndarray:
    xc = decode_np(x)
    return np.stack([xc.real, xc.imag], axis=-1).astype(np.int8)


# ---------------------------------------------------------------- decode ---

def test_decode_hand_bytes():
    # real in the high nibble, imaginary in the low nibble, two's complement
    assert oracle.decode_ci4(0x7F) == (7, -1)
    assert oracle.decode_ci4(0x80) == (-8, 0)
    assert oracle.decode_ci4(0x08) == (0, -8)
    assert oracle.decode_ci4(0x10) == (1, 0)
    assert oracle.decode_ci4(0x01) == (0, 1)
    assert oracle.decode_ci4(0xFF) == (-1, -1)
    assert oracle.decode_ci4(0x9E) == (-7, -2)


def test_decode_all_bytes_against_shift_arithmetic():
    codes = np.arange(256, dtype=np.uint8)
    xc = decode_np(codes)
    for b in range(256):
        assert oracle.decode_ci4(b) == (int(xc[b].real), int(xc[b].imag))


def test_generator_round_trip():
    re = np.arange(-8, 8).repeat(16)
    im = np.tile(np.arange(-8, 8), 16)
    xc = decode_np(synth.pack_ci4(re, im))
    assert np.array_equal(xc.real, re) and np.array_equal(xc.imag, im)


# ------------------------------------------------------------ brute force ---

@pytest.mark.parametrize("n_sta", [1, 2, 3])
@pytest.mark.parametrize("n_time", [1, 2, 3])
@pytest.mark.parametrize("n_chan", [1, 2])
def test_tiny_against_full_matrix(n_sta, n_time, n_chan):
    rng = np.random.default_rng(1000 * n_sta + 10 * n_time + n_chan)
    x = rng.integers(0, 256, size=(n_time, n_chan, n_sta, 2), dtype=np.uint8)
    want = lower(full_matrix(decode_np(x).reshape(n_time, n_chan, 2 * n_sta)))
    got = oracle.correlate(FMT_CI4, x)
    assert got.dtype == np.int64
    assert np.array_equal(got, want.astype(np.int64))


def test_every_code_pair_single_sample():
    # inputs 0..255 carry codes 0..255 and inputs 256..511 carry them again, so
    # pairs (256 + a, b) cover every ordered pair of byte codes (a, b).
    codes = np.concatenate([np.arange(256), np.arange(256)]).astype(np.uint8)
    x = codes.reshape(1, 1, 256, 2)
    got = oracle.correlate(FMT_CI4, x)
    want = lower(full_matrix(decode_np(x).reshape(1, 1, 512)))
    assert np.array_equal(got, want.astype(np.int64))


def test_python_loop_small():
    # an independent scalar loop with Python complex numbers
    x = synth.uniform_ci4(5, 2, 3, seed=7, lo=-8, hi=7)
    xc = decode_np(x).reshape(5, 2, 6)
    got = oracle.correlate(FMT_CI4, x)
    for c in range(2):
        p = 0
        for i in range(6):
            for j in range(i + 1):
                v = sum(complex(xc[t, c, i]) * complex(xc[t, c, j]).conjugate() for t in range(5))
                assert (got[c, p, 0], got[c, p, 1]) == (int(v.real), int(v.imag))
                p += 1


def test_random_medium_against_full_matrix():
    x = synth.uniform_ci4(97, 3, 20, seed=3, lo=-8, hi=7)
    want = lower(full_matrix(decode_np(x).reshape(97, 3, 40)))
    assert np.array_equal(oracle.correlate(FMT_CI4, x, threads=3), want.astype(np.int64))


# ---------------------------------------------------------- closed forms ---

@pytest.mark.parametrize("byte,value", [(0x10, 1), (0x11, 2), (0xF0, 1), (0x88, 128), (0x77, 98)])
def test_constant_input(byte, value):
    # x = a + jb at every input and time: V_ij = K |x|^2 + 0j for every pair
    k = 37
    x = np.full((k, 2, 4, 2), byte, dtype=np.uint8)
    got = oracle.correlate(FMT_CI4, x)
    assert np.all(got[..., 0] == k * value) and np.all(got[..., 1] == 0)


def test_real_against_imaginary_input():
    # input 0 carries 1, input 1 carries j: V_10 = j * conj(1) = j
    k = 11
    x = np.zeros((k, 1, 1, 2), dtype=np.uint8)
    x[..., 0] = 0x10
    x[..., 1] = 0x01
    got = oracle.correlate(FMT_CI4, x)[0]
    assert got[oracle.pair_index(1, 0)].tolist() == [0, k]
    assert got[oracle.pair_index(0, 0)].tolist() == [k, 0]
    assert got[oracle.pair_index(1, 1)].tolist() == [k, 0]


@pytest.mark.parametrize("amp", [1, 3, 5, 7])
def test_quarter_turn_tone(amp):
    k, nc, ns = 19, 4, 6
    x, q = synth.quarter_turn_tone_ci4(k, nc, ns, seed=amp, amp=amp)
    got = oracle.correlate(FMT_CI4, x)
    unit = {0: (1, 0), 1: (0, 1), 2: (-1, 0), 3: (0, -1)}
    for c in range(nc):
        for i in range(2 * ns):
            for j in range(i + 1):
                re, im = unit[(int(q[c, i]) - int(q[c, j])) % 4]
                p = oracle.pair_index(i, j)
                assert got[c, p, 0] == k * amp * amp * re
                assert got[c, p, 1] == k * amp * amp * im


# ------------------------------------------------------------- invariants ---

def test_autos_real_and_sum_of_squares():
    x = synth.uniform_ci4(64, 3, 5, seed=11, lo=-8, hi=7)
    xc = decode_np(x).reshape(64, 3, 10)
    got = oracle.correlate(FMT_CI4, x)
    for i in range(10):
        p = oracle.pair_index(i, i)
        assert np.all(got[:, p, 1] == 0)
        power = (xc[:, :, i].real ** 2 + xc[:, :, i].imag ** 2).sum(axis=0)
        assert np.array_equal(got[:, p, 0], power.astype(np.int64))
        assert np.all(got[:, p, 0] >= 0)


def test_additive_over_time():
    x = synth.uniform_ci4(50, 2, 4, seed=5)
    whole = oracle.correlate(FMT_CI4, x)
    parts = oracle.correlate(FMT_CI4, x[:17]) + oracle.correlate(FMT_CI4, x[17:])
    assert np.array_equal(whole, parts)


def test_station_permutation_equivariance():
    ns, k = 5, 23
    x = synth.uniform_ci4(k, 2, ns, seed=13, lo=-8, hi=7)
    perm = np.array([3, 0, 4, 2, 1])  # new station s carries old station perm[s]
    xp = x[:, :, perm, :]
    base = oracle.correlate(FMT_CI4, x)
    got = oracle.correlate(FMT_CI4, xp)
    old_of_new = (2 * perm[:, None] + np.arange(2)[None, :]).reshape(-1)
    for c in range(2):
        for i in range(2 * ns):
            for j in range(i + 1):
                a, b = old_of_new[i], old_of_new[j]
                v = got[c, oracle.pair_index(i, j)]
                if a >= b:
                    w = base[c, oracle.pair_index(a, b)]
                    assert v.tolist() == w.tolist()
                else:  # stored the other way round: V_ab = conj(V_ba)
                    w = base[c, oracle.pair_index(b, a)]
                    assert v.tolist() == [w[0], -w[1]]


def test_ci8_matches_ci4():
    x = synth.uniform_ci4(41, 3, 7, seed=17, lo=-8, hi=7)
    assert np.array_equal(oracle.correlate(FMT_CI4, x), oracle.correlate(FMT_CI8, ci4_to_ci8(x)))


def test_ci8_against_full_matrix_full_code_range():
    x = synth.uniform_ci8(29, 2, 6, seed=19)
    assert x.min() == -128 and x.max() == 127
    xc = (x[..., 0].astype(np.int64) + 1j * x[..., 1].astype(np.int64)).reshape(29, 2, 12)
    want = lower(full_matrix(xc))
    assert np.array_equal(oracle.correlate(FMT_CI8, x), want.astype(np.int64))


def test_ci8_extreme_codes():
    k = 65535  # the longest integration whose sums fit in int32 with -128 codes
    x = np.full((k, 1, 1, 2, 2), -128, dtype=np.int8)
    got = oracle.correlate(FMT_CI8, x)[0]
    assert got[:, 0].tolist() == [32768 * k] * 3 and got[:, 1].tolist() == [0] * 3
    assert 32768 * k <= 2**31 - 1 < 32768 * (k + 1)


def test_cf32_integer_valued_is_exact():
    x8 = synth.uniform_ci8(33, 2, 5, seed=23, lo=-127, hi=127)
    got = oracle.correlate(FMT_CF32, x8.astype(np.float32))
    assert got.dtype == np.float64
    assert np.array_equal(got, oracle.correlate(FMT_CI8, x8).astype(np.float64))


def test_cf32_against_full_matrix():
    x = synth.gaussian_cf32(40, 2, 6, seed=29)
    xc = (x[..., 0].astype(np.float64) + 1j * x[..., 1]).reshape(40, 2, 12)
    want = lower(full_matrix(xc))
    got = oracle.correlate(FMT_CF32, x)
    scale = np.abs(want).max()
    assert np.max(np.abs(got - want)) <= 1e-12 * scale


def float_edge_input(seed: int) -> np.ndarray:
    """Gaussian float spectra whose stations sit at magnitudes 2^-135 (every
    sample subnormal), 2^-100, 1 and 2^40, with a few subnormal samples inside
    normal windows."""
    x = synth.gaussian_cf32(50, 2, 8, seed=seed).astype(np.float64)
    scales = np.array([2.0**-135, 2.0**-100, 1.0, 2.0**40] * 2)
    x *= scales[None, None, :, None, None]
    x[3, 0, 2, 1, 0] = 1e-40
    x[7, 1, 6, 0, 1] = -3e-42
    return x.astype(np.float32)


def test_cf32_edge_magnitudes_against_full_matrix():
    # subnormal and very small or large finite inputs: double holds every product exactly
    # enough, so the oracle equals numpy's complex128 brute force to 1e-12 of each entry's
    # Cauchy-Schwarz scale sqrt(V_ii V_jj)
    x = float_edge_input(37)
    assert np.count_nonzero((x != 0) & (np.abs(x) < np.finfo(np.float32).tiny)) > 200
    xc = (x[..., 0].astype(np.float64) + 1j * x[..., 1]).reshape(50, 2, 16)
    want = lower(full_matrix(xc))
    got = oracle.correlate(FMT_CF32, x)
    idx = np.arange(16)
    autos = want[:, idx * (idx + 1) // 2 + idx, 0]
    ii, jj = np.tril_indices(16)
    order = np.argsort(ii * (ii + 1) // 2 + jj)
    scale = np.sqrt(autos[:, ii[order]] * autos[:, jj[order]])
    assert np.all(scale > 0)
    assert np.all(np.abs(got - want).max(axis=-1) <= 1e-12 * scale)


def test_cf32_non_finite_samples_reach_exactly_their_pairs():
    # a NaN or an infinity at (t, c, input) makes the real part of every pair of that input
    # in channel c non-finite (inf * x or NaN), as numpy's complex arithmetic does; every
    # other entry stays finite and equal to the brute force
    x = synth.gaussian_cf32(30, 2, 5, seed=41)
    x[4, 1, 3, 0, 0] = np.nan    # channel 1, input 6
    x[9, 0, 1, 1, 1] = np.inf    # channel 0, input 3
    x[20, 1, 0, 1, 0] = -np.inf  # channel 1, input 1
    got = oracle.correlate(FMT_CF32, x)
    xc = np.empty((30, 2, 10), dtype=np.complex128)  # set apart: 1j * inf would make a NaN real part
    xc.real = x[..., 0].reshape(30, 2, 10)
    xc.imag = x[..., 1].reshape(30, 2, 10)
    with np.errstate(invalid="ignore"):
        want = lower(full_matrix(xc))
    ii, jj = np.tril_indices(10)
    order = np.argsort(ii * (ii + 1) // 2 + jj)
    i, j = ii[order], jj[order]
    bad = {0: {3}, 1: {6, 1}}
    for c in range(2):
        poisoned = np.isin(i, list(bad[c])) | np.isin(j, list(bad[c]))
        assert np.all(~np.isfinite(got[c, poisoned, 0]))
        assert np.all(np.isfinite(got[c, ~poisoned]))
        assert np.allclose(got[c, ~poisoned], want[c, ~poisoned], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("fmt", [FMT_CI4, FMT_CI8, FMT_CF32])
def test_pairs_entry_point(fmt):
    k, nc, ns = 21, 3, 4
    if fmt == FMT_CI4:
        x = synth.uniform_ci4(k, nc, ns, seed=31, lo=-8, hi=7)
    elif fmt == FMT_CI8:
        x = synth.uniform_ci8(k, nc, ns, seed=31)
    else:
        x = synth.gaussian_cf32(k, nc, ns, seed=31)
    full = oracle.correlate(fmt, x)
    trips = [(c, i, j) for c in range(nc) for i in range(2 * ns) for j in range(i + 1)]
    got = oracle.correlate_pairs(fmt, x, np.array(trips))
    want = np.array([full[c, oracle.pair_index(i, j)] for c, i, j in trips])
    assert np.array_equal(got, want)


def test_bad_arguments_rejected():
    x = synth.uniform_ci4(4, 2, 2, seed=1)
    with pytest.raises(RuntimeError):
        oracle.correlate_pairs(FMT_CI4, x, np.array([[0, 1, 2]]))  # j > i
    with pytest.raises(ValueError):
        oracle.correlate(FMT_CI8, x)  # wrong dtype for the format


# ------------------------------------------------------------ statistics ---

def test_uniform_auto_power_expectation():
    # components uniform on [-7, 7]: E[re^2] = E[im^2] = 2 * (1 + 4 + ... + 49) / 15
    k = 4096
    x = synth.uniform_ci4(k, 4, 16, seed=37)
    got = oracle.correlate(FMT_CI4, x)
    autos = np.array([got[:, oracle.pair_index(i, i), 0] for i in range(32)], dtype=np.float64)
    expect = k * 2 * (2 * sum(v * v for v in range(1, 8)) / 15)
    assert abs(autos.mean() / expect - 1) < 0.01


def test_planewave_phase():
    k, nc, ns = 16384, 3, 6
    x = synth.gaussian_planewave_ci4(k, nc, ns, seed=41)
    phi = synth.planewave_phases(nc, ns, seed=41)
    got = oracle.correlate(FMT_CI4, x)
    errs = []
    for c in range(nc):
        for a in range(ns):
            for b in range(a):
                for p in range(2):
                    v = got[c, oracle.pair_index(2 * a + p, 2 * b + p)]
                    d = np.angle(complex(v[0], v[1]) * np.exp(-1j * (phi[c, a] - phi[c, b])))
                    errs.append(abs(d))
    errs = np.array(errs)
    assert errs.mean() < 0.1 and errs.max() < 0.5
