"""GPU parity of the float (CF32) path at its edges, against the FP64 oracle.

The header's policy for float spectra (Sec. 1: spectra from a GPU F-stage):
no finite input is flushed, results beyond the float range come out
non-finite, and a NaN or infinity poisons exactly the pairs of its input in
its channel.  The tolerance is the float path's own: per entry
|V - V_fp64| <= 1e-6 sqrt(V_ii V_jj), the Cauchy-Schwarz scale of the entry
(a raw relative error is unbounded for cross terms that sum to about zero),
plus 2^-120 for entries whose exact value lies below the normal float range,
where a float result can only be a subnormal or zero.

Every case runs with the input at four placements: 16-byte aligned with an
input count that is a multiple of 32 (the unpack that stages each window in
shared memory and reads it once; the stations are padded with zero stations,
and the original triangle is the first N_i (N_i + 1) / 2 entries of the
padded one), 16-byte aligned otherwise (the two-inputs-per-thread unpack), and
at byte offsets 4 and 8 (the scalar unpack, which reads single floats).
"""

import numpy as np
import pytest

import oracle
from paper_1401_8288_gb300 import synth, xcorr

pytestmark = pytest.mark.gpu

LAYOUTS = ["tile", "aligned", "offset4", "offset8"]
REL = 1e-6
FLOOR = 2.0**-120


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1401_8288_gb300 import build
    build.build()
    return torch


def correlate(torch, x, layout, chunks=None):
    """One integration of x (host float32 [t][c][s][2][2]) on the tensor engine,
    the input placed as layout says; chunks: several executes."""
    n_pairs = (2 * x.shape[2]) * (2 * x.shape[2] + 1) // 2
    if layout == "tile":
        pad = (-x.shape[2]) % 16
        x = np.concatenate([x, np.zeros(x.shape[:2] + (pad,) + x.shape[3:], dtype=x.dtype)], axis=2)
    elif layout == "aligned":
        assert (2 * x.shape[2]) % 32 != 0, "this placement is for input counts the staged unpack does not take"
    n_time, n_chan, n_sta = x.shape[0], x.shape[1], x.shape[2]
    chunks = chunks or [n_time]
    flat = torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).cuda()
    off = {"tile": 0, "aligned": 0, "offset4": 4, "offset8": 8}[layout]
    buf = torch.zeros(flat.numel() + 8, dtype=torch.float32, device="cuda")
    buf[off // 4:off // 4 + flat.numel()] = flat
    base = buf.data_ptr() + off
    assert (base % 16 == 0) == (layout in ("tile", "aligned"))
    row = n_chan * n_sta * 2 * 2 * 4  # bytes of one time sample
    with xcorr.Plan(n_sta, n_chan, max(chunks), fmt="cf32", engine="tensor") as plan:
        t0 = 0
        for k in chunks:
            xcorr.xcorr_execute(plan.handle, base + t0 * row, k, 0)
            t0 += k
        out = plan.dump(stream=0)
        plan.sync(0)
        return out.cpu().numpy().astype(np.float64)[:, :n_pairs]


def pair_axes(n_inputs):
    ii, jj = np.tril_indices(n_inputs)
    order = np.argsort(ii * (ii + 1) // 2 + jj)
    return ii[order], jj[order]


def cs_scale(want, n_inputs):
    """sqrt(V_ii V_jj) of every packed entry, from the FP64 autocorrelations."""
    idx = np.arange(n_inputs)
    autos = want[:, idx * (idx + 1) // 2 + idx, 0]
    i, j = pair_axes(n_inputs)
    return np.sqrt(autos[:, i] * autos[:, j])


def assert_within(got, want, scale, mask=None):
    with np.errstate(invalid="ignore", over="ignore"):
        err = np.abs((got[..., 0] - want[..., 0]) + 1j * (got[..., 1] - want[..., 1]))
        ok = err <= REL * scale + FLOOR
    if mask is not None:
        ok = ok | ~mask
    bad = np.argwhere(~ok)
    assert bad.size == 0, (f"{len(bad)} entries outside the bound, first (channel, pair) {bad[0]}: "
                           f"got {got[tuple(bad[0])]}, want {want[tuple(bad[0])]}")


@pytest.mark.parametrize("layout", LAYOUTS)
def test_gaussian_at_every_placement(torch, layout):
    x = synth.gaussian_cf32(700, 3, 37, seed=5)
    got = correlate(torch, x, layout)
    want = oracle.correlate(oracle.FMT_CF32, x)
    assert_within(got, want, cs_scale(want, 74))


@pytest.mark.parametrize("layout", LAYOUTS)
def test_one_sample_a_million_times_its_neighbours(torch, layout):
    # the spike sets its window's scale: the other samples of that input and window are
    # quantised on a grid 2^20 times coarser, and stay within the bound because the spike
    # also dominates the input's autocorrelation
    x = synth.gaussian_cf32(1000, 2, 40, seed=11)
    x[123, 0, 5, 1] *= np.float32(1e6)
    x[700, 1, 17, 0, 1] = np.float32(-3e6)
    got = correlate(torch, x, layout)
    want = oracle.correlate(oracle.FMT_CF32, x)
    assert_within(got, want, cs_scale(want, 80))
    idx = np.arange(80)
    autos = idx * (idx + 1) // 2 + idx
    assert np.max(np.abs(got[:, autos, 0] / want[:, autos, 0] - 1)) <= REL


@pytest.mark.parametrize("layout", LAYOUTS)
def test_inputs_and_channels_whose_power_differs_by_1e8(torch, layout):
    x = synth.gaussian_cf32(800, 2, 36, seed=12)
    amp = np.array([1e-2, 1.0, 1e2])[np.arange(36) % 3]  # input powers span 1e8
    x *= amp[None, None, :, None, None].astype(np.float32)
    x[:, 1] *= np.float32(1e-4)  # the second channel 1e8 below the first
    got = correlate(torch, x, layout)
    want = oracle.correlate(oracle.FMT_CF32, x)
    assert_within(got, want, cs_scale(want, 72))


def edge_magnitudes(n_time, n_chan, n_sta, seed):
    """Stations at 2^-135 (every sample subnormal), 2^-100 (below the float
    grid of a window clamped at 2^-64), 1 and 2^40; some subnormal samples
    inside normal windows."""
    x = synth.gaussian_cf32(n_time, n_chan, n_sta, seed=seed).astype(np.float64)
    scales = np.array([2.0**-135, 2.0**-100, 1.0, 2.0**40])[np.arange(n_sta) % 4]
    x *= scales[None, None, :, None, None]
    x[5::97, :, 2::4, 0, 1] = 1e-40
    return x.astype(np.float32)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_subnormal_and_tiny_inputs_are_not_flushed(torch, layout):
    # a subnormal input times a 2^40 one is a normal float (about 2^-90); so is a 2^-100
    # input times a 2^40 one, which a flush at 2^-64 would have made zero
    x = edge_magnitudes(900, 2, 24, seed=13)
    assert np.count_nonzero((x != 0) & (np.abs(x) < np.finfo(np.float32).tiny)) > 10000
    got = correlate(torch, x, layout)
    want = oracle.correlate(oracle.FMT_CF32, x)
    assert_within(got, want, cs_scale(want, 48))
    # the entries that carry the small inputs' information are well inside the float range
    i, j = pair_axes(48)
    sta_scale = np.array([-135, -100, 0, 40])[(np.arange(48) // 2) % 4]
    big = (sta_scale[i] == 40) | (sta_scale[j] == 40)
    small = (sta_scale[i] <= -100) | (sta_scale[j] <= -100)
    cross = big & small
    assert np.median(np.abs(want[:, cross, 0])) > 2.0**-100
    assert np.mean(got[:, cross, 0] != 0) > 0.99


@pytest.mark.parametrize("layout", LAYOUTS)
def test_results_beyond_the_float_range_are_non_finite(torch, layout):
    x = synth.gaussian_cf32(512, 1, 12, seed=14).astype(np.float64)
    scales = np.array([1.0, 2.0**50, 2.0**70])[np.arange(12) % 3]
    x *= scales[None, None, :, None, None]
    x = x.astype(np.float32)
    got = correlate(torch, x, layout)
    want = oracle.correlate(oracle.FMT_CF32, x)
    i, j = pair_axes(24)
    sta = (np.arange(24) // 2) % 3
    huge = (sta[i] == 2) & (i == j)            # autocorrelations ~ 2^149: past the float range
    assert np.all(np.abs(want[:, huge, 0]) > 2.0**129)
    assert np.all(~np.isfinite(got[:, huge]).all(axis=-1))
    fine = (sta[i] < 2) & (sta[j] < 2) | ((sta[i] == 2) ^ (sta[j] == 2)) & ((sta[i] == 0) | (sta[j] == 0))
    assert np.all(np.isfinite(got[:, fine]))
    assert_within(got, want, cs_scale(want, 24), mask=np.broadcast_to(fine, got.shape[:2]))


@pytest.mark.parametrize("layout", LAYOUTS)
def test_nan_and_inf_poison_exactly_their_inputs_pairs(torch, layout):
    x = synth.gaussian_cf32(900, 2, 20, seed=15)
    x[10, 1, 3, 0, 0] = np.nan     # channel 1, input 6
    x[500, 0, 7, 1, 1] = np.inf    # channel 0, input 15
    x[899, 1, 0, 1, 0] = -np.inf   # channel 1, input 1, the last sample
    # two executes: the poison of the first stays for the rest of the integration
    got = correlate(torch, x, layout, chunks=[450, 450])
    want = oracle.correlate(oracle.FMT_CF32, x)
    i, j = pair_axes(40)
    bad = {0: [15], 1: [6, 1]}
    for c in range(2):
        poisoned = np.isin(i, bad[c]) | np.isin(j, bad[c])
        assert np.all(np.isnan(got[c, poisoned]))
        assert np.all(~np.isfinite(want[c, poisoned, 0]))
        assert np.all(np.isfinite(got[c, ~poisoned]))
        clean = np.broadcast_to(~poisoned, (1, poisoned.size))
        with np.errstate(invalid="ignore"):
            assert_within(got[c:c + 1], want[c:c + 1], cs_scale(want, 40)[c:c + 1], mask=clean)


def test_poison_ends_with_the_integration_and_survives_the_wide_fold(torch):
    x = synth.gaussian_cf32(384, 1, 8, seed=16)
    y = x.copy()
    y[7, 0, 2, 1, 0] = np.nan  # input 5
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    want = oracle.correlate(oracle.FMT_CF32, x)
    i, j = pair_axes(16)
    poisoned = (i == 5) | (j == 5)
    with xcorr.Plan(8, 1, 384, fmt="cf32") as plan:
        wide = torch.zeros((1, plan.info["n_pairs"], 2), dtype=torch.float64, device="cuda")
        plan.execute(yd)
        plan.dump(out=wide, wide=True, reset=True)  # a poisoned dump folded into double
        plan.execute(xd)
        clean = plan.dump()                         # the next integration is clean
        plan.execute(xd)
        plan.dump(out=wide, wide=True, reset=True)  # the fold keeps the poison
        plan.sync()
    w = wide.cpu().numpy()
    assert np.all(np.isnan(w[0, poisoned])) and np.all(np.isfinite(w[0, ~poisoned]))
    got = clean.cpu().numpy().astype(np.float64)
    assert_within(got, want, cs_scale(want, 16))


def test_misaligned_float_pointer_is_refused(torch):
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    with xcorr.Plan(1, 1, 4, fmt="cf32") as plan:
        with pytest.raises(xcorr.XcorrError) as e:
            xcorr.xcorr_execute(plan.handle, x.data_ptr() + 2, 4, 0)
        assert e.value.status == 1  # INVALID_ARG
