"""GPU parity: the CUDA library (through the C ABI) against the oracle.

Integer inputs must match bit for bit.  Sizes span several 128 x 128 tensor
tiles (and 64 x 64 CUDA-core tiles) with ragged input and time tails; the
full-size workloads are checked on sampled channels and sampled pairs, which
the oracle computes one by one.
"""

import numpy as np
import pytest

import oracle
from paper_1401_8288_gb300 import synth, xcorr

pytestmark = pytest.mark.gpu

ENGINES = ["tensor", "cuda_core"]


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1401_8288_gb300 import build
    build.build()
    return torch


def run(torch, x, engine, fmt="ci4", n_time=None, chunks=None, tuning=None):
    """Correlate x (host array) with one plan; optionally in several executes."""
    n_time = x.shape[0] if n_time is None else n_time
    n_sta, n_chan = x.shape[2], x.shape[1]
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    max_t = n_time if chunks is None else max(chunks)
    with xcorr.Plan(n_sta, n_chan, max_t, fmt=fmt, engine=engine) as plan:
        if tuning is not None:
            plan.set_tuning(*tuning)
        if chunks is None:
            plan.execute(xd)
        else:
            t0 = 0
            for k in chunks:
                plan.execute(xd[t0:t0 + k])
                t0 += k
        out = plan.dump()
        plan.sync()
        got = out.cpu().numpy()
        return (got if fmt == "cf32" else got.astype(np.int64)), plan.samples


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("n_sta,n_chan,n_time", [
    (1, 1, 1), (1, 2, 5), (3, 2, 33), (8, 1, 128), (32, 3, 129), (64, 2, 256),
    (70, 3, 300), (100, 2, 200), (136, 2, 131), (200, 1, 385)])
def test_small_shapes_bit_exact(torch, engine, n_sta, n_chan, n_time):
    x = synth.uniform_ci4(n_time, n_chan, n_sta, seed=n_sta * 1000 + n_time, lo=-8, hi=7)
    got, n = run(torch, x, engine)
    assert n == n_time
    want = oracle.correlate(oracle.FMT_CI4, x)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


@pytest.mark.parametrize("engine", ENGINES)
def test_odd_input_count_not_multiple_of_16(torch, engine):
    # 2 * 9 = 18 inputs: the unpack and the loaders take their unaligned paths
    x = synth.uniform_ci4(77, 3, 9, seed=5, lo=-8, hi=7)
    got, _ = run(torch, x, engine)
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


@pytest.mark.parametrize("engine", ENGINES)
def test_extreme_codes(torch, engine):
    # every sample -8 - 8j: the largest per-sample products
    k = 1000
    x = np.full((k, 2, 70, 2), 0x88, dtype=np.uint8)
    got, _ = run(torch, x, engine)
    assert np.all(got[..., 0] == 128 * k) and np.all(got[..., 1] == 0)


@pytest.mark.parametrize("engine", ENGINES)
def test_quarter_turn_tone(torch, engine):
    x, q = synth.quarter_turn_tone_ci4(257, 2, 66, seed=9, amp=7)
    got, _ = run(torch, x, engine)
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


@pytest.mark.parametrize("engine", ENGINES)
def test_integration_over_several_executes(torch, engine):
    chunks = [200, 77, 256, 1]
    x = synth.uniform_ci4(sum(chunks), 2, 70, seed=13, lo=-8, hi=7)
    got, n = run(torch, x, engine, chunks=chunks)
    assert n == sum(chunks)
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


def test_tensor_window_drain_beyond_2_24_partial_sums(torch):
    # 140,000 samples, mostly -8 - 8j (|x|^2 = 128) with 7 - 2j (|x|^2 = 53,
    # odd) every 101st sample: the autocorrelations pass 2^24, where FP32
    # cannot hold odd increments, so the kernel must drain windows into int32.
    k = 140000
    x = np.full((k, 1, 8, 2), 0x88, dtype=np.uint8)
    x[::101] = 0x7E
    want = oracle.correlate(oracle.FMT_CI4, x)
    assert want[0, 0, 0] > 2**24
    got, _ = run(torch, x, "tensor")
    assert np.array_equal(got, want)


@pytest.mark.parametrize("engine", ENGINES)
def test_dump_reset_and_wide_fold(torch, engine):
    x = synth.uniform_ci4(96, 2, 40, seed=21, lo=-8, hi=7)
    want = oracle.correlate(oracle.FMT_CI4, x)
    xd = torch.from_numpy(x).cuda()
    with xcorr.Plan(40, 2, 96, engine=engine) as plan:
        wide = torch.zeros((2, plan.info["n_pairs"], 2), dtype=torch.int64, device="cuda")
        plan.execute(xd)
        a = plan.dump(reset=False)                      # keep integrating
        plan.dump(out=wide, wide=True, reset=True)      # fold into int64, restart
        plan.execute(xd)
        plan.execute(xd)
        plan.dump(out=wide, wide=True, reset=True)      # + two more passes
        empty = plan.dump()                             # nothing since the reset
        plan.sync()
        assert np.array_equal(a.cpu().numpy(), want)
        assert np.array_equal(wide.cpu().numpy(), 3 * want)
        assert np.all(empty.cpu().numpy() == 0)
        host = np.zeros_like(want, dtype=np.int32)
        plan.execute(xd)
        n = xcorr.xcorr_dump(plan.handle, host.ctypes.data, False, xcorr.XCORR_DUMP_RESET, 0)
        plan.sync(0)
        torch.cuda.synchronize()
        assert n == 96 and np.array_equal(host, want)


@pytest.mark.parametrize("fmt,engine", [("ci4", "tensor"), ("ci4", "cuda_core"), ("ci8", "tensor"),
                                        ("ci8", "cuda_core"), ("cf32", "tensor")])
def test_resume_an_integration_from_a_dump(torch, fmt, engine):
    # checkpoint / restart: a dump taken without reset (to host memory), loaded into a new plan,
    # continues the integration; the result is the uninterrupted one, bit for bit
    x = {"ci4": lambda: synth.uniform_ci4(300, 3, 40, seed=91, lo=-8, hi=7),
         "ci8": lambda: synth.uniform_ci8(300, 3, 40, seed=92),
         "cf32": lambda: synth.gaussian_cf32(300, 3, 40, seed=93)}[fmt]()
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    with xcorr.Plan(40, 3, 200, fmt=fmt, engine=engine) as a:
        a.execute(xd[:120])
        ck = torch.zeros((3, a.info["n_pairs"], 2), dtype=a._out_dtype(False)).pin_memory()
        a.dump(out=ck, reset=False)
        a.execute(xd[120:])
        whole = a.dump(reset=True)
        a.sync()
        n_ck = 120
        # the plan holds nothing after the reset dump: a load is accepted, a second one is not
        a.accum_load(ck, n_ck)
        with pytest.raises(xcorr.XcorrError):
            a.accum_load(ck, n_ck)
    with xcorr.Plan(40, 3, 200, fmt=fmt, engine=engine) as b:
        with pytest.raises(xcorr.XcorrError):
            b.accum_load(ck, -1)
        with pytest.raises(xcorr.XcorrError):
            b.accum_load(ck, b.info["max_integration"] + 1)
        b.accum_load(ck, n_ck)
        b.execute(xd[120:])
        got = b.dump(reset=True)
        b.sync()
        assert b.samples == 300
    assert np.array_equal(got.cpu().numpy(), whole.cpu().numpy())
    if fmt == "cf32":
        e, _ = normalised_error(got.cpu().numpy(), oracle.correlate(oracle.FMT_CF32, x), 80)
        assert e.max() <= 1e-6, e.max()
    else:
        assert np.array_equal(got.cpu().numpy(), oracle.correlate(oracle.FMT_CI4 if fmt == "ci4" else oracle.FMT_CI8, x))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("fmt", ["ci4", "ci8"])
def test_input_at_any_byte_offset(torch, engine, fmt):
    # a time slice of a larger buffer starts at an arbitrary byte: the kernels
    # take their unaligned paths and stay exact (4-bit on the tensor engine: the
    # planes path, as the fused kernel needs 16-byte alignment; int8: the
    # element-wise unpack into BF16 planes)
    n_time, n_chan, n_sta = 50, 2, 32
    if fmt == "ci4":
        x = synth.uniform_ci4(n_time, n_chan, n_sta, seed=31, lo=-8, hi=7)
    else:
        x = synth.uniform_ci8(n_time, n_chan, n_sta, seed=31)
    raw = x.view(np.uint8).reshape(-1)
    for off in (1, 2, 4, 8):
        buf = torch.zeros(raw.size + 64, dtype=torch.uint8, device="cuda")
        buf[off:off + raw.size] = torch.from_numpy(raw).cuda()
        with xcorr.Plan(n_sta, n_chan, n_time, fmt=fmt, engine=engine) as plan:
            xcorr.xcorr_execute(plan.handle, buf.data_ptr() + off, n_time, 0)
            got = plan.dump(stream=0).cpu().numpy().astype(np.int64)
            plan.sync(0)
        want = oracle.correlate(oracle.FMT_CI4 if fmt == "ci4" else oracle.FMT_CI8, x)
        assert np.array_equal(got, want), off


@pytest.mark.parametrize("n_chan", [500, 700])
def test_tensor_channel_groups(torch, n_chan):
    # 256 inputs (3 tile pairs per channel): 500 channels run as 2 groups of
    # 250 and 700 channels as 3 groups (234, 234, 232), unpack and X
    # overlapping on the plan's internal streams
    x = synth.uniform_ci4(64, n_chan, 128, seed=n_chan, lo=-8, hi=7)
    got, _ = run(torch, x, "tensor")
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


@pytest.mark.parametrize("engine", ENGINES)
def test_execute_dump_fused_and_plain(torch, engine):
    x = synth.uniform_ci4(200, 3, 70, seed=77, lo=-8, hi=7)
    y = synth.uniform_ci4(200, 3, 70, seed=78, lo=-8, hi=7)
    want_x = oracle.correlate(oracle.FMT_CI4, x)
    want_y = oracle.correlate(oracle.FMT_CI4, y)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    with xcorr.Plan(70, 3, 200, engine=engine) as plan:
        a = plan.execute_dump(xd)                 # fused: straight into the output
        b = plan.execute_dump(yd)                 # fused again: nothing leaks from x
        plan.execute(xd)                          # an integration in progress ...
        c = plan.execute_dump(yd)                 # ... so this one is execute + dump
        d = plan.execute_dump(xd, reset=False)    # not reset: execute + dump, keeps integrating
        e = plan.dump()
        host = np.zeros_like(want_x, dtype=np.int32)
        n = xcorr.xcorr_execute_dump(plan.handle, yd.data_ptr(), 200, host.ctypes.data, False,
                                     xcorr.XCORR_DUMP_RESET, 0)  # host output: execute + dump
        plan.sync()
        torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy(), want_x)
    assert np.array_equal(b.cpu().numpy(), want_y)
    assert np.array_equal(c.cpu().numpy(), want_x + want_y)
    assert np.array_equal(d.cpu().numpy(), want_x) and np.array_equal(e.cpu().numpy(), want_x)
    assert n == 200 and np.array_equal(host, want_y)


def test_ci8_cuda_core_full_code_range(torch):
    x = synth.uniform_ci8(150, 3, 37, seed=23)  # includes -128
    got, _ = run(torch, x, "cuda_core", fmt="ci8")
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI8, x))


def test_ci8_extreme_codes_at_the_int32_bound(torch):
    # 65,535 samples of -128 - 128j: Re = 32768 * K = 2^31 - 32768, the largest exact sum
    k = 65535
    x = np.full((k, 1, 1, 2, 2), -128, dtype=np.int8)
    got, _ = run(torch, x, "cuda_core", fmt="ci8")
    assert np.all(got[..., 0] == 32768 * k) and np.all(got[..., 1] == 0)


def test_errors_are_reported_not_raised_on_device(torch):
    x = torch.zeros((16, 1, 4, 2), dtype=torch.uint8, device="cuda")
    with xcorr.Plan(4, 1, 16, fmt="ci4") as plan:
        with pytest.raises(xcorr.XcorrError) as e:
            xcorr.xcorr_execute(plan.handle, x.data_ptr(), 17, 0)  # n_time > max
        assert e.value.status == 1
        with pytest.raises(xcorr.XcorrError) as e:
            xcorr.xcorr_execute(plan.handle, x.data_ptr(), 0, 0)   # an empty execute
        assert e.value.status == 1
        # an empty integration dumps as zeros, with zero samples
        empty = torch.ones((1, 36, 2), dtype=torch.int32, device="cuda")
        assert xcorr.xcorr_dump(plan.handle, empty.data_ptr(), True, xcorr.XCORR_DUMP_RESET, 0) == 0
        plan.sync()
        assert int(empty.abs().sum()) == 0
        with pytest.raises(xcorr.XcorrError):
            xcorr.xcorr_dump(plan.handle, 0, True, 0, 0)
        with pytest.raises(xcorr.XcorrError):
            xcorr.xcorr_dump(plan.handle, x.data_ptr(), False, xcorr.XCORR_DUMP_ADD_WIDE, 0)
    with xcorr.Plan(1, 1, 40000, fmt="ci8", engine="cuda_core") as plan:
        y = torch.zeros((40000, 1, 1, 2, 2), dtype=torch.int8, device="cuda")
        plan.execute(y)
        with pytest.raises(xcorr.XcorrError) as e:
            plan.execute(y)  # 80,000 samples would pass the exact int32 bound
        assert e.value.status == 4
        plan.dump(reset=True)
        plan.execute(y)  # fine after the reset
        plan.sync()


def test_budget_and_query(torch):
    with pytest.raises(xcorr.XcorrError) as e:
        xcorr.Plan(256, 64, 2048, hbm_budget_bytes=1 << 20)
    assert e.value.status == 7
    with xcorr.Plan(256, 64, 2048) as plan:
        info = plan.query()
        assert info["n_inputs"] == 512 and info["n_pairs"] == 131328
        assert info["engine"] == xcorr.XCORR_ENGINE_TENSOR
        assert info["max_integration"] == 16777215
        assert info["output_bytes"] == 64 * 131328 * 8


def test_auto_engine_and_default_shape_follow_the_measured_rule(torch):
    # AUTO: CUDA-core only at most 16 channels, below 16 inputs for 4-bit, up to 64 inputs for int8
    cases = [((4, 8, 1024, "ci4"), xcorr.XCORR_ENGINE_CUDA_CORE), ((4, 16, 256, "ci8"), xcorr.XCORR_ENGINE_CUDA_CORE),
             ((8, 8, 1024, "ci4"), xcorr.XCORR_ENGINE_TENSOR), ((4, 17, 64, "ci4"), xcorr.XCORR_ENGINE_TENSOR),
             ((32, 16, 1024, "ci8"), xcorr.XCORR_ENGINE_CUDA_CORE), ((33, 16, 1024, "ci8"), xcorr.XCORR_ENGINE_TENSOR),
             ((32, 17, 1024, "ci8"), xcorr.XCORR_ENGINE_TENSOR), ((2, 4, 64, "cf32"), xcorr.XCORR_ENGINE_TENSOR)]
    for (ns, nc, nt, fmt), engine in cases:
        with xcorr.Plan(ns, nc, nt, fmt=fmt, engine="auto") as plan:
            assert plan.query()["engine"] == engine, (ns, nc, nt, fmt)
    # a 4-bit plan's first shape: the small-problem layout for N_i <= 64 with K >= 1024 or C >= 256
    for (ns, nc, nt), shape in [((32, 64, 1024), 10), ((8, 256, 256), 10), ((32, 64, 256), 4),
                                ((256, 64, 2048), 4), ((40, 64, 2048), 4)]:
        with xcorr.Plan(ns, nc, nt, engine="tensor") as plan:
            assert plan.query()["tuning"]["stage_variant"] == shape, (ns, nc, nt)
    # and the answers stay the oracle's on the CUDA-core side of the rule
    x = synth.uniform_ci4(1024, 8, 4, seed=81, lo=-8, hi=7)
    got, _ = run(torch, x, "auto")
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))
    y = synth.uniform_ci8(1024, 16, 32, seed=82)
    got, _ = run(torch, y, "auto", fmt="ci8")
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI8, y))


# -------------------------------------------------- int8 on tensor cores ---

@pytest.mark.parametrize("n_sta,n_chan,n_time", [(1, 2, 7), (37, 3, 150), (70, 2, 1000), (136, 2, 385)])
def test_ci8_tensor_bit_exact(torch, n_sta, n_chan, n_time):
    # full code range with -128; K beyond one 384-sample window drains int32 sums
    x = synth.uniform_ci8(n_time, n_chan, n_sta, seed=n_sta + n_time)
    got, _ = run(torch, x, "tensor", fmt="ci8")
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI8, x))


def test_ci8_tensor_extreme_codes_at_the_int32_bound(torch):
    k = 65535
    x = np.full((k, 1, 4, 2, 2), -128, dtype=np.int8)
    got, _ = run(torch, x, "tensor", fmt="ci8")
    assert np.all(got[..., 0] == 32768 * k) and np.all(got[..., 1] == 0)


def test_ci8_tensor_gaussian_sigma20(torch):
    x = synth.gaussian_ci8(512, 4, 128, seed=14018288 + 3)
    got, _ = run(torch, x, "tensor", fmt="ci8")
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI8, x))


# --------------------------------------------------------- float input ---

def normalised_error(got, want, n_inputs):
    """|V - V_fp64| / sqrt(V_ii V_jj): the error scaled by the Cauchy-Schwarz
    bound of each entry (a raw relative error is unbounded for cross terms
    that happen to sum to about zero)."""
    idx = np.arange(n_inputs)
    autos = want[:, idx * (idx + 1) // 2 + idx, 0]  # [C][N]
    ii, jj = np.tril_indices(n_inputs)
    order = np.argsort(ii * (ii + 1) // 2 + jj)
    scale = np.sqrt(autos[:, ii[order]] * autos[:, jj[order]])
    err = np.abs((got[..., 0] - want[..., 0]) + 1j * (got[..., 1] - want[..., 1]))
    return err / scale, np.abs(got[:, idx * (idx + 1) // 2 + idx, 0] / autos - 1)


@pytest.mark.parametrize("n_sta,n_chan,n_time", [(1, 1, 3), (37, 2, 129), (70, 3, 700), (256, 2, 4096)])
def test_cf32_tensor_within_1e6_of_fp64(torch, n_sta, n_chan, n_time):
    x = synth.gaussian_cf32(n_time, n_chan, n_sta, seed=n_sta * 7 + n_time)
    got, _ = run(torch, x, "tensor", fmt="cf32")
    want = oracle.correlate(oracle.FMT_CF32, x)
    e, e_auto = normalised_error(got.astype(np.float64), want, 2 * n_sta)
    assert e.max() <= 1e-6, e.max()
    assert e_auto.max() <= 1e-6, e_auto.max()


def test_cf32_integer_valued_is_exact(torch):
    # integer-valued floats have exact pieces and exact short sums
    x8 = synth.uniform_ci8(300, 2, 50, seed=5, lo=-127, hi=127)
    got, _ = run(torch, x8.astype(np.float32), "tensor", fmt="cf32")
    assert np.array_equal(got.astype(np.float64), oracle.correlate(oracle.FMT_CI8, x8).astype(np.float64))


def test_cf32_wide_fold_into_double(torch):
    x = synth.gaussian_cf32(256, 2, 40, seed=8)
    want = oracle.correlate(oracle.FMT_CF32, x)
    xd = torch.from_numpy(x).cuda()
    with xcorr.Plan(40, 2, 256, fmt="cf32") as plan:
        wide = torch.zeros((2, plan.info["n_pairs"], 2), dtype=torch.float64, device="cuda")
        for _ in range(3):
            plan.execute(xd)
            plan.dump(out=wide, wide=True, reset=True)
        plan.sync()
    e, _ = normalised_error(wide.cpu().numpy() / 3.0, want, 80)
    assert e.max() <= 1e-6


# ------------------------------------------------------ tuning shapes ---

@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("groups,x_streams", [(1, 1), (2, 1), (3, 2), (8, 2)])
def test_every_launch_shape_is_exact(torch, variant, groups, x_streams):
    # 96 stations: N_i = 192 is a multiple of 16, so the planes path is forced
    x = synth.uniform_ci4(333, 9, 96, seed=variant * 10 + groups, lo=-8, hi=7)
    got, _ = run(torch, x, "tensor", tuning=(variant, groups, x_streams, 1))
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
@pytest.mark.parametrize("n_sta,n_chan,n_time", [(8, 1, 1), (8, 2, 65), (64, 3, 300), (72, 2, 257),
                                                 (200, 2, 385), (256, 3, 1000)])
def test_fused_4bit_kernel_bit_exact(torch, variant, n_sta, n_chan, n_time):
    # N_i a multiple of 16: the unpack runs inside the X kernel (raw bytes
    # decoded on chip to offset E4M3 codes); ragged input blocks and time tails
    x = synth.uniform_ci4(n_time, n_chan, n_sta, seed=variant * 1000 + n_sta + n_time, lo=-8, hi=7)
    got, _ = run(torch, x, "tensor", tuning=(variant, 0, 2, 0))
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


@pytest.mark.parametrize("unfused", [0, 1])
def test_fused_and_planes_paths_agree_over_several_executes(torch, unfused):
    chunks = [128, 77, 300, 5]
    x = synth.uniform_ci4(sum(chunks), 4, 96, seed=31, lo=-8, hi=7)
    got, n = run(torch, x, "tensor", chunks=chunks, tuning=(1, 0, 2, unfused))
    assert n == sum(chunks)
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


@pytest.mark.parametrize("variant", [7, 8, 9])
@pytest.mark.parametrize("n_sta,n_chan,n_time", [(288, 2, 130), (320, 1, 64), (392, 2, 200), (512, 1, 96)])
def test_pair_kernel_every_tile_count(torch, variant, n_sta, n_chan, n_time):
    # The CTA-pair kernel groups a channel's tile pairs by column tile: 5 tiles
    # (15 tile pairs: one entry keeps a single, one pair is transposed), 5 full
    # tiles, 7 tiles with a 16-input last tile (a column half wholly past the
    # inputs), 8 tiles (two transposed tile pairs).
    x = synth.uniform_ci4(n_time, n_chan, n_sta, seed=variant * 100 + n_sta, lo=-8, hi=7)
    got, _ = run(torch, x, "tensor", tuning=(variant, 0, 2, 0))
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


@pytest.mark.parametrize("n_sta", [256, 392])
def test_pair_kernel_accumulates_over_executes(torch, n_sta):
    # later executes add into the accumulator, transposed tile pairs included
    chunks = [96, 300, 7]
    x = synth.uniform_ci4(sum(chunks), 2, n_sta, seed=n_sta + 1, lo=-8, hi=7)
    got, n = run(torch, x, "tensor", chunks=chunks, tuning=(7, 0, 2, 0))
    assert n == sum(chunks)
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


FUSED_BLOCK = 37248  # samples per exactly-summed block of the fused kernel


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
@pytest.mark.parametrize("pattern", ["max", "extremes"])
def test_fused_exact_across_blocks_at_the_bound(torch, variant, pattern):
    # Two full blocks and a tail.  "max": every sample 7 + 7i, so each block's
    # offset sums reach 450 T, the largest the FP32 accumulator holds exactly;
    # "extremes": components drawn from {-8, 7}.
    n_time, n_chan, n_sta = 2 * FUSED_BLOCK + 77, 2, 16
    shape = (n_time, n_chan, n_sta, 2)
    if pattern == "max":
        x = synth.pack_ci4(np.full(shape, 7), np.full(shape, 7))
    else:
        rng = np.random.default_rng(variant + 5)
        x = synth.pack_ci4(np.where(rng.random(shape) < 0.5, -8, 7), np.where(rng.random(shape) < 0.5, -8, 7))
    got, n = run(torch, x, "tensor", tuning=(variant, 0, 2, 0))
    assert n == n_time
    want = oracle.correlate(oracle.FMT_CI4, x)
    if pattern == "max":
        assert (want[..., 0] == 98 * n_time).all() and (want[..., 1] == 0).all()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n_sta,n_chan,n_time", [
    (8, 37, 1000),   # 16 inputs: 8 channels per tile, a ragged last group of 5
    (16, 9, 640),    # 32 inputs: 4 per tile
    (24, 7, 513),    # 48 inputs: 2 per tile (rows 96-127 of each tile unused), a ragged stage
    (32, 64, 1024),  # 64 inputs: 2 per tile, the small field-system-sized workload
    (32, 3, 4096),   # few tiles: 32 stages split over the SMs
    (100, 2, 1100),  # 200 inputs: no packing, 3 tile pairs per channel, time split
])
def test_small_problem_layout_bit_exact(torch, n_sta, n_chan, n_time):
    # Shape 10: channels packed side by side into one 128-row tile (N_i <= 64) and each
    # tile's stages split over the SMs, the split items adding their sums atomically
    x = synth.uniform_ci4(n_time, n_chan, n_sta, seed=n_sta * 31 + n_chan, lo=-8, hi=7)
    got, _ = run(torch, x, "tensor", tuning=(10, 0, 2, 0))
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


def test_small_problem_layout_over_several_executes_and_execute_dump(torch):
    chunks = [300, 128, 77]
    x = synth.uniform_ci4(sum(chunks), 10, 16, seed=91, lo=-8, hi=7)
    got, n = run(torch, x, "tensor", chunks=chunks, tuning=(10, 0, 2, 0))
    assert n == sum(chunks)
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))
    # execute_dump into the caller's buffer: split items clear it first, every call
    y = synth.uniform_ci4(512, 10, 16, seed=92, lo=-8, hi=7)
    yd = torch.from_numpy(y).cuda()
    with xcorr.Plan(16, 10, 512) as plan:
        plan.set_tuning(10, 0, 2, 0)
        out = torch.full((10, plan.info["n_pairs"], 2), 99, dtype=torch.int32, device="cuda")
        for _ in range(2):
            plan.execute_dump(yd, out)
        plan.sync()
    assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, y))


@pytest.mark.parametrize("engine,tuning", [("tensor", (4, 0, 2, 0)), ("tensor", (10, 0, 2, 0)),
                                           ("cuda_core", None)])
def test_execute_dump_replayed_from_a_cuda_graph(torch, engine, tuning):
    # one execute_dump recorded in a CUDA graph (the way small problems are driven without a
    # host call per integration); replays read the input buffer in place
    sizes = (32, 12, 512)  # 64 inputs, 12 channels: packed in the small layout, time split
    x, y = (synth.uniform_ci4(sizes[2], sizes[1], sizes[0], seed=s, lo=-8, hi=7) for s in (61, 62))
    xd = torch.from_numpy(x).cuda()
    with xcorr.Plan(sizes[0], sizes[1], sizes[2], engine=engine) as plan:
        if tuning is not None:
            plan.set_tuning(*tuning)
        out = torch.zeros((sizes[1], plan.info["n_pairs"], 2), dtype=torch.int32, device="cuda")
        plan.execute_dump(xd, out)  # warm-up outside the capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            plan.execute_dump(xd, out)
        out.fill_(-1)
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, x))
        xd.copy_(torch.from_numpy(y).cuda())
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, y))
        plan.sync()


def test_fused_falls_back_for_unaligned_input(torch):
    # a pointer that is not 16-byte aligned takes the planes path, same result
    x = synth.uniform_ci4(100, 2, 64, seed=3, lo=-8, hi=7)
    raw = x.reshape(-1)
    buf = torch.zeros(raw.size + 32, dtype=torch.uint8, device="cuda")
    buf[3:3 + raw.size] = torch.from_numpy(raw).cuda()
    with xcorr.Plan(64, 2, 100) as plan:
        xcorr.xcorr_execute(plan.handle, buf.data_ptr() + 3, 100, 0)
        got = plan.dump(stream=0).cpu().numpy().astype(np.int64)
        plan.sync(0)
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_every_launch_shape_ci8(torch, variant):
    x = synth.uniform_ci8(500, 5, 70, seed=variant)
    got, _ = run(torch, x, "tensor", fmt="ci8", tuning=(variant, 2, 2))
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI8, x))


def test_autotune_keeps_results_exact(torch):
    x = synth.uniform_ci4(256, 64, 128, seed=12, lo=-8, hi=7)
    xd = torch.from_numpy(x).cuda()
    with xcorr.Plan(128, 64, 256) as plan:
        plan.execute(xd)  # an integration in progress is discarded by the autotuner
        best, ms = plan.autotune(xd)
        assert 0 <= best["stage_variant"] <= 10 and 1 <= best["groups"] <= 8 and ms > 0
        assert plan.query()["samples_integrated"] == 0
        assert plan.query()["tuning"]["stage_variant"] == best["stage_variant"]
        plan.execute(xd)
        got = plan.dump().cpu().numpy()
        plan.sync()
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


# ------------------------------------------------------------- batches ---

def batch_inputs(sizes, seed):
    return [synth.uniform_ci4(nt, nc, ns, seed=seed + k, lo=-8, hi=7)
            for k, (ns, nc, nt) in enumerate(sizes)]


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_batch_uneven_subarrays_bit_exact(torch, variant):
    # uneven station, channel and sample counts, ragged tiles, one launch
    sizes = [(8, 3, 512), (70, 2, 200), (200, 1, 385), (1, 4, 33), (140, 2, 1024)]
    xs = batch_inputs(sizes, 100 * variant)
    with xcorr.Batch(sizes) as batch:
        batch.set_variant(variant)
        outs = batch.execute([torch.from_numpy(x).cuda() for x in xs])
        batch.sync()
        for x, o in zip(xs, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, x))


def test_batch_graph_replay(torch):
    sizes = [(16, 2, 256), (64, 3, 512), (100, 1, 128)]
    xs = batch_inputs(sizes, 7)
    ys = batch_inputs(sizes, 8)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    with xcorr.Batch(sizes) as batch:
        batch.capture(xd)
        for _ in range(3):
            outs = batch.replay()
        batch.sync()
        for x, o in zip(xs, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, x))
        for dst, y in zip(xd, ys):  # the graph reads the same buffers: new data, new result
            dst.copy_(torch.from_numpy(y).cuda())
        outs = batch.replay()
        batch.sync()
        for y, o in zip(ys, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, y))


# every input count a multiple of 16 (ragged 128-input tiles at 144, 400, 272), time tails
FUSABLE = [(8, 3, 512), (72, 2, 200), (200, 1, 385), (24, 4, 33), (136, 2, 1024), (256, 1, 96)]


@pytest.mark.parametrize("variant", [3, 4, 5])
def test_fused_batch_bit_exact(torch, variant):
    xs = batch_inputs(FUSABLE, 300 + variant)
    with xcorr.Batch(FUSABLE) as batch:
        batch.set_variant(variant)
        outs = batch.execute([torch.from_numpy(x).cuda() for x in xs])
        batch.sync()
        for x, o in zip(xs, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, x))


def test_fused_batch_is_the_default_and_replays_new_data(torch):
    sizes = FUSABLE[:4]
    xs, ys = batch_inputs(sizes, 41), batch_inputs(sizes, 42)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    with xcorr.Batch(sizes) as batch:
        batch.capture(xd)
        outs = batch.replay()
        batch.sync()
        for x, o in zip(xs, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, x))
        for dst, y in zip(xd, ys):  # the fused kernel reads the inputs in place
            dst.copy_(torch.from_numpy(y).cuda())
        outs = batch.replay()
        batch.sync()
        for y, o in zip(ys, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, y))


def test_batch_a_shape_per_subarray(torch):
    # shared classes of the tensor-memory-A shapes (4, 5, 6) and subarrays launched alone (the
    # CTA-pair kernel 8, the small-problem layout 10, the shared-memory kernel 1), all on their
    # own streams, in an execute and in a graph
    variants = [4, 5, 6, 8, 10, 1]
    xs, ys = batch_inputs(FUSABLE, 500), batch_inputs(FUSABLE, 501)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    with xcorr.Batch(FUSABLE) as batch:
        batch.set_subarray_variants(variants)
        assert batch.subarray_variants() == variants
        outs = batch.execute(xd)
        batch.sync()
        for x, o in zip(xs, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, x))
        batch.capture(xd)
        for dst, y in zip(xd, ys):
            dst.copy_(torch.from_numpy(y).cuda())
        outs = batch.replay()
        batch.sync()
        for y, o in zip(ys, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, y))
        with pytest.raises(xcorr.XcorrError):
            batch.set_subarray_variants([4, 4, 4, 11, 4, 4])  # 11 is no plan shape
        batch.set_variant(4)  # batch-wide shape 4: plan shape 5 for every subarray
        assert batch.subarray_variants() == [5] * len(FUSABLE)


def test_batch_autotune_per_subarray_and_its_cache(torch, tmp_path):
    import json
    sizes = FUSABLE[:3]
    xs = batch_inputs(sizes, 600)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    xcorr.xcorr_tuning_cache_clear()
    with xcorr.Batch(sizes) as batch:
        picked = batch.autotune(xd)
        assert all(0 <= v <= 10 for v in picked) and batch.subarray_variants() == picked
        outs = batch.execute(xd)
        batch.sync()
        for x, o in zip(xs, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.int64), oracle.correlate(oracle.FMT_CI4, x))
    path = tmp_path / "tuning.jsonl"
    assert xcorr.xcorr_tuning_cache_save(str(path)) == 3
    entries = [json.loads(line) for line in path.read_text().splitlines()]
    assert {(e["n_inputs"], e["n_channels"], e["n_time"]) for e in entries} == \
        {(2 * ns, nc, nt) for ns, nc, nt in sizes}
    assert all(e["scope"] == "batch" for e in entries)
    # a fresh process state with the file loaded: the same shapes without timing
    xcorr.xcorr_tuning_cache_clear()
    assert xcorr.xcorr_tuning_cache_load(str(path)) == (3, 0)
    with xcorr.Batch(sizes) as batch:
        assert batch.autotune(xd) == picked
    xcorr.xcorr_tuning_cache_clear()


def test_plan_autotune_through_the_cache(torch):
    x = synth.uniform_ci4(256, 8, 32, seed=71, lo=-8, hi=7)
    xd = torch.from_numpy(x).cuda()
    xcorr.xcorr_tuning_cache_clear()
    with xcorr.Plan(32, 8, 256) as plan:
        best, ms, hit = plan.autotune(xd, cached=True)
        assert not hit and ms > 0
    with xcorr.Plan(32, 8, 256) as plan:
        best2, ms2, hit2 = plan.autotune(xd, cached=True)
        assert hit2 and best2 == best and ms2 == pytest.approx(ms, abs=1e-3)
        plan.execute(xd)
        got = plan.dump().cpu().numpy()
        plan.sync()
    assert np.array_equal(got.astype(np.int64), oracle.correlate(oracle.FMT_CI4, x))
    xcorr.xcorr_tuning_cache_clear()


def test_fused_shapes_refused_for_batches_they_do_not_fit(torch):
    with xcorr.Batch([(70, 2, 200)]) as batch:  # 140 inputs: not a multiple of 16
        with pytest.raises(xcorr.XcorrError) as e:
            batch.set_variant(3)
        assert e.value.status == 2  # UNSUPPORTED
        with pytest.raises(xcorr.XcorrError) as e:
            batch.set_subarray_variants([4])
        assert e.value.status == 2
        batch.set_variant(0)


def test_batch_rejects_what_it_does_not_serve(torch):
    with pytest.raises(xcorr.XcorrError):
        xcorr.Batch([(8, 2, 200000)])  # more than one window per execute


# ------------------------------------------------- full-size workloads ---

def sample_check(got, x, fmt, channels, n_pairs_sample, seed):
    """Whole triangles of a few channels, then single pairs across all channels."""
    for c in channels:
        want = oracle.correlate(fmt, x, c0=c, c1=c + 1)[0]
        assert np.array_equal(got[c], want), f"channel {c}"
    rng = np.random.default_rng(seed)
    n_chan, ni = got.shape[0], int((np.sqrt(8 * got.shape[1] + 1) - 1) / 2)
    i = rng.integers(0, ni, size=n_pairs_sample)
    j = (rng.random(n_pairs_sample) * (i + 1)).astype(np.int64)
    c = rng.integers(0, n_chan, size=n_pairs_sample)
    trips = np.stack([c, i, j], axis=1)
    want = oracle.correlate_pairs(fmt, x, trips)
    assert np.array_equal(got[c, i * (i + 1) // 2 + j], want)


@pytest.mark.parametrize("engine", ENGINES)
def test_workload_64_inputs_64_channels_1024_samples(torch, engine):
    # 32 stations x 2 pols, 64 channels, K = 1024, uniform [-7, 7]: checked whole
    x = synth.uniform_ci4(1024, 64, 32, seed=14018288 + 1)
    got, _ = run(torch, x, engine)
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))


@pytest.fixture(scope="module")
def workload_512():
    # 256 stations x 2 pols, 512 channels, K = 2048, Gaussian sigma 2.5 + plane wave
    return synth.gaussian_planewave_ci4(2048, 512, 256, seed=14018288 + 2)


@pytest.mark.parametrize("engine,tuning", [
    ("tensor", (1, 0, 2, 0)),   # the shared-memory fused kernel's shapes
    ("tensor", (0, 0, 2, 0)), ("tensor", (3, 0, 2, 0)),
    ("tensor", (4, 0, 2, 0)), ("tensor", (5, 0, 2, 0)), ("tensor", (6, 0, 2, 0)),  # A in tensor memory
    ("tensor", (7, 0, 2, 0)), ("tensor", (8, 0, 2, 0)), ("tensor", (9, 0, 2, 0)),  # CTA pairs
    ("tensor", (10, 0, 2, 0)),  # the small-problem layout (at this size: neither packed nor split)
    ("tensor", (0, 1, 1, 1)),   # the planes path
    ("cuda_core", None)])
def test_workload_512_inputs_512_channels_2048_samples(torch, workload_512, engine, tuning):
    got, _ = run(torch, workload_512, engine, tuning=tuning)
    sample_check(got, workload_512, oracle.FMT_CI4, channels=[0, 137, 511], n_pairs_sample=400,
                 seed=3)


@pytest.mark.parametrize("variant", [4, 8, 10])
def test_workload_512_execute_dump_into_the_callers_buffer(torch, workload_512, variant):
    # The benchmark's timed call: one execute_dump with reset into a device buffer the caller
    # owns, which the fused kernel writes directly (no accumulator copy).  Twice in a row into
    # the same buffer: the second call must store, not add.  Shape 4 is the default kernel
    # (A operand in tensor memory), 8 the CTA-pair kernel.
    xd = torch.from_numpy(np.ascontiguousarray(workload_512)).cuda()
    with xcorr.Plan(256, 512, 2048) as plan:
        plan.set_tuning(variant, 0, 2, 0)
        out = torch.full((512, plan.info["n_pairs"], 2), -77, dtype=torch.int32, device="cuda")
        for _ in range(2):
            plan.execute_dump(xd, out)
        assert plan.samples == 2048
        plan.sync()
        assert plan.query()["samples_integrated"] == 0
    got = out.cpu().numpy().astype(np.int64)
    sample_check(got, workload_512, oracle.FMT_CI4, channels=[0, 255, 511], n_pairs_sample=400,
                 seed=5 + variant)


@pytest.mark.parametrize("variant", [1, 10])
def test_workload_512_host_to_host(torch, workload_512, variant):
    # the benchmark's end-to-end call: pinned host input and output, channel groups pipelined
    # (each group's launch reads a channel slice of rows that hold all channels)
    with xcorr.Plan(256, 512, 2048) as plan:
        plan.set_tuning(variant, 0, 2, 0)
        xh = torch.from_numpy(np.ascontiguousarray(workload_512)).pin_memory()
        out = plan.execute_dump_host(xh)
        plan.sync()
        got = out.numpy().astype(np.int64)
    sample_check(got, workload_512, oracle.FMT_CI4, channels=[5, 300], n_pairs_sample=400, seed=4)


@pytest.mark.parametrize("fmt,n_sta,n_chan,n_time,n_groups", [
    ("ci4", 64, 13, 300, 0), ("ci4", 72, 9, 129, 4), ("ci4", 8, 3, 65, 8), ("ci4", 70, 4, 100, 0),
    ("ci8", 32, 5, 200, 0)])
def test_host_to_host_execute_matches_oracle(torch, fmt, n_sta, n_chan, n_time, n_groups):
    # channel groups copied up, correlated and copied down in a pipeline (the
    # fused 4-bit path); other inputs (70 stations: N_i not a multiple of 16,
    # int8) take the one-piece path; either way the result is the oracle's
    gen = synth.uniform_ci4 if fmt == "ci4" else synth.uniform_ci8
    x = gen(n_time, n_chan, n_sta, seed=n_sta + n_time)
    with xcorr.Plan(n_sta, n_chan, n_time, fmt=fmt) as plan:
        xh = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        out = plan.execute_dump_host(xh, n_groups=n_groups)
        plan.sync()
        got = out.numpy().astype(np.int64)
        # the plan holds nothing afterwards: a second call gives the same answer
        out2 = plan.execute_dump_host(xh, n_groups=n_groups)
        plan.sync()
    want = oracle.correlate(oracle.FMT_CI4 if fmt == "ci4" else oracle.FMT_CI8, x)
    assert np.array_equal(got, want)
    assert np.array_equal(out2.numpy().astype(np.int64), want)


def test_a_stalled_wait_is_reported_and_the_context_survives(torch):
    # a wait that can never complete gives up after the 2 s limit and turns the
    # plan's status to DEVICE; nothing faults, and a new plan works as before
    import time
    x = synth.uniform_ci4(16, 1, 8, seed=9, lo=-8, hi=7)
    xd = torch.from_numpy(x).cuda()
    with xcorr.Plan(8, 1, 16) as plan:
        t0 = time.perf_counter()
        xcorr.xcorr_watchdog_selftest(plan.handle, 0)
        with pytest.raises(xcorr.XcorrError) as e:
            plan.sync(0)
        assert e.value.status == 6
        assert time.perf_counter() - t0 > 1.0
        with pytest.raises(xcorr.XcorrError) as e:
            plan.execute(xd)  # the plan refuses work until destroyed
        assert e.value.status == 6
    got, _ = run(torch, x, "tensor")
    assert np.array_equal(got, oracle.correlate(oracle.FMT_CI4, x))
