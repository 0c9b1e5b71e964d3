"""The allocation-free entry point against the oracle and the plan-based path.

``xcorr_correlate_ci4_noalloc`` exists for callers that cannot allocate device
memory when they correlate (a real-time capture loop, where cudaMalloc would
synchronise the device, or code running inside another framework's fixed
memory pool).  It keeps its staging planes in one fixed array per GPU, which
each call reuses, so two calls in a row must not see each other's leftovers.
This file is named to run last; it passes on its own and after the rest.
"""

import numpy as np
import pytest

import oracle
from paper_1401_8288_gb300 import synth, xcorr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1401_8288_gb300 import build
    build.build()
    return torch


def plan_result(torch, xd, n_sta, n_chan, n_time):
    with xcorr.Plan(n_sta, n_chan, n_time, fmt="ci4", engine="tensor") as plan:
        plan.execute(xd)
        out = plan.dump()
        plan.sync()
    return out.cpu().numpy()


def noalloc_result(torch, xd, n_sta, n_chan, n_time):
    n_pairs = 2 * n_sta * (2 * n_sta + 1) // 2
    out = torch.full((n_chan, n_pairs, 2), -12345, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    xcorr.xcorr_correlate_ci4_noalloc(xd.data_ptr(), n_time, n_chan, n_sta, out.data_ptr(),
                                      status.data_ptr(), stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return out.cpu().numpy()


# (stations, channels, samples, seed): 200 inputs take the byte-wise unpack; 128 inputs with a
# 16-byte aligned buffer take the 128-bit unpack, twice with the same shape and new data, so
# that planes left from the first call would change the second result
CASES = [(100, 16, 512, 41), (64, 8, 1024, 42), (64, 8, 1024, 43)]


def test_noalloc_matches_the_oracle_and_the_plan_on_calls_in_a_row(torch):
    for n_sta, n_chan, n_time, seed in CASES:
        x = synth.gaussian_planewave_ci4(n_time, n_chan, n_sta, seed=seed)
        xd = torch.from_numpy(x).cuda()
        assert xd.data_ptr() % 16 == 0
        got = noalloc_result(torch, xd, n_sta, n_chan, n_time)
        assert np.array_equal(got.astype(np.int64), oracle.correlate(oracle.FMT_CI4, x)), (n_sta, seed)
        assert np.array_equal(got, plan_result(torch, xd, n_sta, n_chan, n_time)), (n_sta, seed)


def test_noalloc_refuses_sizes_beyond_its_scratch(torch):
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(xcorr.XcorrError) as e:
        # 512 stations x 64 channels x 8192 samples needs 1 GiB of planes
        xcorr.xcorr_correlate_ci4_noalloc(x.data_ptr(), 8192, 64, 512, out.data_ptr())
    assert e.value.status == 1  # INVALID_ARG
    assert "scratch" in str(e.value)
    with pytest.raises(xcorr.XcorrError) as e:
        # a station count whose input count would overflow an int is refused before any arithmetic
        xcorr.xcorr_correlate_ci4_noalloc(x.data_ptr(), 1, 1, 2**30 + 1, out.data_ptr())
    assert e.value.status == 1
