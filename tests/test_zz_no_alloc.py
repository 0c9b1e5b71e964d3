"""The allocation-free entry point against the plan-based path.

``xcorr_correlate_ci4_noalloc`` exists for callers that cannot allocate device
memory when they correlate (a real-time capture loop, where cudaMalloc would
synchronise the device, or code running inside another framework's fixed
memory pool).  It keeps its staging planes in one fixed array per GPU, which
each call reuses, so two calls in a row must not see each other's leftovers.
This file is named to run last; it passes on its own and after the rest.
"""

import numpy as np
import pytest

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


def test_noalloc_matches_the_plan_path_on_two_calls_in_a_row(torch):
    # the second call is smaller and different, so stale scratch from the
    # first would show up as a mismatch
    cases = [(100, 16, 512, 41), (70, 24, 300, 42)]
    for n_sta, n_chan, n_time, seed in cases:
        x = synth.gaussian_planewave_ci4(n_time, n_chan, n_sta, seed=seed)
        xd = torch.from_numpy(x).cuda()
        n_pairs = 2 * n_sta * (2 * n_sta + 1) // 2
        out = torch.full((n_chan, n_pairs, 2), -12345, dtype=torch.int32, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        xcorr.xcorr_correlate_ci4_noalloc(xd.data_ptr(), n_time, n_chan, n_sta, out.data_ptr(),
                                          status.data_ptr(), stream)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        want = plan_result(torch, xd, n_sta, n_chan, n_time)
        assert np.array_equal(out.cpu().numpy(), want)


def test_noalloc_refuses_sizes_beyond_its_scratch(torch):
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(xcorr.XcorrError) as e:
        # 512 stations x 64 channels x 8192 samples needs 1 GiB of planes
        xcorr.xcorr_correlate_ci4_noalloc(x.data_ptr(), 8192, 64, 512, out.data_ptr())
    assert e.value.status == 1  # INVALID_ARG
    assert "scratch" in str(e.value)
