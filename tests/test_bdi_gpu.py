"""Baseline-dependent integration (Sec. 6: per-baseline integration lengths,
longer for short baselines): each 128 x 128 tile pair is integrated over its
own number of base integrations, checked against the oracle summed over
exactly those integrations."""

import ctypes

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


def tile_block(tri, I, J, n_in):
    """Dense [C][128][128][2] block of tile pair (I, J) from a packed triangle."""
    out = np.zeros((tri.shape[0], 128, 128, 2), dtype=np.int64)
    for r in range(128):
        i = I * 128 + r
        if i >= n_in:
            break
        j0, j1 = J * 128, min(i, J * 128 + 127)
        if j1 < j0:
            continue
        p0 = i * (i + 1) // 2 + j0
        out[:, r, :j1 - j0 + 1] = tri[:, p0:p0 + j1 - j0 + 1]
    return out


def tiles_of(nb):
    return [(I, J) for I in range(nb) for J in range(I + 1)]


@pytest.mark.parametrize("n_sta,cadence", [(100, [1, 2, 4]), (150, [3, 1, 2, 2, 4, 1])])
def test_each_tile_pair_integrates_over_its_cadence(torch, n_sta, cadence):
    C, K, steps = 3, 50, 8
    n_in = 2 * n_sta
    tiles = tiles_of((n_in + 127) // 128)
    assert len(tiles) == len(cadence)
    xs = [synth.uniform_ci4(K, C, n_sta, seed=300 + s, lo=-8, hi=7) for s in range(steps)]
    V = [oracle.correlate(oracle.FMT_CI4, x) for x in xs]
    with xcorr.Plan(n_sta, C, K) as plan, xcorr.BDI(plan, cadence) as bdi:
        for s in range(steps):
            plan.execute(torch.from_numpy(xs[s]).cuda())
            blocks, due, smp = bdi.step()
            assert due == [t for t in range(len(cadence)) if (s + 1) % cadence[t] == 0]
            got = blocks.cpu().numpy().astype(np.int64)
            for k, t in enumerate(due):
                m = cadence[t]
                assert smp[k] == m * K
                want = tile_block(sum(V[s - m + 1:s + 1]), *tiles[t], n_in)
                assert np.array_equal(got[k], want), f"step {s}, tile pair {t}"


def test_host_output_and_empty_steps(torch):
    # a step with nothing executed adds nothing; the output may be host memory
    n_sta, C, K = 40, 2, 64
    x = synth.uniform_ci4(K, C, n_sta, seed=7, lo=-8, hi=7)
    with xcorr.Plan(n_sta, C, K) as plan, xcorr.BDI(plan, [2]) as bdi:
        plan.execute(torch.from_numpy(x).cuda())
        _, due, _ = bdi.step()          # step 0: not due
        assert due == []
        host = np.zeros((1, C, 128, 128, 2), dtype=np.int32)
        n, due_c = ctypes.c_int(), (ctypes.c_int * 1)()
        smp = (ctypes.c_int64 * 1)()
        st = xcorr.load().xcorr_bdi_step(bdi.handle, host.ctypes.data, 0, 0, ctypes.byref(n), due_c, smp)
        assert st == 0 and n.value == 1 and smp[0] == K   # step 1 emits one base integration
        torch.cuda.synchronize()
        want = tile_block(oracle.correlate(oracle.FMT_CI4, x), 0, 0, 2 * n_sta)
        assert np.array_equal(host[0].astype(np.int64), want)


def test_a_cadence_past_the_exact_bound_is_refused(torch):
    # int8 sums are exact for 65,535 samples: two base integrations of 40,000 are not
    n_sta, C, K = 8, 1, 40000
    x = synth.uniform_ci8(K, C, n_sta, seed=3)
    with xcorr.Plan(n_sta, C, K, fmt="ci8") as plan, xcorr.BDI(plan, [2]) as bdi:
        xd = torch.from_numpy(x).cuda()
        plan.execute(xd)
        bdi.step()
        plan.execute(xd)
        with pytest.raises(xcorr.XcorrError) as e:
            bdi.step()
        assert e.value.status == 4  # OVERFLOW


def test_invalid_cadences_are_rejected(torch):
    with xcorr.Plan(100, 2, 16) as plan:
        for bad in ([1, 2], [1, 0, 1], [1, 1, 1, 1]):
            with pytest.raises(xcorr.XcorrError) as e:
                xcorr.BDI(plan, bad)
            assert e.value.status == 1
    with xcorr.Plan(10, 2, 16, fmt="cf32") as plan:
        with pytest.raises(xcorr.XcorrError) as e:
            xcorr.BDI(plan, [1])
        assert e.value.status == 2
