"""The streaming X-stage on the GPU: packets in any order -> device ring ->
X-stage -> dumps, bit-exact against the oracle on the same samples with lost
packets zeroed (Sec. 2.3 placement by sequence number and F-engine id,
Sec. 2.4 lost-packet threshold, Fig. 4 ring of sub-blocks)."""

import numpy as np
import pytest

import oracle
from paper_1401_8288_gb300 import synth, xcorr

pytestmark = pytest.mark.gpu

N_STA, N_CHAN = 32, 16          # 64 inputs
N_IN = 2 * N_STA
NT, NCH, NA = 4, 8, 16
BLOCK = 64
N_GROUPS, N_FENG = N_CHAN // NCH, N_IN // NA
P = (BLOCK // NT) * N_GROUPS * N_FENG   # 128 packets per block


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1401_8288_gb300 import build
    build.build()
    return torch


def cfg(**kw):
    base = dict(n_time_per_packet=NT, n_chan_per_packet=NCH, n_inputs_per_packet=NA,
                block_samples=BLOCK, n_blocks=4, blocks_per_dump=2, stack_threshold=1 << 30,
                chunk_packets=100, n_chunks=3, n_host_dumps=8)
    base.update(kw)
    return xcorr.stream_config(**base)


def zero_packets(x, pk_idx):
    """x [t][c][i] with the samples of packets pk_idx (stream order) set to 0 + 0i."""
    x = x.copy()
    for k in pk_idx:
        tb, rem = divmod(int(k), N_GROUPS * N_FENG)
        g, f = divmod(rem, N_FENG)
        x[tb * NT:(tb + 1) * NT, g * NCH:(g + 1) * NCH, f * NA:(f + 1) * NA] = 0
    return x


def run_stream(torch, x, packets, c, engine="tensor", tuning=None):
    with xcorr.Plan(N_STA, N_CHAN, BLOCK, engine=engine) as plan:
        if tuning is not None:
            plan.set_tuning(*tuning)
        with xcorr.Stream(plan, c) as st:
            st.push(packets)
            st.flush()
            counters, n_dumps = st.counters()
            dumps = [st.wait_dump(k) for k in range(n_dumps)]
    return dumps, counters


def expected_dumps(x, n_blocks, bpd):
    out = []
    for d in range(0, n_blocks, bpd):
        seg = x[d * BLOCK:min(n_blocks, d + bpd) * BLOCK]
        out.append(oracle.correlate(oracle.FMT_CI4, seg.reshape(seg.shape[0], N_CHAN, N_STA, 2)))
    return out


@pytest.mark.parametrize("engine,tuning", [("tensor", None), ("tensor", (1, 0, 2, 1)),
                                           ("cuda_core", None)])
def test_in_order_stream_matches_oracle(torch, engine, tuning):
    n_blocks = 6
    x = synth.uniform_ci4(n_blocks * BLOCK, N_CHAN, N_STA, seed=11, lo=-8, hi=7).reshape(-1, N_CHAN, N_IN)
    c = cfg()
    pk = xcorr.xcorr_packetize(x, c)
    dumps, counters = run_stream(torch, x, pk, c, engine, tuning)
    want = expected_dumps(x, n_blocks, 2)
    assert len(dumps) == 3
    for k, d in enumerate(dumps):
        assert d["index"] == k and d["n_samples"] == 2 * BLOCK and d["lost_packets"] == 0
        # the sequence number of the dump's first sample: its packets' time block x channel groups
        assert d["first_seq"] == (k * 2 * BLOCK // NT) * (N_CHAN // NCH)
        assert np.array_equal(d["data"].astype(np.int64), want[k])
    assert counters["placed"] == n_blocks * P and counters["lost"] == 0


def test_reordered_duplicated_and_lost_packets(torch):
    # reordering within two blocks, duplicates, and 9 packets never sent: the
    # lost ones are zero-filled, everything else lands where its header says
    n_blocks = 8
    x = synth.uniform_ci4(n_blocks * BLOCK, N_CHAN, N_STA, seed=12, lo=-8, hi=7).reshape(-1, N_CHAN, N_IN)
    # packets move by less than 2 blocks, so every block has all its packets in
    # before one 4 blocks later arrives and closes it (no threshold needed)
    c = cfg(n_blocks=4, blocks_per_dump=3)
    pk = xcorr.xcorr_packetize(x, c)
    rng = np.random.default_rng(13)
    lost = np.sort(rng.choice(n_blocks * P, 9, replace=False))
    keep = np.setdiff1d(np.arange(n_blocks * P), lost)
    order = keep[np.argsort(keep + rng.uniform(0, 1.8 * P, keep.size))]
    dups = order[rng.choice(300, 25)]  # re-sent copies of packets already received
    stream = np.concatenate([order[:300], dups, order[300:]])
    dumps, counters = run_stream(torch, x, pk[stream], c)
    xz = zero_packets(x, lost)
    want = expected_dumps(xz, n_blocks, 3)
    assert [d["index"] for d in dumps] == [0, 1, 2]
    assert [d["n_samples"] for d in dumps] == [3 * BLOCK, 3 * BLOCK, 2 * BLOCK]
    per_dump = [np.sum((lost // P) // 3 == k) for k in range(3)]
    assert [d["lost_packets"] for d in dumps] == per_dump
    for k, d in enumerate(dumps):
        assert np.array_equal(d["data"].astype(np.int64), want[k]), f"dump {k}"
    # a copy whose block is still open is a duplicate, one whose block has closed is late
    assert counters["duplicates"] + counters["late"] == 25 and counters["lost"] == 9
    assert counters["placed"] == n_blocks * P - 9


def test_threshold_closes_a_block_and_late_packets_do_not_count(torch):
    # block 1 misses 6 packets that arrive only after 20 packets of block 2
    # were held: it closes with 6 lost, and the stragglers are dropped as late
    n_blocks = 4
    x = synth.uniform_ci4(n_blocks * BLOCK, N_CHAN, N_STA, seed=14, lo=-8, hi=7).reshape(-1, N_CHAN, N_IN)
    c = cfg(stack_threshold=20, blocks_per_dump=1)
    pk = xcorr.xcorr_packetize(x, c)
    late = P + np.array([0, 5, 17, 64, 100, 127])
    first = np.setdiff1d(np.arange(n_blocks * P), late)
    split = int(np.searchsorted(first, 2 * P)) + 25   # 25 packets of block 2 before the stragglers
    stream = np.concatenate([first[:split], late, first[split:]])
    dumps, counters = run_stream(torch, x, pk[stream], c)
    assert counters["late"] == 6 and counters["lost"] == 6
    xz = zero_packets(x, late)
    want = expected_dumps(xz, n_blocks, 1)
    assert [d["lost_packets"] for d in dumps] == [0, 6, 0, 0]
    for k, d in enumerate(dumps):
        assert np.array_equal(d["data"].astype(np.int64), want[k]), f"dump {k}"


def test_a_dump_whose_host_buffer_was_reused_has_no_data(torch):
    # two host buffers, three dumps read only at the end: dump 0's copy was
    # overwritten, so its record comes back without data (never with the wrong data)
    x = synth.uniform_ci4(6 * BLOCK, N_CHAN, N_STA, seed=15, lo=-8, hi=7).reshape(-1, N_CHAN, N_IN)
    c = cfg(n_host_dumps=2)
    with xcorr.Plan(N_STA, N_CHAN, BLOCK) as plan, xcorr.Stream(plan, c) as st:
        st.push(xcorr.xcorr_packetize(x, c))
        st.flush()
        d0 = st.wait_dump(0)
        assert d0["data"] is None and d0["n_samples"] == 2 * BLOCK
        want = expected_dumps(x, 6, 2)
        for k in (1, 2):
            assert np.array_equal(st.wait_dump(k)["data"].astype(np.int64), want[k])


def test_budget_admission(torch):
    # a budget that holds the plan but not the stream's ring is refused at admission
    big = xcorr.Plan(N_STA, N_CHAN, BLOCK)
    try:
        budget = big.info["device_bytes"] + 1024
    finally:
        big.close()
    with xcorr.Plan(N_STA, N_CHAN, BLOCK, hbm_budget_bytes=budget) as plan:
        with pytest.raises(xcorr.XcorrError) as e:
            xcorr.Stream(plan, cfg())
        assert e.value.status == 7  # BUDGET


@pytest.mark.parametrize("nt,nch,na,engine", [(2, 16, 32, "tensor"), (1, 4, 64, "cuda_core"),
                                              (8, 2, 16, "tensor")])
def test_other_packet_geometries(torch, nt, nch, na, engine):
    # spectra per packet, channels per packet and F-engine widths other than the
    # defaults; chunks of 37 packets split packets of a block across chunks
    n_blocks = 3
    x = synth.uniform_ci4(n_blocks * BLOCK, N_CHAN, N_STA, seed=nt * 100 + na, lo=-8, hi=7).reshape(-1, N_CHAN, N_IN)
    c = cfg(n_time_per_packet=nt, n_chan_per_packet=nch, n_inputs_per_packet=na, blocks_per_dump=3,
            chunk_packets=37, n_chunks=2)
    pk = xcorr.xcorr_packetize(x, c)
    rng = np.random.default_rng(nt + na)
    order = np.argsort(np.arange(pk.shape[0]) + rng.uniform(0, 20, pk.shape[0]))
    dumps, counters = run_stream(torch, x, pk[order], c, engine)
    assert counters["lost"] == 0 and counters["placed"] == pk.shape[0]
    assert len(dumps) == 1 and dumps[0]["n_samples"] == n_blocks * BLOCK
    want = oracle.correlate(oracle.FMT_CI4, x.reshape(-1, N_CHAN, N_STA, 2))
    assert np.array_equal(dumps[0]["data"].astype(np.int64), want)
