"""Host logic of the streaming X-stage, no GPU: the packetizer and the packet
tracker (placement by sequence number and F-engine id, Sec. 2.3 and Fig. 3;
buffers marked full with missing packets recorded lost once the held packets
of later buffers reach a threshold, Sec. 2.4)."""

import numpy as np
import pytest

from paper_1401_8288_gb300 import synth, xcorr

# 64 inputs, 16 channels; packets of 4 samples x 8 channels x 16 inputs
N_IN, N_CHAN = 64, 16
NT, NCH, NA = 4, 8, 16
BLOCK = 32                                   # samples per ring block
N_GROUPS, N_FENG = N_CHAN // NCH, N_IN // NA  # 2 channel groups, 4 F-engines
P = (BLOCK // NT) * N_GROUPS * N_FENG        # 64 packets per block


def cfg(**kw):
    base = dict(n_time_per_packet=NT, n_chan_per_packet=NCH, n_inputs_per_packet=NA,
                block_samples=BLOCK, n_blocks=4, blocks_per_dump=2, stack_threshold=1 << 30,
                chunk_packets=50, n_chunks=3, n_host_dumps=2)
    base.update(kw)
    return xcorr.stream_config(**base)


def samples(n_time, seed=0):
    x = synth.uniform_ci4(n_time, N_CHAN, N_IN // 2, seed=seed, lo=-8, hi=7)
    return x.reshape(n_time, N_CHAN, N_IN)


def header(pk):
    seq = pk[:, :8].copy().view("<u8")[:, 0].astype(np.int64)
    fid = pk[:, 8:12].copy().view("<u4")[:, 0].astype(np.int64)
    return seq, fid


def expected_pidx(seq, fid):
    tblock, grp = seq // N_GROUPS, seq % N_GROUPS
    tl = tblock % (BLOCK // NT)
    return (tl * N_GROUPS + grp) * N_FENG + fid, tblock // (BLOCK // NT)


def test_packetize_round_trip():
    # every sample lands in exactly one packet at the place its header names
    x = samples(3 * BLOCK, seed=1)
    c = cfg()
    pk = xcorr.xcorr_packetize(x, c, first_time_block=5)
    assert pk.shape == (3 * P, 16 + NT * NCH * NA)
    seq, fid = header(pk)
    assert (pk[:, 12:16] == 0).all()
    back = np.zeros_like(x)
    for k in range(pk.shape[0]):
        tb, g = seq[k] // N_GROUPS - 5, seq[k] % N_GROUPS
        pay = pk[k, 16:].reshape(NT, NCH, NA)
        back[tb * NT:(tb + 1) * NT, g * NCH:(g + 1) * NCH, fid[k] * NA:(fid[k] + 1) * NA] = pay
    assert np.array_equal(back, x)
    # F-engine order: time block, channel group, F-engine
    assert np.array_equal(fid[:N_FENG], np.arange(N_FENG))
    assert np.array_equal(seq[:2 * N_FENG], np.repeat(np.arange(5 * N_GROUPS, 5 * N_GROUPS + 2), N_FENG))


def test_in_order_stream_places_every_packet_and_closes_complete_blocks():
    pk = xcorr.xcorr_packetize(samples(3 * BLOCK), cfg())
    with xcorr.Tracker(cfg(), N_IN, N_CHAN) as tr:
        codes, ev = tr.feed(pk)
        seq, fid = header(pk)
        pidx, blk = expected_pidx(seq, fid)
        assert np.array_equal(codes, ((blk % 4) << 40) | pidx)
        # a complete oldest block closes right after its last packet
        closes = [e for e in ev if e["kind"] == xcorr.XCORR_EVENT_CLOSE]
        opens = [e for e in ev if e["kind"] == xcorr.XCORR_EVENT_OPEN]
        assert [(e["block"], e["position"]) for e in opens] == [(0, 0), (1, P), (2, 2 * P)]
        assert [(e["block"], e["position"], e["received"], e["lost"]) for e in closes] == \
            [(b, (b + 1) * P, P, 0) for b in range(3)]
        c = tr.counters()
        assert c["placed"] == 3 * P and c["lost"] == 0 and c["blocks_closed"] == 3
        assert tr.finish() == []


def test_duplicates_are_dropped_once_placed():
    pk = xcorr.xcorr_packetize(samples(BLOCK), cfg())
    dup = pk[[3, 7, 7]]
    with xcorr.Tracker(cfg(), N_IN, N_CHAN) as tr:
        codes, ev = tr.feed(np.concatenate([pk[:10], dup, pk[10:]]))
        assert (codes[10:13] == -1).all() and (codes[:10] >= 0).all() and (codes[13:] >= 0).all()
        assert tr.counters()["duplicates"] == 3
        assert ev[-1]["kind"] == xcorr.XCORR_EVENT_CLOSE and ev[-1]["lost"] == 0


def test_threshold_closes_incomplete_block_and_late_packets_are_dropped():
    # block 0 misses 5 packets; once 7 packets of block 1 are held, block 0 is
    # marked full with 5 lost; the missing ones arriving afterwards are late
    pk = xcorr.xcorr_packetize(samples(2 * BLOCK, seed=2), cfg())
    missing = [2, 9, 30, 31, 63]
    keep0 = [k for k in range(P) if k not in missing]
    order = keep0 + list(range(P, 2 * P)) + missing
    with xcorr.Tracker(cfg(stack_threshold=7), N_IN, N_CHAN) as tr:
        codes, ev = tr.feed(pk[order])
        close0 = [e for e in ev if e["kind"] == xcorr.XCORR_EVENT_CLOSE and e["block"] == 0]
        assert len(close0) == 1
        assert close0[0]["position"] == len(keep0) + 7
        assert close0[0]["received"] == P - 5 and close0[0]["lost"] == 5
        assert (codes[-5:] == -1).all()
        c = tr.counters()
        assert c["late"] == 5 and c["lost"] == 5 and c["placed"] == 2 * P - 5


def test_reordering_within_the_ring_loses_nothing():
    pk = xcorr.xcorr_packetize(samples(4 * BLOCK, seed=3), cfg())
    rng = np.random.default_rng(4)
    order = np.argsort(np.arange(4 * P) + rng.uniform(0, 1.5 * P, 4 * P))  # displacement < 2 blocks
    with xcorr.Tracker(cfg(), N_IN, N_CHAN) as tr:
        codes, ev = tr.feed(pk[order])
        assert (codes >= 0).all()
        closes = [e for e in ev if e["kind"] == xcorr.XCORR_EVENT_CLOSE]
        assert [e["block"] for e in closes] == [0, 1, 2, 3]
        assert all(e["lost"] == 0 for e in closes)
        # blocks close in order, each as soon as it is complete and the one before it closed
        prev = 0
        for e in closes:
            last = np.nonzero(order // P == e["block"])[0].max()
            assert e["position"] == max(last + 1, prev)
            prev = e["position"]
        # the code of every packet still names its own slot and index
        seq, fid = header(pk[order])
        pidx, blk = expected_pidx(seq, fid)
        assert np.array_equal(codes, ((blk % 4) << 40) | pidx)


def test_packet_past_the_ring_closes_the_oldest_blocks():
    # a 2-block ring: a packet of block 3 forces blocks 0 and 1 closed first
    c = cfg(n_blocks=2)
    pk = xcorr.xcorr_packetize(samples(4 * BLOCK, seed=5), c)
    order = list(range(10)) + [3 * P] + [P + 1]
    with xcorr.Tracker(c, N_IN, N_CHAN) as tr:
        codes, ev = tr.feed(pk[order])
        kinds = [(e["kind"], e["block"], e["position"]) for e in ev]
        assert kinds == [(1, 0, 0), (2, 0, 10), (2, 1, 10), (1, 3, 10)]
        assert ev[1]["lost"] == P - 10 and ev[2]["lost"] == P
        assert codes[10] == ((3 % 2) << 40) | expected_pidx(*header(pk[[3 * P]]))[0][0]
        assert codes[11] == -1  # block 1 is closed: late
        fin = tr.finish()
        assert [(e["block"], e["received"]) for e in fin] == [(2, 0), (3, 1)]


def test_bad_fengine_ids_are_counted():
    pk = xcorr.xcorr_packetize(samples(BLOCK), cfg())
    bad = pk[:3].copy()
    bad[:, 8] = N_FENG + 1
    with xcorr.Tracker(cfg(), N_IN, N_CHAN) as tr:
        codes, _ = tr.feed(bad)
        assert (codes == -1).all() and tr.counters()["bad"] == 3


def test_small_event_buffer_gives_the_same_result():
    pk = xcorr.xcorr_packetize(samples(6 * BLOCK, seed=6), cfg(n_blocks=2))
    rng = np.random.default_rng(7)
    sel = np.sort(rng.choice(pk.shape[0], pk.shape[0] - 40, replace=False))
    results = []
    for max_events in (1, 2, 1024):
        with xcorr.Tracker(cfg(n_blocks=2, stack_threshold=20), N_IN, N_CHAN,
                           max_events=max_events) as tr:
            codes, ev = tr.feed(pk[sel])
            ev += tr.finish()
            results.append((codes, [tuple(e.values()) for e in ev], tr.counters()))
    for r in results[:-1]:
        assert np.array_equal(r[0], results[-1][0])
        assert r[1] == results[-1][1]
        assert r[2] == results[-1][2]


@pytest.mark.parametrize("bad", [dict(n_inputs_per_packet=8), dict(n_chan_per_packet=3),
                                 dict(block_samples=30), dict(n_blocks=1), dict(stack_threshold=0),
                                 dict(n_chunks=1)])
def test_invalid_stream_configs_are_rejected(bad):
    with pytest.raises(xcorr.XcorrError) as e:
        xcorr.Tracker(cfg(**bad), N_IN, N_CHAN)
    assert e.value.status == 1


def test_packets_advance_moves_sequence_numbers_only():
    pk = xcorr.xcorr_packetize(samples(BLOCK), cfg())
    moved = pk.copy()
    xcorr.xcorr_packets_advance(moved.ctypes.data, moved.shape[1], moved.shape[0], 12345)
    seq0, fid0 = header(pk)
    seq1, fid1 = header(moved)
    assert np.array_equal(seq1, seq0 + 12345) and np.array_equal(fid1, fid0)
    assert np.array_equal(moved[:, 8:], pk[:, 8:])


def test_a_jump_past_the_event_buffer_still_progresses():
    # a packet 50 blocks ahead needs 48 closes: with room for 5 events per call
    # the tracker emits them over several calls and then places the packet
    pk = xcorr.xcorr_packetize(samples(BLOCK), cfg())
    far = pk[:1].copy()
    xcorr.xcorr_packets_advance(far.ctypes.data, far.shape[1], 1, 50 * (BLOCK // NT) * N_GROUPS)
    with xcorr.Tracker(cfg(n_blocks=2), N_IN, N_CHAN, max_events=5) as tr:
        codes, ev = tr.feed(np.concatenate([pk[:3], far]))
        closes = [e["block"] for e in ev if e["kind"] == xcorr.XCORR_EVENT_CLOSE]
        assert closes == list(range(49))
        assert codes[3] == ((50 % 2) << 40) | 0
        assert tr.counters()["lost"] == 49 * P - 3
