"""Frequency-parallel sharding on the host: two gloo ranks on CPU.

Each rank owns a contiguous channel band (Sec. 2.1: the X-stage is parallel in
frequency) and correlates it on its own; no visibility data crosses ranks.
Here the per-rank X-stage is the oracle, so this covers the host logic of the
sharded path (bands, barrier, max-over-ranks timing) without a GPU.
"""

import os
import socket

import numpy as np
import pytest

from paper_1401_8288_gb300 import dist


def test_channel_bands_partition_the_band():
    for total in (1, 7, 512, 1000):
        for world in (1, 2, 3, 8):
            if world > total:
                continue
            bands = [dist.channel_band(r, world, total) for r in range(world)]
            assert bands[0][0] == 0 and bands[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
            sizes = [b - a for a, b in bands]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        dist.channel_band(2, 2, 10)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, x, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import oracle
    info = dist.init("gloo")
    c0, c1 = dist.channel_band(info.rank, info.world, x.shape[1])
    vis = oracle.correlate(oracle.FMT_CI4, x, c0=c0, c1=c1, threads=1)
    dist.barrier()
    slowest = dist.max_over_ranks(float(rank + 1))
    total = dist.sum_over_ranks(float(c1 - c0))
    np.save(os.path.join(out_dir, f"vis{rank}.npy"), vis)
    np.save(os.path.join(out_dir, f"stats{rank}.npy"), np.array([slowest, total, c0, c1]))
    import torch.distributed as tdist
    tdist.destroy_process_group()


def test_two_ranks_cover_all_channels(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_1401_8288_gb300 import synth
    oracle.build()
    x = synth.uniform_ci4(40, 7, 6, seed=99)
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, x, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    parts, stats = [], []
    for r in range(2):
        parts.append(np.load(tmp_path / f"vis{r}.npy"))
        stats.append(np.load(tmp_path / f"stats{r}.npy"))
    assert all(s[0] == 2.0 for s in stats)  # max over ranks seen by both
    assert all(s[1] == 7.0 for s in stats)  # every channel owned once
    assert stats[0][3] == stats[1][2]
    whole = oracle.correlate(oracle.FMT_CI4, x)
    assert np.array_equal(np.concatenate(parts), whole)
