"""Host-side sharding across ranks (CPU only; gloo process groups).

The degridding path splits by whole subgrids with no exchange of data, so
what needs checking without GPUs is the partition (every subgrid owned by
exactly one rank, loads balanced), the per-rank input assembly, and the
cross-rank reductions the benchmark uses (max of step times, sum of counts).
"""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2102_12739_gb300 import shard, synth


def test_partition_covers_every_subgrid_once_and_balances():
    counts = synth.batched_counts(512)
    for world in (1, 2, 3, 8):
        parts = shard.partition_subgrids(counts, world)
        allsub = np.sort(np.concatenate(parts))
        np.testing.assert_array_equal(allsub, np.arange(512))
        loads = np.array([counts[p].sum() for p in parts])
        assert loads.max() - loads.min() <= counts.max()


def test_equal_counts_split_evenly():
    parts = shard.partition_subgrids([250_000] * 128, 2)
    assert [len(p) for p in parts] == [64, 64]


def test_shard_inputs_reassemble_to_the_global_lists():
    w = synth.lines_workload("t", [30, 0, 12, 7, 50])
    parts = shard.partition_subgrids(w.counts(), 2)
    seen = []
    for owned in parts:
        ranges, local = shard.shard_offsets(w.vis_offsets, owned)
        uvw = shard.gather_uvw(w.uvw, ranges)
        assert uvw.shape[0] == local[-1]
        for k, s in enumerate(owned):
            np.testing.assert_array_equal(uvw[local[k]:local[k + 1]],
                                          w.uvw[w.vis_offsets[s]:w.vis_offsets[s + 1]])
            seen.append(int(s))
    assert sorted(seen) == list(range(5))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        counts = synth.batched_counts(64)
        owned = shard.partition_subgrids(counts, world)[rank]
        n_local = int(counts[owned].sum())
        total = shard.sum_over_ranks(n_local)
        step_ms = 1.0 + rank            # a slower rank decides the job time
        worst = shard.max_over_ranks(step_ms)
        out[rank] = (total, worst, len(owned))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_reduce_counts_and_times():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    counts = synth.batched_counts(64)
    for r in range(2):
        total, worst, n_owned = out[r]
        assert total == int(counts.sum())
        assert worst == 2.0
    assert out[0][2] + out[1][2] == 64
