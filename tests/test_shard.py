"""Ligand sharding over ranks: the LPT split, and a two-rank gloo run whose gathered results equal an
unsharded run (the docking on each rank is the FP64 oracle, so this runs without a GPU)."""
import socket

import numpy as np
import pytest

from paper_1901_06363_gb300 import shard


def test_lpt_partition_is_exact_and_balanced():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(0, 1, 1000)
    for world in (1, 2, 3, 8):
        parts = shard.lpt_shards(costs, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(1000))
        loads = np.array([costs[p].sum() for p in parts])
        # Graham's bound for LPT: no rank exceeds the mean load by more than the largest item
        assert loads.max() <= costs.sum() / world + costs.max() + 1e-9


def test_lpt_small_cases():
    assert [list(p) for p in shard.lpt_shards([5, 1, 4, 2], 2)] == [[0, 1], [2, 3]]
    assert [list(p) for p in shard.lpt_shards([1.0], 3)] == [[0], [], []]


def test_fragment_sizes_and_costs():
    import indep
    import synth
    l, t = synth.ligand_sizes(42, 40, 0, [10, 60, 0, 8])
    b = synth.ligand_batch(42, l, t)
    fs = shard.fragment_sizes(b)
    for i in range(b.n):
        x, bonds, rot = indep.ligand(b, i)
        sides = indep.sides(len(x), bonds, rot)
        assert fs[i] == [int(sides[2 * k][0].sum()) for k in range(len(rot))]
    # the cost of a ligand: candidates x (moving atoms + weighted bump pairs) over its sweeps, per pose and repetition
    c = shard.ligand_costs(b, 37, 4, 2)
    for i in range(b.n):
        want = 0.0
        for m in fs[i]:
            r = int(l[i]) - m
            want += (m - 1) + (r - 1) + shard.PAIR_WEIGHT * 2 * (m - 1) * (r - 1)
        assert c[i] == (36 * want + int(l[i])) * 4 * 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_rank_gloo_sharded_equals_unsharded():
    mp = pytest.importorskip("torch.multiprocessing")
    import shard_worker
    q = mp.get_context("spawn").SimpleQueue()
    mp.spawn(shard_worker.worker, args=(2, _free_port(), q), nprocs=2, join=True)
    sharded, whole, idx0 = q.get()
    assert np.array_equal(sharded, whole)
    assert 0 < len(idx0) < 9
