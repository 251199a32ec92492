"""Ligand sharding across GPUs (one process per GPU).

(pocket, ligand) pairs are independent (Sec. 3.2: the paper dispatches them
from an MPI master to slaves with no synchronisation), so a database is
split by ligands with no data-path exchange: each rank docks its own shard
with dock_run and only the per-pair results travel, gathered to rank 0.

The split is a greedy longest-processing-time assignment on the work model
of a ligand: n_poses * repetitions * sum over its fragment sweeps of
candidates * (moving atoms + PAIR_WEIGHT * moving-fixed atom pairs), the
sweep's rotations and lookups plus its bump check; ligands in decreasing
cost, each to the currently least-loaded rank. Ligand identity (hence its
seeded initial poses) travels with it, so a sharded run returns exactly the
results of an unsharded one.
"""
from __future__ import annotations

import numpy as np

# Relative cost of one (moving, fixed) atom pair of the bump check against one moving-atom rotation and
# lookup: the exact circle bound rejects most pairs at one test per sweep, and the rest cost a few FP32
# operations per candidate, so a pair weighs a fraction of a lookup.
PAIR_WEIGHT = 0.1


def fragment_sizes(batch):
    """Per ligand, the atom count of the side of each rotatable bond that holds its lower atom index
    (Alg. 1's left fragment), from one depth-first search per ligand: removing a bridge splits a ligand into
    the subtree below it and the rest."""
    out = []
    for b in range(batch.n):
        a0, a1 = int(batch.atom_off[b]), int(batch.atom_off[b + 1])
        l = a1 - a0
        bonds = batch.bonds[batch.bond_off[b]:batch.bond_off[b + 1]]
        adj = [[] for _ in range(l)]
        for u, v in bonds:
            adj[int(u)].append(int(v))
            adj[int(v)].append(int(u))
        parent = [-1] * l
        order, seen, stack = [], [False] * l, [0]
        seen[0] = True
        while stack:
            x = stack.pop()
            order.append(x)
            for y in adj[x]:
                if not seen[y]:
                    seen[y] = True
                    parent[y] = x
                    stack.append(y)
        size = [1] * l
        for x in reversed(order):
            if parent[x] >= 0:
                size[parent[x]] += size[x]
        left = []
        for e in batch.rot[batch.rot_off[b]:batch.rot_off[b + 1]]:
            u, v = sorted(int(a) for a in bonds[int(e)])
            below = v if parent[v] == u else u  # the bond's atom on the far side from atom 0
            left.append(l - size[below] if below == v else size[below])
        out.append(left)
    return out


def ligand_costs(batch, n_angles_hp: int, n_poses: int, repetitions: int) -> np.ndarray:
    """Work model per ligand: poses x repetitions x sum over the 2T sweeps of candidates x (moving atoms +
    PAIR_WEIGHT x bump pairs). A bond whose sides hold m and l - m atoms gives the sweeps m - 1 and l - m - 1
    moving atoms and (m - 1)(l - m - 1) bump pairs each."""
    l, _ = batch.sizes()
    cost = np.zeros(batch.n)
    for b, left in enumerate(fragment_sizes(batch)):
        c = 0.0
        for m in left:
            r = int(l[b]) - m
            c += (m - 1) + (r - 1) + PAIR_WEIGHT * 2 * (m - 1) * (r - 1)
        cost[b] = (n_angles_hp - 1) * c + int(l[b])
    return cost * n_poses * max(repetitions, 1)


def lpt_shards(costs, world: int):
    """Greedy longest-processing-time split of items with the given costs over `world` ranks.

    Returns one sorted index array per rank; every item appears exactly once."""
    costs = np.asarray(costs, np.float64)
    order = np.argsort(-costs, kind="stable")
    load = np.zeros(world)
    parts = [[] for _ in range(world)]
    for i in order:
        r = int(np.argmin(load))
        parts[r].append(int(i))
        load[r] += costs[i]
    return [np.array(sorted(p), np.int64) for p in parts]


def gather_results(local_idx, local_res, n_total: int, group=None):
    """Gather each rank's (ligand indices, structured results) to rank 0 and scatter them back into
    one array in ligand order. Returns the array on rank 0, None elsewhere."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    payload = (np.asarray(local_idx, np.int64), np.asarray(local_res))
    objs = [None] * world if rank == 0 else None
    dist.gather_object(payload, objs, dst=0, group=group)
    if rank != 0:
        return None
    out = np.zeros(n_total, dtype=local_res.dtype)
    seen = np.zeros(n_total, bool)
    for idx, res in objs:
        assert not seen[idx].any(), "a ligand was docked on two ranks"
        out[idx] = res
        seen[idx] = True
    assert seen.all(), "a ligand was docked on no rank"
    return out


def dock_shard(batch, rank: int, world: int, dock_fn, costs=None):
    """Dock this rank's shard: dock_fn(sub_batch, ids) -> per-ligand results (structured array).

    ids are the ligands' global ids (batch.id_base + index), which seed their initial poses."""
    if costs is None:
        costs = np.ones(batch.n)
    idx = lpt_shards(costs, world)[rank]
    sub = batch.subset(idx)
    return idx, dock_fn(sub, idx + batch.id_base)
