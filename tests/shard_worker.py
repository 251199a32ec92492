"""Worker of the sharding test: one gloo rank docks its LPT shard with the FP64 oracle (test infrastructure)."""
import os

import numpy as np


def worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    import synth
    import synth.configs as C
    from paper_1901_06363_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pk = synth.pocket(8, 48, 0.5, C.ELLIPSOID)
    opk = oracle.OraclePocket(pk)
    l, t = synth.ligand_sizes(41, 9, 0, [16, 30, 0, 5])
    b = synth.ligand_batch(41, l, t)
    kn = C.knobs(n_poses=4, hp_step=30.0, lp_step=30.0, repetitions=1, seed=2)
    dt = np.dtype([("score", np.float64), ("pose", np.int32), ("status", np.int32)])

    def dock_fn(sub, ids):
        r = oracle.dock(opk, sub, kn, ids=ids, nthreads=1)
        out = np.zeros(sub.n, dt)
        out["score"], out["pose"], out["status"] = r["best_score"], r["best_pose"], r["status"]
        return out

    costs = shard.ligand_costs(b, oracle.n_angles(kn["hp_step"]), kn["n_poses"], kn["repetitions"])
    idx, res = shard.dock_shard(b, rank, world, dock_fn, costs)
    full = shard.gather_results(idx, res, b.n)
    if rank == 0:
        whole = dock_fn(b, np.arange(b.n) + b.id_base)
        q.put((full, whole, idx))
    dist.barrier()
    dist.destroy_process_group()


def gpu_worker(rank, world, port, q):
    """One gloo rank docks its LPT shard through the CUDA path (every rank on cuda:0, independent launches)."""
    import torch
    import torch.distributed as dist

    import synth
    import synth.configs as C
    from paper_1901_06363_gb300 import Docker, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    dk = Docker(0)
    pk = synth.pocket(8, 64, 0.5, C.ELLIPSOID)
    pid = dk.init_pocket(pk)
    l, t = synth.ligand_sizes(43, 300, 0, [16, 64, 2, 12])
    b = synth.ligand_batch(43, l, t)
    kn = C.knobs(n_poses=32, hp_step=15.0, lp_step=15.0, repetitions=2, seed=7)

    def dock_fn(sub, ids):
        bid = dk.upload_ligands(sub, ids=ids)
        res, _ = dk.run(bid, [pid], kn, sub.n, int(sub.atom_off[-1]), xyz=False)
        dk.release_batch(bid)
        return res

    costs = shard.ligand_costs(b, 24, kn["n_poses"], kn["repetitions"])
    idx, res = shard.dock_shard(b, rank, world, dock_fn, costs)
    full = shard.gather_results(idx, res, b.n)
    if rank == 0:
        whole = dock_fn(b, np.arange(b.n) + b.id_base)
        q.put((full, whole, idx, float(costs[idx].sum() / costs.sum())))
    dist.barrier()
    dk.close()
    dist.destroy_process_group()
