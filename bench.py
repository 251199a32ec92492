"""Benchmark of batched pose evaluation: docked ligands/s and pose-evals/s on GB300.

Workload: 1,024 synthetic ligands (16-64 atoms, 2-12 rotatable bonds) x one
64^3 pocket at 0.5 Å; 64 initial poses, 10 degree step, 4 repetitions, bump
threshold 2.0 Å, nearest-voxel score, FP32. A step docks the whole batch
(every (ligand, pose) through the full greedy sweep, best pose per ligand).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--scaling weak|strong]

Prints one JSON line. Under torchrun each rank docks its own 1,024 ligands
(weak scaling, no collective on the data path); rank 0 prints the line.
--scaling strong splits the one workload over the ranks (LPT on the work
model) and gathers its results. --impl reference times the FP64 CPU oracle
(the reference arm) on the host. Besides the headline workload the line
carries the other workloads (single ligand, a knob-sweep point,
differentiation, multi-pocket), each batched against the plain form, the
roofline of the sweep kernel by its algorithmic work
(FP32 operations, field gathers of feasible candidates, HBM bytes), and the
oracle on bounded samples of each workload (16 host cores and one).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "docked ligands/s & pose-evals/s, batched vs plain, 1 GB300, score err <=1e-4 rel"
UNIT = "ligands/s"
WORKLOAD = "batched: 1024 ligands (16-64 atoms, 2-12 rotatable bonds) x 1 pocket 64^3 @0.5A, 64 poses, 10 deg, 4 reps"


# DRAM bytes (read + write) of one sweep launch on this workload, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the kernel
# code whose sha256 (comments and blank lines removed) has this prefix;
# reported as null for any other code.
NCU_TRAFFIC = {"kernel_code_sha256": "5eb6084cdc90ce8c", "bytes": 2527232 + 6656}


def kernel_code_sha(src=None):
    """sha256 prefix of the sweep kernel's source (or of src) without comments and blank lines."""
    import hashlib
    import re
    if src is None:
        with open(os.path.join(ROOT, "paper_1901_06363_gb300", "csrc", "geodock_kernels.cuh")) as f:
            src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = "\n".join(ln.split("//")[0].rstrip() for ln in src.splitlines())
    src = "\n".join(ln for ln in src.splitlines() if ln.strip())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def _traffic():
    return NCU_TRAFFIC["bytes"] if kernel_code_sha() == NCU_TRAFFIC["kernel_code_sha256"] else None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload(rank=0):
    import synth.configs as C
    pks, batch, kn = C.batched()
    if rank:
        # weak scaling: every rank docks its own 1,024 ligands of the same distribution
        import synth
        l, t = synth.ligand_sizes(1, 1024, 0, [16, 64, 2, 12], id0=1024 * rank)
        batch = synth.ligand_batch(1, l, t, id0=1024 * rank)
    return pks[0], batch, kn


def repeat_batch(batch, k):
    """k copies of a batch, one after another, with ids continuing past the batch (each copy docks new poses)."""
    import synth
    na, nb = int(batch.atom_off[-1]), int(batch.bond_off[-1])
    nr = int(batch.rot_off[-1])
    cat = lambda off, tot: np.concatenate([off[:-1] + i * tot for i in range(k)] + [off[-1:] + (k - 1) * tot])  # noqa: E731
    return synth.LigandBatch(cat(batch.atom_off, na), cat(batch.bond_off, nb), cat(batch.rot_off, nr),
                             np.tile(batch.xyz, (k, 1)), np.tile(batch.bonds, (k, 1)), np.tile(batch.rot, k),
                             id_base=batch.id_base)


def input_bytes(batch):
    return sum(a.nbytes for a in (batch.atom_off, batch.xyz, batch.bond_off, batch.bonds, batch.rot_off, batch.rot))


def cpu_baseline(pk, batch, kn, target_s=12.0):
    """The FP64 oracle as it stands, on the host cores, over a bounded sample of the workload's ligands."""
    import oracle
    opk = oracle.OraclePocket(pk)
    cores = os.cpu_count() or 1
    done, elapsed, start = 0, 0.0, 0
    chunk = 2 * cores
    while elapsed < target_s and start < batch.n:
        idx = np.arange(start, min(start + chunk, batch.n))
        sub = batch.subset(idx)
        t0 = time.perf_counter()
        oracle.dock(opk, sub, kn, nthreads=cores, ids=idx + batch.id_base)
        elapsed += time.perf_counter() - t0
        done += len(idx)
        start += len(idx)
    return {"value": done / elapsed, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {done} of the {batch.n} workload ligands, all 64 poses each ({elapsed:.1f} s)"}


def sweep_nmov(batch):
    """Moving atoms (the fragment minus its bond atom) of every fragment sweep of each ligand, in sweep order
    (per rotatable bond: the left fragment, then the right one; Alg. 1)."""
    from paper_1901_06363_gb300 import shard
    l, _ = batch.sizes()
    out = []
    for b, left in enumerate(shard.fragment_sizes(batch)):
        out.append(np.array([v for m in left for v in (m - 1, int(l[b]) - m - 1)], np.int64))
    return out


def feasible_work(dk, bid, pid, kn, batch):
    """Exact work counts of the batched run, from a traced run of the same batch and knobs: the trace records
    every repetition, and those after a pose's first repetition without a commit (a fixed point, which the
    batched run does not compute) are dropped here. Returns evaluated and feasible candidates, and their
    moving-atom lookups (Alg. 1 scores only the feasible candidates)."""
    import torch
    bufs, _, pmax, _ = dk.run_trace_device(bid, pid, kn, batch)
    N, R = int(kn["n_poses"]), int(kn["repetitions"])
    _, t = batch.sizes()
    nsw = R * 2 * t.astype(np.int64)
    total = int((nsw * N).sum())
    st = bufs["cand_status"][:total * pmax].view(total, pmax)[:, 1:]
    feas = (st == 1).sum(1).cpu().numpy()
    ev = (st != -2).sum(1).cpu().numpy()
    ck = bufs["chosen_k"][:total].cpu().numpy()
    live = bufs["pose_status"][:batch.n * N].cpu().numpy() == 0
    del bufs, st
    torch.cuda.empty_cache()
    nmov = sweep_nmov(batch)
    c = dict(candidates=0, feasible=0, lookups=0, feasible_lookups=0)
    s0 = 0
    for b in range(batch.n):
        ns = int(t[b]) * 2
        n = N * R * ns
        if ns == 0 or R == 0:
            continue
        moved = (ck[s0:s0 + n].reshape(N, R, ns) != 0).any(2)
        still = ~moved
        first = np.where(still.any(1), still.argmax(1), R - 1)
        comp = (np.arange(R)[None, :] <= first[:, None]) & live[b * N:(b + 1) * N, None]
        m = np.broadcast_to(comp[:, :, None], (N, R, ns)).ravel()
        w = np.tile(nmov[b], N * R)
        f, e = feas[s0:s0 + n][m], ev[s0:s0 + n][m]
        c["candidates"] += int(e.sum())
        c["feasible"] += int(f.sum())
        c["lookups"] += int((e * w[m]).sum())
        c["feasible_lookups"] += int((f * w[m]).sum())
        s0 += n
    return c


def roofline_8d(st, fw, sweep_s, rates, traffic, hbm_gbs):
    """Roofline of the sweep kernel by the algorithmic work per pose-eval (candidate): FP32 operations
    6 m (rotation) + (m - 1)(l - m - 1) x 3 (bump test, every pair at every candidate: 2 FMA + 1 compare) +
    m (score adds) + 1 (the division), counted as lane operations at the measured FMA rate; field gathers
    m per feasible candidate at the measured texture-fetch rate; HBM bytes at the copy bandwidth. The bound is
    the resource whose time at its peak is largest; frac = that time / the measured kernel time."""
    placements = st["atom_updates"] + st["lookups_skipped"]
    fp32 = 7.0 * placements + 3.0 * st["bump_pairs"] + st["candidates"]
    t_fp32 = fp32 / rates["fma_per_s"]
    t_tex = fw["feasible_lookups"] / rates["tex_local_per_s"]
    t_hbm = (traffic or 0) / (hbm_gbs * 1e9)
    res = {
        "fp32": {"work": fp32, "unit": "lane-ops", "peak": rates["fma_per_s"], "time_s": t_fp32,
                 "achieved": fp32 / sweep_s, "frac": t_fp32 / sweep_s},
        "texture": {"work": fw["feasible_lookups"], "unit": "fetches", "peak": rates["tex_local_per_s"],
                    "time_s": t_tex, "achieved": fw["feasible_lookups"] / sweep_s, "frac": t_tex / sweep_s},
        "hbm": {"work": traffic, "unit": "bytes", "peak": hbm_gbs * 1e9, "time_s": t_hbm,
                "achieved": (traffic or 0) / sweep_s, "frac": t_hbm / sweep_s},
    }
    bound = max(res, key=lambda r: res[r]["time_s"])
    return bound, res


def _device_time(fn, torch, stream, reps=3):
    """Median CUDA-event time (s) of fn() on `stream` over `reps` runs, after one warm-up run."""
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return float(np.median(ts))


def leg_single(dk, torch, stream):
    """One ligand x one pocket (24 atoms, 4 rotatable bonds, 48^3, 8 poses, 10 degrees, 1 repetition)."""
    import synth.configs as C
    pks, b, kn = C.single()
    pid = dk.init_pocket(pks[0])
    bid = dk.upload_ligands(b)
    natoms = int(b.atom_off[-1])
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    xyz = torch.empty(natoms * 3, dtype=torch.float32, device="cuda")
    t = _device_time(lambda: dk.run(bid, [pid], kn, 1, natoms, out=out, xyz_out=xyz, stream=stream), torch, stream, 20)
    cand = dk.stats()["candidates"]
    tp = _device_time(lambda: dk.run(bid, [pid], dict(kn, plain_mode=1), 1, natoms, out=out, xyz_out=xyz,
                                     stream=stream), torch, stream, 20)
    dk.release_batch(bid)
    return {"workload": "1 ligand (24 atoms, 4 rotatable bonds) x 1 pocket 48^3, 8 poses, 10 deg, 1 rep",
            "ligands_per_s": 1 / t, "pose_evals_per_s": cand / t, "atoms_per_s": natoms / t, "ms": 1e3 * t,
            "plain_ligands_per_s": 1 / tp, "batched_vs_plain": tp / t,
            "note": "one ligand: the batched form (one graph launch) against the plain form (its own launches)"}


def leg_diff(dk, torch, stream, plain_n=64):
    """4,096 ligands (20-60 atoms, 3-10 rotatable bonds) on a 64^3 trilinear field: sampled stage (64 poses,
    10 degrees, 4 repetitions), then 20 refinement steps from each ligand's best pose."""
    import synth.configs as C
    pks, b, kn = C.differentiation()
    pid = dk.init_pocket(pks[0])
    bid = dk.upload_ligands(b)
    n, natoms = b.n, int(b.atom_off[-1])
    out = torch.empty(n * 4, dtype=torch.int32, device="cuda")
    xyz = torch.empty(natoms * 3, dtype=torch.float32, device="cuda")
    t_s = _device_time(lambda: dk.run(bid, [pid], kn, n, natoms, out=out, xyz_out=xyz, stream=stream), torch, stream)
    cand = dk.stats()["candidates"]
    rout = torch.empty(n * 4, dtype=torch.int32, device="cuda")
    rxyz = torch.empty_like(xyz)
    t_r = _device_time(lambda: dk.refine(bid, [pid], kn, xyz, out=rout, xyz_out=rxyz, stream=stream), torch, stream)
    o0 = dk.score_trilinear(bid, pid, xyz)
    gain = float((rout.view(torch.float32).reshape(-1, 4)[:, 0] / o0).mean().item())
    dk.release_batch(bid)
    sub = b.subset(np.arange(plain_n))
    sb = dk.upload_ligands(sub, ids=np.arange(plain_n) + b.id_base)
    sat = int(sub.atom_off[-1])
    so = torch.empty(plain_n * 4, dtype=torch.int32, device="cuda")
    sx = torch.empty(sat * 3, dtype=torch.float32, device="cuda")
    tp = _device_time(lambda: dk.run(sb, [pid], dict(kn, plain_mode=1), plain_n, sat, out=so, xyz_out=sx,
                                     stream=stream), torch, stream, 1)
    dk.release_batch(sb)
    return {"workload": "4096 ligands (20-60 atoms, 3-10 rotatable bonds) x 1 pocket 64^3 trilinear, 64 poses, "
                        "10 deg, 4 reps, then 20 refinement steps",
            "ligands_per_s": n / (t_s + t_r), "sampled_ligands_per_s": n / t_s, "refined_ligands_per_s": n / t_r,
            "pose_evals_per_s": cand / t_s, "atoms_per_s": natoms / (t_s + t_r), "ms_sampled": 1e3 * t_s,
            "ms_refined": 1e3 * t_r, "refined_over_sampled_score": gain,
            "plain_ligands_per_s": plain_n / tp, "batched_vs_plain": (n / t_s) / (plain_n / tp),
            "note": f"plain form of the sampled stage on the first {plain_n} ligands"}


def leg_multi(dk, torch, stream, plain_pairs=64):
    """16 pockets (48^3-128^3) x 50,000 lognormal ligands in one grouped launch; 32 poses, 15 deg, 2 reps."""
    import synth.configs as C
    pks, b, kn = C.multi_pocket()
    pids = [dk.init_pocket(p) for p in pks]
    bid = dk.upload_ligands(b)
    n, natoms = b.n, int(b.atom_off[-1])
    npk = len(pks)
    out = torch.empty(npk * n * 4, dtype=torch.int32, device="cuda")
    t = _device_time(lambda: dk.run(bid, pids, kn, n, natoms, out=out, xyz_out=None, stream=stream), torch, stream, 2)
    cand = dk.stats()["candidates"]
    dk.release_batch(bid)
    # plain form: one launch per pair, on the first plain_pairs / 16 ligands of every pocket
    k = plain_pairs // npk
    sub = b.subset(np.arange(k))
    sb = dk.upload_ligands(sub, ids=np.arange(k) + b.id_base)
    so = torch.empty(npk * k * 4, dtype=torch.int32, device="cuda")
    tp = _device_time(lambda: dk.run(sb, pids, dict(kn, plain_mode=1), k, int(sub.atom_off[-1]), out=so,
                                     xyz_out=None, stream=stream), torch, stream, 1)
    dk.release_batch(sb)
    return {"workload": "16 pockets (48^3-128^3) x 50000 ligands (lognormal, median 32 atoms), 32 poses, 15 deg, "
                        "2 reps, one grouped launch",
            "ligands_per_s": n / t, "pairs_per_s": npk * n / t, "pose_evals_per_s": cand / t,
            "atoms_per_s": npk * natoms / t, "s": t, "plain_pairs_per_s": npk * k / tp,
            "batched_vs_plain": (npk * n / t) / (npk * k / tp),
            "note": f"ligands_per_s counts a ligand once for all 16 pockets; plain form on {npk * k} pairs"}


def leg_sweep(dk, torch, stream):
    """The 100,000 lognormal ligands x the 64^3 pocket at one point of the knob grid (10 deg, 32 poses, 4 reps)."""
    import synth.configs as C
    pks, b, combos = C.knob_sweep()
    kn = [c for c in combos if (c["hp_step"], c["n_poses"], c["repetitions"]) == (10.0, 32, 4)][0]
    pid = dk.init_pocket(pks[0])
    bid = dk.upload_ligands(b)
    n, natoms = b.n, int(b.atom_off[-1])
    out = torch.empty(n * 4, dtype=torch.int32, device="cuda")
    t = _device_time(lambda: dk.run(bid, [pid], kn, n, natoms, out=out, xyz_out=None, stream=stream), torch, stream, 2)
    cand = dk.stats()["candidates"]
    dk.release_batch(bid)
    return {"workload": "100000 ligands (lognormal, median 32 atoms, Poisson(6) rotatable bonds) x 1 pocket 64^3, "
                        "10 deg, 32 poses, 4 reps (one point of the 45-point knob grid)",
            "ligands_per_s": n / t, "pose_evals_per_s": cand / t, "atoms_per_s": natoms / t, "s": t}


def cpu_configs(cores):
    """The FP64 oracle on bounded samples of the other workloads (whole ligands, all poses), on the host cores."""
    import oracle
    import synth.configs as C
    out = {}

    def timed(name, pks, b, kn, idx, pairs=1):
        opks = [oracle.OraclePocket(p) for p in pks]
        sub = b.subset(idx)
        t0 = time.perf_counter()
        for opk in opks:
            oracle.dock(opk, sub, kn, nthreads=cores, ids=idx + b.id_base)
        dt = time.perf_counter() - t0
        out[name] = {"ligands_per_s": len(idx) / dt, "pairs_per_s": len(idx) * len(opks) / dt,
                     "sample": f"{len(idx)} ligands x {len(opks)} pocket(s), {dt:.1f} s"}

    pks, b, kn = C.single()
    timed("single", pks, b, kn, np.arange(1))
    pks, b, kn = C.differentiation()
    timed("differentiation", pks, b, kn, np.arange(2 * cores))
    pks, b, kn = C.multi_pocket()
    timed("multi_pocket", pks[::5], b, kn, np.arange(cores))
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pk, batch, kn = workload(0)
    import oracle
    opk = oracle.OraclePocket(pk)
    cores = os.cpu_count() or 1
    per_step = 2 * cores
    for w in range(args.warmup):
        idx = np.arange(w * per_step % batch.n, w * per_step % batch.n + per_step) % batch.n
        oracle.dock(opk, batch.subset(idx), kn, nthreads=cores, ids=idx)
    times, n = [], 0
    for s in range(args.steps):
        idx = np.arange((args.warmup + s) * per_step, (args.warmup + s + 1) * per_step) % batch.n
        sub = batch.subset(idx)
        t0 = time.perf_counter()
        oracle.dock(opk, sub, kn, nthreads=cores, ids=idx)
        times.append(time.perf_counter() - t0)
        n += len(idx)
    tot = sum(times)
    value = n / tot
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "step_sample": f"{per_step} ligands per step on the host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} workload ligands per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_strong(args):
    """Strong scaling: the one 1,024-ligand workload split over the ranks by the LPT work model (shard.py);
    each rank docks its shard, the results are gathered to rank 0 once after the timed steps and checked to
    cover every ligand once. Prints the timed throughput of the whole workload."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1901_06363_gb300 import Docker, shard
    pk, batch, kn = workload(0)
    costs = shard.ligand_costs(batch, 36, kn["n_poses"], kn["repetitions"])
    idx = shard.lpt_shards(costs, world)[rank]
    sub = batch.subset(idx)
    dk = Docker(local)
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(sub, ids=idx + batch.id_base)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n, natoms = sub.n, int(sub.atom_off[-1])
    out = torch.zeros(max(n, 1) * 4, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        dk.run(bid, [pid], kn, n, natoms, out=out, xyz_out=None, stream=stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            dk.run(bid, [pid], kn, n, natoms, out=out, xyz_out=None, stream=stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    if dist:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    from paper_1901_06363_gb300 import RESULT_DTYPE
    local_res = out[:n * 4].cpu().numpy().view(RESULT_DTYPE)
    res = shard.gather_results(idx, local_res, batch.n) if dist else local_res
    if rank == 0:
        line = {"metric": METRIC, "value": batch.n * args.steps / total_s, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "parallelism": f"ligand shards over {world} rank(s), LPT on the "
                           "work model", "shard_sizes": [int(len(p)) for p in shard.lpt_shards(costs, world)],
                           "l2": "flushed between timed steps (256 MiB write)"},
                "all_ligands_docked": bool(len(res) == batch.n and np.all(res["status"] == 0)),
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    dk.close()
    if dist:
        dist.destroy_process_group()


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1901_06363_gb300 import Docker

    pk, batch, kn = workload(rank)
    n, natoms = batch.n, int(batch.atom_off[-1])
    dk = Docker(local)
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(batch)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    out = torch.zeros(n * 4, dtype=torch.int32, device=dev)
    xyz = torch.zeros(natoms * 3, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # larger than the 129 MB L2

    def step():
        dk.run(bid, [pid], kn, n, natoms, out=out, xyz_out=xyz, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sweep_ms = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.zero_()  # L2 flushed between timed steps (outside the events)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            sweep_ms.append(dk.stats()["sweep_ms"])
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    if dist:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
        dist.barrier()
    st = dk.stats()
    cand_per_step = st["candidates"]  # evaluated candidates (repetitions left out at a fixed point excluded)
    value = world * n * args.steps / total_s

    if args.no_baselines:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": world * n * args.steps / total_s, "unit": UNIT,
                              "sweep_ms": statistics.mean(sweep_ms), "note": "timed steps only"}), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    # end to end through the C ABI with host buffers: the database call docks e2e_steps batches of the
    # workload (distinct ligand ids, so distinct poses) from host memory, one chunk per step: host
    # preparation and upload (H2D) of each chunk, its sweep, and its results and coordinates back (D2H)
    e2e_steps = max(2, min(args.steps, 10))  # chunks of one database call: the pipeline fills once
    db = repeat_batch(batch, e2e_steps)
    dk.run_database(repeat_batch(batch, 2), [pid], kn, chunk=n)  # warm: both pipeline stages' buffers
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    res_host, xyz_host = dk.run_database(db, [pid], kn, chunk=n)
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * n * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": input_bytes(batch),
           "d2h_bytes_per_step": int((res_host.nbytes + xyz_host.nbytes) // e2e_steps),
           "api": "dock_run_database, one chunk of the workload per step"}

    # local refinement of the docked poses (20 ascent steps on the trilinear score), device timed
    rk = dict(kn, refine_steps=20)
    rout = torch.empty(n * 4, dtype=torch.int32, device=dev)
    rxyz = torch.empty_like(xyz)
    dk.refine(bid, [pid], rk, xyz, out=rout, xyz_out=rxyz, stream=stream)  # warm
    torch.cuda.synchronize()
    re0, re1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    re0.record(stream)
    for _ in range(5):
        dk.refine(bid, [pid], rk, xyz, out=rout, xyz_out=rxyz, stream=stream)
    re1.record(stream)
    torch.cuda.synchronize()
    refine_ms = re0.elapsed_time(re1) / 5
    rscore = rout.view(torch.float32).reshape(-1, 4)[:, 0]
    sscore = dk.score_trilinear(bid, pid, xyz)
    refine = {"ligands_per_s": world * n / (refine_ms / 1e3), "ms_per_batch": refine_ms, "steps": 20,
              "improved_fraction": float((rscore > sscore).float().mean().item()),
              "note": "refinement of the best docked pose per ligand on the trilinear form of the score"}

    # exact point-set score (Eq. 1's inner minimum without the grid) on a subset of the ligands
    sub_n = 64
    sub = batch.subset(np.arange(sub_n))
    sbid = dk.upload_ligands(sub, ids=np.arange(sub_n) + batch.id_base)
    sat = int(sub.atom_off[-1])
    kx = dict(kn, score_mode=2)
    xo_ = torch.empty(sub_n * 4, dtype=torch.int32, device=dev)
    xx_ = torch.empty(sat * 3, dtype=torch.float32, device=dev)
    dk.run(sbid, [pid], kx, sub_n, sat, out=xo_, xyz_out=xx_, stream=stream)  # warm
    torch.cuda.synchronize()
    xe0, xe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    xe0.record(stream)
    dk.run(sbid, [pid], kx, sub_n, sat, out=xo_, xyz_out=xx_, stream=stream)
    xe1.record(stream)
    torch.cuda.synchronize()
    exact_ms = xe0.elapsed_time(xe1)
    o_exact = xo_.view(torch.float32).reshape(-1, 4)[:, 0].cpu().numpy()
    o_grid = out.view(torch.float32).reshape(-1, 4)[:sub_n, 0].cpu().numpy()
    exact = {"ligands_per_s": sub_n / (exact_ms / 1e3), "ms": exact_ms, "ligands": sub_n,
             "npts": int(len(pk.pts)), "best_o_nearest_over_exact": float(np.mean(o_grid / o_exact)),
             "note": "score_mode 2 on the first 64 workload ligands (same knobs)"}
    dk.release_batch(sbid)

    # plain per-ligand form (one launch per pair, no graph), one step
    torch.cuda.synchronize()
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dk.run(bid, [pid], dict(kn, plain_mode=1), n, natoms, out=out, xyz_out=xyz, stream=stream)  # warm
    torch.cuda.synchronize()
    pe0.record(stream)
    dk.run(bid, [pid], dict(kn, plain_mode=1), n, natoms, out=out, xyz_out=xyz, stream=stream)
    pe1.record(stream)
    torch.cuda.synchronize()
    plain_s = pe0.elapsed_time(pe1) / 1e3

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks, src = _peaks()
    f_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sweep_avg = statistics.mean(sweep_ms)
    sweep_s = sweep_avg / 1e3
    clocks = clk.summary()
    rates = dk.measure_peaks(pid, stream=stream)  # after the timed region
    # exact feasible-candidate counts of the timed launch (from a traced run of the same batch and knobs)
    fw = feasible_work(dk, bid, pid, kn, batch)
    traffic = _traffic()
    bound, res = roofline_8d(st, fw, sweep_s, rates, traffic, float(peaks.get("hbm_gbs", 6800.0)))
    rb = res[bound]
    roofline = {"bound": bound, "achieved": rb["achieved"], "peak": rb["peak"],
                "unit": {"texture": "fetches/s", "fp32": "lane-ops/s", "hbm": "B/s"}[bound], "frac": rb["frac"],
                "traffic": traffic, "traffic_unit": "DRAM bytes per launch (ncu)", "kernel": "sweep_kernel",
                "sweep_ms": sweep_avg, "feasible_fraction": fw["feasible"] / max(fw["candidates"], 1),
                "peak_source": "texture: point-sampled fetches within 16^3-voxel cubes (the locality of one "
                               "ligand's poses), the higher of the two fetch rates dock_measure_peaks measured in "
                               "this run; fp32: its FMA rate; hbm: " + src + " copy bandwidth",
                "resources": res,
                "work": {"candidates": fw["candidates"], "feasible_candidates": fw["feasible"],
                         "feasible_lookups": fw["feasible_lookups"], "placements": fw["lookups"],
                         "lookups_done": int(st["atom_updates"]), "bump_pairs": int(st["bump_pairs"]),
                         "counts_match_run": fw["candidates"] == st["candidates"] and
                         fw["lookups"] == st["atom_updates"] + st["lookups_skipped"]}}
    # issue-slot view of the same kernel (secondary): 16 lane instructions per lookup made and 8 per circle bound
    peak_inst = sms * 4 * 32 * f_mhz * 1e6
    inst = 16.0 * st["atom_updates"] + 8.0 * st["pair_bounds"]
    issue = {"achieved": inst / sweep_s, "peak": peak_inst, "unit": "lane-instructions/s",
             "frac": inst / sweep_s / peak_inst,
             "note": f"{sms} SMs x 4 schedulers x 32 lanes x sm_max_mhz {f_mhz:.0f}; 16 per lookup made (6 FMA, 3 "
                     "floor, 3 bound tests, 2 index, 1 load, 1 add), 8 per circle bound (3 sub, 3 FMA, compare, vote)"}
    # the other workloads on this GPU (batched against plain), then the oracle on host cores
    configs = {"single": leg_single(dk, torch, stream), "knob_sweep_point": leg_sweep(dk, torch, stream),
               "differentiation": leg_diff(dk, torch, stream), "multi_pocket": leg_multi(dk, torch, stream)}
    cpu = None
    if world == 1:
        cpu = cpu_baseline(pk, batch, kn)
        t0 = time.perf_counter()
        import oracle
        one = batch.subset(np.arange(8))
        oracle.dock(oracle.OraclePocket(pk), one, kn, nthreads=1, ids=np.arange(8) + batch.id_base)
        dt = time.perf_counter() - t0
        cpu["one_core"] = {"value": 8 / dt, "unit": UNIT, "cores": 1, "sample": f"first 8 workload ligands ({dt:.1f} s)"}
        cpu["configs"] = cpu_configs(cpu["cores"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "ligands_per_gpu": n, "poses": kn["n_poses"], "step_deg": kn["hp_step"],
                   "repetitions": kn["repetitions"], "grid": list(pk.dims), "score": "nearest",
                   "l2": "flushed between timed steps (256 MiB write)"},
        "pose_evals_per_s": world * cand_per_step * args.steps / total_s,
        "atoms_per_s": world * natoms * args.steps / total_s,
        "plain_ligands_per_s": world * n / plain_s,
        "batched_vs_plain": (value / world) / (n / plain_s),
        "roofline": roofline,
        "roofline_issue": issue,
        "measured_rates": rates,
        "configs": configs,
        "refine": refine,
        "exact_score": exact,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(st["kernel_launches"]) * args.steps,
        "work_per_step": {k: int(st[k]) for k in ("candidates", "atom_updates", "pair_bounds", "bump_pairs")},
        "pose_reps_skipped_per_step": int(st["pose_reps_skipped"]),
        "lookups_skipped_per_step": int(st["lookups_skipped"]),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scaling", choices=["weak", "strong"], default="weak",
                    help="weak: every rank docks its own 1,024 ligands; strong: the ranks split one 1,024-ligand "
                         "workload (LPT) and gather its results")
    ap.add_argument("--no-baselines", action="store_true",
                    help="skip the CPU oracle, end-to-end and plain-form legs (for profiling the timed steps)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.scaling == "strong":
        run_strong(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
