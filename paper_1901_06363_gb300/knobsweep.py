"""Design-space exploration of the knobs on the GPU (Sec. 4.3-4.4): time-to-solution vs overlap
degradation (Eq. 5) over the (step, initial poses, repetitions) grid, and the Eq. 4 time model fitted
per configuration and validated leave-one-pocket-out.

    python -m paper_1901_06363_gb300.knobsweep [--ligands 100000] [--fit-ligands 4000] [--out FILE]
                                               [--checkpoint DIR]

Inputs are the seeded synthetic workloads: lognormal ligands (median 32 atoms, Poisson(6) rotatable
bonds) on the 64^3 ellipsoid pocket for the sweep, and that pocket plus four pockets of 48^3-128^3 x four
ligand groups (quartiles of atoms x rotatable bonds) for the model. Every run is a batched dock_run
timed with CUDA events on its stream after one warm-up run of the same plan (the median of three
runs); the plain per-pair form is timed on a subset. Prints one JSON document. With --checkpoint,
every finished shard (one configuration on the sweep set, its plain-form timing, one fit row) is kept
in DIR and skipped when the run is restarted.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


class Checkpoint:
    """Finished result shards under a directory (one .npz per key); a restarted run loads them
    instead of recomputing. Without a directory every shard is computed."""

    def __init__(self, path=None):
        self.path = path
        if path:
            os.makedirs(path, exist_ok=True)

    def get(self, key, compute):
        if not self.path:
            return compute()
        f = os.path.join(self.path, key + ".npz")
        if os.path.exists(f):
            with np.load(f) as z:
                return {k: z[k] for k in z.files}
        res = compute()
        tmp = os.path.join(self.path, key + ".part.npz")
        np.savez(tmp, **res)
        os.replace(tmp, f)  # a shard appears whole or not at all
        return res


def _timed_run(dk, bid, pids, kn, n, natoms, out, xyz, stream, torch, repeats=3):
    """Median of `repeats` runs timed by CUDA events, after one warm-up run (plan build and capture)."""
    dk.run(bid, pids, kn, n, natoms, out=out, xyz_out=xyz, stream=stream)
    times = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        dk.run(bid, pids, kn, n, natoms, out=out, xyz_out=xyz, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return float(np.median(times))


def run(ligands=100_000, fit_ligands=4_000, plain_ligands=128, seed=3, combos=None, log=None, checkpoint=None):
    import torch

    import synth
    import synth.configs as C
    from paper_1901_06363_gb300 import Docker, tuning

    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    dk = Docker(torch.cuda.current_device())
    say = log or (lambda *a: None)
    ck = Checkpoint(checkpoint)
    tag = lambda k: f"{k[0]:g}_{k[1]}_{k[2]}"  # noqa: E731

    # ---- sweep: every combination on the full ligand set, one pocket
    pk = synth.pocket(1 + 7, 64, 0.5, C.ELLIPSOID)
    pid = dk.init_pocket(pk)
    b = C.sweep_batch(ligands, seed)
    bid = dk.upload_ligands(b)
    n, natoms = b.n, int(b.atom_off[-1])
    out = torch.empty(n * 4, dtype=torch.int32, device=dev)
    xyz = torch.empty(natoms * 3, dtype=torch.float32, device=dev)
    combos = combos or [C.knobs(hp_step=s, lp_step=s, n_poses=p, repetitions=r, seed=seed)
                        for s in C.SWEEP_STEPS for p in C.SWEEP_POSES for r in C.SWEEP_REPS]
    key = lambda k: (k["hp_step"], k["n_poses"], k["repetitions"])  # noqa: E731
    sweep = {}
    for kn in combos:
        def one(kn=kn):
            t = _timed_run(dk, bid, [pid], kn, n, natoms, out, xyz, stream, torch)
            sc = out.view(torch.float32).reshape(-1, 4)[:, 0].cpu().numpy().copy()
            return dict(seconds=np.float64(t), scores=sc)
        r = ck.get(f"sweep_{n}_{tag(key(kn))}", one)
        t = float(r["seconds"])
        sweep[key(kn)] = dict(seconds=t, ligands_per_s=n / t, scores=r["scores"])
        say(f"sweep {key(kn)}: {t:.3f} s, {n / t:.0f} ligands/s")
    base = max(sweep, key=lambda c: (-c[0], c[1], c[2]))  # finest step, most poses, most repetitions
    # plain per-pair form on a subset, per configuration
    sub = b.subset(np.arange(plain_ligands))
    sbid = dk.upload_ligands(sub, ids=np.arange(plain_ligands) + b.id_base)
    sat = int(sub.atom_off[-1])
    so = torch.empty(plain_ligands * 4, dtype=torch.int32, device=dev)
    sx = torch.empty(sat * 3, dtype=torch.float32, device=dev)
    for kn in combos:
        r = ck.get(f"plain_{plain_ligands}_{tag(key(kn))}", lambda kn=kn: dict(seconds=np.float64(_timed_run(
            dk, sbid, [pid], dict(kn, plain_mode=1), plain_ligands, sat, so, sx, stream, torch))))
        sweep[key(kn)]["plain_ligands_per_s"] = plain_ligands / float(r["seconds"])
    dk.release_batch(sbid)
    dk.release_batch(bid)

    # ---- Eq. 4: per configuration, times over pockets x ligand groups
    pks = C.multi_pocket_pockets()
    fit_pockets = [pk] + [pks[i] for i in (0, 4, 8, 12)]  # the sweep's pocket, then 48^3, 64^3, 96^3, 128^3
    fpids = [dk.init_pocket(p) for p in fit_pockets]
    fb = C.sweep_batch(4 * fit_ligands, seed + 100, id0=10_000_000)
    l, t = fb.sizes()
    order = np.argsort(l * (t + 1), kind="stable")
    groups = np.array_split(order, 4)
    rows = []
    for gi, g in enumerate(groups):
        g = np.sort(g)
        gb = fb.subset(g)
        gbid = dk.upload_ligands(gb, ids=g + fb.id_base)
        gn, gat = gb.n, int(gb.atom_off[-1])
        go = torch.empty(gn * 4, dtype=torch.int32, device=dev)
        gx = torch.empty(gat * 3, dtype=torch.float32, device=dev)
        gl, gt = gb.sizes()
        for p_i, (fp, fpid) in enumerate(zip(fit_pockets, fpids)):
            for kn in combos:
                secs = float(ck.get(f"fit_{fit_ligands}_{gi}_{p_i}_{tag(key(kn))}", lambda kn=kn, fpid=fpid: dict(
                    seconds=np.float64(_timed_run(dk, gbid, [fpid], kn, gn, gat, go, gx, stream, torch))))["seconds"])
                rows.append(dict(config=key(kn), pocket=p_i, group=gi, npts=len(fp.pts), mean_atoms=float(gl.mean()),
                                 mean_rot=float(gt.mean()), nu=gn, seconds=secs))
        dk.release_batch(gbid)
        say(f"fit group {gi} done")
    models = tuning.fit_models(rows)
    # leave one pocket out
    loo = {}
    for c in models:
        errs = []
        for p_i in range(len(fit_pockets)):
            train = [r for r in rows if r["config"] == c and r["pocket"] != p_i]
            test = [r for r in rows if r["config"] == c and r["pocket"] == p_i]
            m = tuning.fit_models(train)[c]
            for r in test:
                pred = m.predict(tuning.features(r["npts"], r["mean_atoms"], r["mean_rot"]), r["nu"])
                errs.append(abs(pred - r["seconds"]) / r["seconds"])
        loo[c] = errs

    # ---- report
    degr = {c: tuning.degradation(v["scores"], sweep[base]["scores"]) for c, v in sweep.items()}
    lsw, tsw = b.sizes()
    x_main = tuning.features(len(pk.pts), lsw.mean(), tsw.mean())
    table = []
    for c in sorted(sweep):
        v = sweep[c]
        table.append(dict(step=c[0], poses=c[1], repetitions=c[2], seconds=v["seconds"],
                          ligands_per_s=v["ligands_per_s"], plain_ligands_per_s=v["plain_ligands_per_s"],
                          degradation_pct=degr[c], model_adj_r2=models[c].adj_r2,
                          model_predicted_s=models[c].predict(x_main, n),
                          loo_mean_err=float(np.mean(loo[c])), loo_max_err=float(np.max(loo[c]))))
    front = []
    for row in sorted(table, key=lambda r: r["seconds"]):
        if not front or row["degradation_pct"] < front[-1]["degradation_pct"]:
            front.append(row)
    tmin = min(r["seconds"] for r in table)
    budgets = [tmin * f for f in (0.5, 1, 2, 4, 8, 16, 64)]
    picks = []
    for B in budgets:
        ch = tuning.select(models, degr, x_main, n, B)
        picks.append(dict(budget_s=B, config=list(ch.config), predicted_s=ch.predicted_s,
                          degradation_pct=ch.degradation, completion=ch.completion))
    dk.close()
    return dict(ligands=n, mean_atoms=float(lsw.mean()), mean_rot=float(tsw.mean()), npts=len(pk.pts),
                baseline=list(base), table=table, pareto=[[r["step"], r["poses"], r["repetitions"]] for r in front],
                selection=picks, fit=dict(pockets=[len(p.pts) for p in fit_pockets], ligands_per_group=fit_ligands,
                                          rows=len(rows)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ligands", type=int, default=100_000)
    ap.add_argument("--fit-ligands", type=int, default=4_000)
    ap.add_argument("--plain-ligands", type=int, default=128)
    ap.add_argument("--out", default=None)
    ap.add_argument("--checkpoint", default=None, help="directory of finished shards (resumes a stopped run)")
    args = ap.parse_args()
    t0 = time.time()
    res = run(args.ligands, args.fit_ligands, args.plain_ligands, log=lambda *a: print(*a, file=sys.stderr),
              checkpoint=args.checkpoint)
    res["wall_s"] = time.time() - t0
    txt = json.dumps(res)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt)
    print(txt)


if __name__ == "__main__":
    main()
