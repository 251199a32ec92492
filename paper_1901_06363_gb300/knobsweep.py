"""Design-space exploration of the knobs on the GPU (Sec. 4.3-4.4 and Sec. 5.2): time-to-solution vs
overlap degradation (Eq. 5), Pareto fronts, and the Eq. 4 time model fitted per configuration and
validated leave-one-pocket-out.

    python -m paper_1901_06363_gb300.knobsweep [--space grid|flat|full] [--ligands N] [--fit-ligands M]
                                               [--poses P] [--out FILE] [--summary FILE] [--checkpoint DIR]

Spaces (full factorial):
  grid  angle step {5,10,20,30,45} x initial poses {8,32,128} x repetitions {1,4,16} (45 points), one
        step for every fragment; degradation against (5, 128, 16)
  flat  the paper's flat space (Sec. 5.2): high-precision step {1,2,3,5,10,15,45,60} x repetitions
        {1,2,3} (24 points), one step for every fragment, no tile peeling
  full  the paper's full space (Sec. 5.2): high-precision step {1,2,3,5} x low-precision step {45,90} x
        threshold {0,0.3,0.6,0.8} x repetitions {1,2,3} x tile peeling {on,off} (192 points)
  flat and full use P initial poses (default 8) and share the paper's baseline: high-precision step 1,
  threshold 0, repetitions 3, no peeling; Eq. 5 compares every point with it.

Inputs are the seeded synthetic workloads: lognormal ligands (median 32 atoms, Poisson(6) rotatable
bonds) on the 64^3 ellipsoid pocket for the exploration, and that pocket plus four pockets of
48^3-128^3 x four ligand groups (quartiles of atoms x rotatable bonds) for the model. Every point is a
batched dock_run timed with CUDA events on its stream after one warm-up run of the same plan (the median
of three runs; the model's rows take one run each); the plain per-pair form is timed on a subset (grid
space). Prints one JSON document; --summary writes a small one (the table, the fronts, the fit summary)
for the record. With --checkpoint, every finished shard is kept in DIR and skipped when the run is
restarted.
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

FLAT_HP = (1.0, 2.0, 3.0, 5.0, 10.0, 15.0, 45.0, 60.0)
FLAT_REPS = (1, 2, 3)
FULL_HP = (1.0, 2.0, 3.0, 5.0)
FULL_LP = (45.0, 90.0)
FULL_THRESHOLD = (0.0, 0.3, 0.6, 0.8)
FULL_REPS = (1, 2, 3)
FULL_PEEL = (0, 1)


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


def space(name, seed=3, poses=8):
    """(knob dicts, key names, baseline key) of a design space; a point's key is the tuple of its
    varying knobs, in the order of the names."""
    import synth.configs as C
    if name == "grid":
        pts = [C.knobs(hp_step=s, lp_step=s, n_poses=p, repetitions=r, seed=seed)
               for s in C.SWEEP_STEPS for p in C.SWEEP_POSES for r in C.SWEEP_REPS]
        return pts, ("hp_step", "n_poses", "repetitions"), (5.0, 128, 16)
    if name == "flat":
        pts = [C.knobs(hp_step=s, lp_step=s, n_poses=poses, repetitions=r, seed=seed)
               for s in FLAT_HP for r in FLAT_REPS]
        return pts, ("hp_step", "repetitions"), (1.0, 3)
    if name == "full":
        pts = [C.knobs(hp_step=s, lp_step=lp, threshold=t, n_poses=poses, repetitions=r, enable_refinement=e,
                       seed=seed)
               for s in FULL_HP for lp in FULL_LP for t in FULL_THRESHOLD for r in FULL_REPS for e in FULL_PEEL]
        return pts, ("hp_step", "lp_step", "threshold", "repetitions", "enable_refinement"), (1.0, 45.0, 0.0, 3, 0)
    raise ValueError(name)


def pareto(rows):
    """Non-dominated rows in (seconds, degradation): sorted by time, each strictly less degraded."""
    front = []
    for row in sorted(rows, key=lambda r: (r["seconds"], r["degradation_pct"])):
        if not front or row["degradation_pct"] < front[-1]["degradation_pct"]:
            front.append(row)
    return front


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


def run(ligands=100_000, fit_ligands=4_000, plain_ligands=128, seed=3, space_name="grid", poses=8, log=None,
        checkpoint=None, fit_repeats=3):
    import torch

    import synth
    import synth.configs as C
    from paper_1901_06363_gb300 import Docker, tuning

    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    dk = Docker(torch.cuda.current_device())
    say = log or (lambda *a: None)
    ck = Checkpoint(checkpoint)
    combos, names, base = space(space_name, seed, poses)
    key = lambda k: tuple(k[nm] for nm in names)  # noqa: E731
    tag = lambda k: space_name + "_" + "_".join(f"{v:g}" for v in k)  # noqa: E731

    # ---- the exploration: every point on the full ligand set, one pocket
    pk = synth.pocket(1 + 7, 64, 0.5, C.ELLIPSOID)
    pid = dk.init_pocket(pk)
    b = C.sweep_batch(ligands, seed)
    bid = dk.upload_ligands(b)
    n, natoms = b.n, int(b.atom_off[-1])
    out = torch.empty(n * 4, dtype=torch.int32, device=dev)
    xyz = torch.empty(natoms * 3, dtype=torch.float32, device=dev)
    sweep = {}
    for kn in combos:
        def one(kn=kn):
            t = _timed_run(dk, bid, [pid], kn, n, natoms, out, xyz, stream, torch)
            sc = out.view(torch.float32).reshape(-1, 4)[:, 0].cpu().numpy().copy()
            st = dk.stats()
            return dict(seconds=np.float64(t), scores=sc, candidates=np.float64(st["candidates"]),
                        atom_updates=np.float64(st["atom_updates"] + st["lookups_skipped"]))
        r = ck.get(f"sweep_{n}_{tag(key(kn))}", one)
        t = float(r["seconds"])
        sweep[key(kn)] = dict(seconds=t, ligands_per_s=n / t, atoms_per_s=natoms / t, scores=r["scores"],
                              pose_evals_per_s=float(r["candidates"]) / t)
        say(f"{space_name} {key(kn)}: {t:.4f} s, {n / t:.0f} ligands/s")
    assert base in sweep
    if space_name == "grid":
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
    rows = []
    if fit_ligands > 0:
        pks = C.multi_pocket_pockets()
        fit_pockets = [pk] + [pks[i] for i in (0, 4, 8, 12)]  # the sweep's pocket, then 48^3, 64^3, 96^3, 128^3
        fpids = [dk.init_pocket(p) for p in fit_pockets]
        fb = C.sweep_batch(4 * fit_ligands, seed + 100, id0=10_000_000)
        l, t = fb.sizes()
        order = np.argsort(l * (t + 1), kind="stable")
        groups = np.array_split(order, 4)
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
                        seconds=np.float64(_timed_run(dk, gbid, [fpid], kn, gn, gat, go, gx, stream, torch,
                                                      repeats=fit_repeats))))["seconds"])
                    rows.append(dict(config=key(kn), pocket=p_i, group=gi, npts=len(fp.pts),
                                     mean_atoms=float(gl.mean()), mean_rot=float(gt.mean()), nu=gn, seconds=secs))
            dk.release_batch(gbid)
            say(f"fit group {gi} done")
    models = tuning.fit_models(rows) if rows else {}
    loo = {}
    for c in models:
        errs = []
        for p_i in sorted({r["pocket"] for r in rows}):
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
        row = dict(zip(names, c))
        row.update(seconds=v["seconds"], ligands_per_s=v["ligands_per_s"], atoms_per_s=v["atoms_per_s"],
                   pose_evals_per_s=v["pose_evals_per_s"], speedup=sweep[base]["seconds"] / v["seconds"],
                   degradation_pct=degr[c])
        if "plain_ligands_per_s" in v:
            row["plain_ligands_per_s"] = v["plain_ligands_per_s"]
        if c in models:
            row.update(model_adj_r2=models[c].adj_r2, model_predicted_s=models[c].predict(x_main, n),
                       loo_mean_err=float(np.mean(loo[c])), loo_max_err=float(np.max(loo[c])))
        table.append(row)
    front = pareto(table)
    picks = []
    if models:
        tmin = min(r["seconds"] for r in table)
        for B in [tmin * f for f in (0.5, 1, 2, 4, 8, 16, 64)]:
            ch = tuning.select(models, degr, x_main, n, B)
            picks.append(dict(budget_s=B, config=list(ch.config), predicted_s=ch.predicted_s,
                              degradation_pct=ch.degradation, completion=ch.completion))
    dk.close()
    res = dict(space=space_name, knobs=list(names), ligands=n, poses=poses if space_name != "grid" else None,
               mean_atoms=float(lsw.mean()), mean_rot=float(tsw.mean()), npts=len(pk.pts), baseline=list(base),
               baseline_seconds=sweep[base]["seconds"], table=table,
               pareto=[[r[nm] for nm in names] for r in front], selection=picks)
    if models:
        r2 = [m.adj_r2 for m in models.values()]
        le = [e for c in loo for e in loo[c]]
        res["fit"] = dict(pockets=[len(p.pts) for p in fit_pockets], ligands_per_group=fit_ligands, rows=len(rows),
                          adj_r2_min=float(np.min(r2)), adj_r2_median=float(np.median(r2)),
                          loo_mean_err=float(np.mean(le)), loo_max_err=float(np.max(le)))
    return res


def summary(res):
    """The record of an exploration: its table (times, rates, degradation, model columns), the Pareto
    front and, for the paper's spaces, the tile-peeling-only point of Sec. 5.2."""
    keep = dict((k, res[k]) for k in ("space", "knobs", "ligands", "poses", "mean_atoms", "mean_rot", "npts",
                                      "baseline", "baseline_seconds", "pareto", "selection") if k in res)
    keep["fit"] = res.get("fit")
    cols = list(res["table"][0].keys()) if res["table"] else []
    sig = lambda v: float(f"{v:.5g}") if isinstance(v, float) else v  # noqa: E731
    keep["columns"] = cols
    keep["table"] = [[sig(r[c]) for c in cols] for r in res["table"]]
    if res["space"] == "full":
        # the baseline with tile peeling switched on and nothing else changed
        names = res["knobs"]
        b = dict(zip(names, res["baseline"]))
        pt = [r for r in res["table"] if all(r[nm] == (1 if nm == "enable_refinement" else b[nm]) for nm in names)]
        pt = [dict(r, speedup=float(f"{r['speedup']:.5g}"), degradation_pct=float(f"{r['degradation_pct']:.5g}"))
              for r in pt]
        if pt:
            keep["peeling_only"] = dict(speedup=pt[0]["speedup"], degradation_pct=pt[0]["degradation_pct"])
    return keep


def dumps_record(s):
    """The summary as JSON with one table row per line."""
    head = ",\n".join(f" {json.dumps(k)}: {json.dumps(v)}" for k, v in s.items() if k != "table")
    rows = ",\n  ".join(json.dumps(r) for r in s.get("table", []))
    return "{\n" + head + ',\n "table": [\n  ' + rows + "\n ]\n}\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--space", choices=["grid", "flat", "full"], default="grid")
    ap.add_argument("--ligands", type=int, default=None, help="default 100,000 (grid) or 20,000 (flat, full)")
    ap.add_argument("--fit-ligands", type=int, default=None, help="default 4,000 (grid) or 1,000; 0: no model")
    ap.add_argument("--poses", type=int, default=8, help="initial poses of the flat and full spaces")
    ap.add_argument("--plain-ligands", type=int, default=128)
    ap.add_argument("--out", default=None)
    ap.add_argument("--summary", default=None, help="also write the summary record here")
    ap.add_argument("--checkpoint", default=None, help="directory of finished shards (resumes a stopped run)")
    args = ap.parse_args()
    grid = args.space == "grid"
    ligands = args.ligands if args.ligands is not None else (100_000 if grid else 20_000)
    fit = args.fit_ligands if args.fit_ligands is not None else (4_000 if grid else 1_000)
    t0 = time.time()
    res = run(ligands, fit, args.plain_ligands, space_name=args.space, poses=args.poses,
              log=lambda *a: print(*a, file=sys.stderr), checkpoint=args.checkpoint, fit_repeats=3 if grid else 1)
    res["wall_s"] = time.time() - t0
    txt = json.dumps(res)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt)
    if args.summary:
        s = summary(res)
        s["wall_s"] = round(res["wall_s"], 1)
        s["command"] = "python -m paper_1901_06363_gb300.knobsweep " + " ".join(sys.argv[1:])
        with open(args.summary, "w") as f:
            f.write(dumps_record(s))
    print(txt)


if __name__ == "__main__":
    main()
