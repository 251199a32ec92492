"""Replay parity between the CUDA trace and the FP64 oracle (test infrastructure).

The greedy sweep is a chain of argmax decisions, so the oracle replays the
GPU's committed choice at every sweep (force_k) and, at that shared state,
checks every candidate the GPU evaluated:

  * feasibility equals the oracle's unless the oracle puts the candidate in a
    feasibility band (bit 1: a pair within AMB_BUMP of thr^2; bit 2: an atom
    within AMB_DELTA of the box edge);
  * S (grid units; o = l / (h^2 S)) lies in the oracle's interval over
    voxel-boundary alternatives within AMB_DELTA, widened by the relative
    tolerance;
  * the GPU's choice is the first minimum of its own values (exact), and it
    equals the oracle's own choice unless the two tie within tolerance, their
    intervals overlap (so either order is a correct rounding of the same
    state), or one of them changed feasibility inside a band.

Final S per pose must equal the GPU's last committed value, and final
coordinates must agree within RMSD.

Why these bands. The GPU works in FP32 grid units (coordinates below 2^8, an
ulp of at most 2^-16) and commits each chosen angle by rounding; over a
run's commits its coordinates drift from the oracle's FP64 ones (the
measured maximum is reported as max_dev_A: typically 2e-5 to 7e-5 Å at the
end of a run, 1.4e-4 Å at most over the GPU suite). A nearest voxel can
differ only for an atom that close to a voxel face, far inside the band of
1e-3 voxel. A squared distance near thr^2 = (2 Å)^2 moves by at most about
2 * 2 Å * (the drift of the pair's difference) plus the FP32 rounding of
the GPU's test value (A - thr^2) + B cos + C sin, whose sign decides (under
1e-5 Å^2): about 2e-4 Å^2 for a typical drift of
5e-5 Å. The band of 4e-4 Å^2 is the parity protocol's; over the GPU suite's
75 million compared candidates every feasibility difference lay inside it
(the suite prints the counts).
"""
from __future__ import annotations

import os

import numpy as np

import oracle

REL = 1e-4          # per-candidate score tolerance (relative)
AMB_DELTA = 1e-3    # voxel-boundary band, grid units
AMB_BUMP = 4e-4     # bump band around thr^2, Å^2
RMSD = 1e-3         # final pose tolerance, Å
MAX_BAND_FRAC = 0.01  # at most this fraction of candidates may sit in a feasibility band (large cases)

RECORD = []  # (label, counts) of every check in this process; the test session prints them at its end


def replay(opk, batch, kn, gpu, nthreads=None, ids=None):
    """Oracle run that commits the GPU's choices, with parity flags."""
    return oracle.dock(opk, batch, kn, trace=True, force_k=gpu["chosen_k"], amb_delta=AMB_DELTA, amb_bump=AMB_BUMP,
                       nthreads=nthreads, xyz_out=True, ids=ids)


def peeled_sweeps(batch, kn):
    """Per sweep (trace order): True where tile peeling applies (hp fragments, Alg. 2)."""
    import indep
    N, R = int(kn["n_poses"]), int(kn["repetitions"])
    out = []
    for b in range(batch.n):
        x, bonds, rot = indep.ligand(batch, b)
        sides = indep.sides(len(x), bonds, rot)
        fine = [not (m.sum() / len(x) <= kn["threshold"]) for m, _, _ in sides]
        out.extend((fine * R) * N)
    return np.array(out, bool) & bool(kn.get("enable_refinement", 0))


def _fail(msg, rows):
    raise AssertionError(f"{msg} at {rows[:10]}")


def check(batch, kn, gpu, orc, rel=REL, max_band_frac=MAX_BAND_FRAC, label=None):
    """Compare a GPU trace with the oracle's replay; returns a dict of counts, raises AssertionError on a mismatch.

    Counts: candidates compared; amb_score / amb_bump / amb_box, the candidates in each band; flips,
    candidates whose feasibility differs (only inside a band); interval_used, feasible candidates whose
    GPU S lies off the oracle's own value but inside its interval; choice_differs and its reasons
    (tie, overlap, flip); max_dev_A and max_rmsd_A of the final coordinates."""
    pmax = gpu["pmax"]
    assert orc["pmax"] == pmax
    N = int(kn["n_poses"])
    total = len(gpu["chosen_k"])
    gS = gpu["cand_S"].reshape(total, pmax).astype(np.float64)
    gst = gpu["cand_status"].reshape(total, pmax)
    oS = orc["cand_S"].reshape(total, pmax)
    olo = orc["cand_lo"].reshape(total, pmax)
    ohi = orc["cand_hi"].reshape(total, pmax)
    ost = orc["cand_status"].reshape(total, pmax)
    oamb = orc["cand_amb"].reshape(total, pmax)
    stats = dict(sweeps=total, candidates=0, amb_score=0, amb_bump=0, amb_box=0, flips=0, interval_used=0,
                 choice_differs=0, choice_tie=0, choice_overlap=0, choice_flip=0, max_dev_A=0.0, max_rmsd_A=0.0)

    # pose-level status and initial scores
    assert np.array_equal(gpu["pose_status"], orc["pose_status"]), "initial-pose skip flags differ"
    live = orc["pose_status"] == 0
    gi = gpu["pose_init_S"].astype(np.float64)
    lo, hi = orc["pose_init_lo"], orc["pose_init_hi"]
    bad = live & ((gi < lo - rel * lo) | (gi > hi + rel * hi))
    assert not np.any(bad), f"initial S differs at poses {np.nonzero(bad)[0][:10]}"

    # sweeps belonging to live poses
    _, t = batch.sizes()
    nsw = kn["repetitions"] * 2 * t.astype(np.int64)
    owner = np.repeat(np.repeat(np.arange(batch.n), N), np.repeat(nsw, N))
    pose_of = np.concatenate([np.repeat(np.arange(N), n) for n in nsw]) if total else np.zeros(0, int)
    live_sweep = live[owner * N + pose_of] if total else np.zeros(0, bool)
    rows = np.nonzero(live_sweep)[0]

    if len(rows):
        gS, gst, oS, olo, ohi, ost, oamb = (a[rows] for a in (gS, gst, oS, olo, ohi, ost, oamb))
        evaluated = ost != -2
        if not np.array_equal(evaluated, gst != -2):
            _fail("evaluated slots differ", rows[np.nonzero((evaluated != (gst != -2)).any(1))[0]])
        ncand = int(evaluated.sum())
        stats["candidates"] = ncand
        stats["amb_score"] = int((evaluated & ((oamb & 1) != 0)).sum())
        stats["amb_bump"] = int((evaluated & ((oamb & 2) != 0)).sum())
        stats["amb_box"] = int((evaluated & ((oamb & 4) != 0)).sum())
        band = evaluated & ((oamb & 6) != 0)
        flip = evaluated & (gst != ost)
        if np.any(flip & ~band):
            r = np.nonzero((flip & ~band).any(1))[0]
            _fail(f"feasibility differs outside the bands (gpu {gst[flip & ~band][:5]}, "
                  f"oracle {ost[flip & ~band][:5]})", rows[r])
        stats["flips"] = int(flip.sum())
        both = evaluated & (gst == 1) & (ost == 1)
        tol = rel * np.abs(oS)
        out = both & ((gS < olo - tol) | (gS > ohi + tol))
        if np.any(out):
            i, j = np.nonzero(out)
            _fail(f"S outside the oracle's interval (gpu {gS[i[0], j[0]]}, oracle {oS[i[0], j[0]]} "
                  f"[{olo[i[0], j[0]]}, {ohi[i[0], j[0]]}])", rows[i])
        stats["interval_used"] = int((both & (np.abs(gS - oS) > tol)).sum())

        # the GPU's choice is the first minimum of its own feasible values (with tile peeling only the
        # incumbent and the tile's angles compete)
        k = gpu["chosen_k"][rows]
        elig = gst == 1
        if kn.get("enable_refinement", 0):
            peeled = peeled_sweeps(batch, kn)[rows]
            cut = 1 + 360 // oracle.peel_tile(kn["hp_step"])
            cols = np.arange(pmax)
            elig = elig & ~(peeled[:, None] & (cols[None, :] > 0) & (cols[None, :] < cut))
        v = np.where(elig, gS, np.inf)
        own = np.argmin(v, axis=1)  # the first minimum
        if not np.array_equal(own, k):
            _fail("committed slot is not the first minimum of the GPU's values", rows[np.nonzero(own != k)[0]])

        # and it agrees with the oracle's own choice unless the two are interchangeable
        ko = orc["own_k"][rows]
        d = np.nonzero(k != ko)[0]
        stats["choice_differs"] = len(d)
        for i in d:
            a, b = k[i], ko[i]
            if abs(oS[i, a] - oS[i, b]) <= rel * abs(oS[i, b]):
                stats["choice_tie"] += 1
            elif gst[i, b] != ost[i, b] or gst[i, a] != ost[i, a]:
                # one of the two changed feasibility inside a band (checked above)
                stats["choice_flip"] += 1
            elif olo[i, a] - rel * abs(oS[i, a]) <= ohi[i, b] + rel * abs(oS[i, b]):
                stats["choice_overlap"] += 1
            else:
                _fail(f"gpu chose {a} (S={oS[i, a]}), oracle {b} (S={oS[i, b]})", rows[i:i + 1])
        if ncand >= 20000 and max_band_frac is not None:
            frac = float(band.sum()) / ncand
            assert frac <= max_band_frac, f"{frac:.4f} of the candidates sit in a feasibility band"

    # final per-pose S is the GPU's own last committed value (each commit was checked against the oracle
    # above), and coordinates agree within RMSD
    gpS = gpu["pose_S"].astype(np.float64)
    kall = gpu["chosen_k"]
    gS_all = gpu["cand_S"].reshape(total, pmax)
    committed = np.nonzero(kall != 0)[0]
    ends = np.cumsum(np.repeat(nsw, N))  # sweeps of pose i: [ends[i] - nsw, ends[i])
    starts = ends - np.repeat(nsw, N)
    for i in np.nonzero(live)[0]:
        s0, s1 = int(starts[i]), int(ends[i])
        j = np.searchsorted(committed, s1) - 1
        if j >= 0 and committed[j] >= s0:
            last = gS_all[committed[j], kall[committed[j]]]
        else:
            last = gpu["pose_init_S"][i]
        assert gpS[i] == np.float32(last), f"pose {i}: final S {gpS[i]} vs last commit {last}"
    gx = gpu["pose_xyz"].reshape(-1, 3).astype(np.float64)
    ox = orc["pose_xyz"].reshape(-1, 3)
    natoms = int(batch.atom_off[-1])
    if natoms:
        l = np.diff(batch.atom_off).astype(np.int64)
        pose_start = (batch.atom_off[:-1].astype(np.int64)[:, None] * N + np.arange(N)[None, :] * l[:, None]).ravel()
        pose_len = np.repeat(l, N)
        d2 = ((gx - ox) ** 2).sum(1)
        msd = np.add.reduceat(d2, pose_start) / pose_len
        rmsd = np.sqrt(msd)[live]
        if np.any(rmsd > RMSD):
            _fail(f"final coordinates differ (RMSD {rmsd.max()} Å)", np.nonzero(live)[0][rmsd > RMSD])
        mask = np.repeat(live, pose_len)
        stats["max_rmsd_A"] = float(rmsd.max()) if len(rmsd) else 0.0
        stats["max_dev_A"] = float(np.sqrt(d2[mask].max())) if mask.any() else 0.0
    stats["natoms"] = natoms
    if label is None:
        label = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0].split("::")[-1]
    RECORD.append((label, stats))
    return stats


def check_best(batch, kn, gpu_result, gpu_pose_S, gpu_pose_status, rel=REL):
    """The reported best pose is the first minimum of the per-pose S, and its score is l / (h^2 S)."""
    N = int(kn["n_poses"])
    for b in range(batch.n):
        S = gpu_pose_S[b * N:(b + 1) * N].astype(np.float64)
        st = gpu_pose_status[b * N:(b + 1) * N]
        r = gpu_result[b]
        if np.all(st != 0):
            assert r["status"] == 1 and r["pose"] == -1
            continue
        cand = np.nonzero(st == 0)[0]
        best = cand[np.argmin(S[cand])]
        assert r["pose"] == best and r["status"] == 0
