"""Replay parity between the CUDA trace and the FP64 oracle (test infrastructure).

The greedy sweep is a chain of argmax decisions, so the oracle replays the
GPU's committed choice at every sweep (force_k) and, at that shared state,
checks every candidate the GPU evaluated:

  * feasibility equals the oracle's unless the oracle flags the candidate as
    ambiguous (a pair within the bump band of the threshold, or an atom within
    the voxel-boundary band of the box edge);
  * S (grid units; o = l / (h^2 S)) lies in the oracle's interval over
    voxel-boundary alternatives, widened by the relative tolerance;
  * the GPU's choice is the first minimum of its own values (exact), and it
    equals the oracle's own choice unless the two tie within tolerance or one
    of them carries an ambiguity flag.

Final S per pose must agree the same way, and final coordinates within RMSD.
"""
from __future__ import annotations

import numpy as np

import oracle

REL = 1e-4          # per-candidate score tolerance (relative)
AMB_DELTA = 1e-3    # voxel-boundary band, grid units
AMB_BUMP = 2e-3     # bump band around thr^2, Å^2
RMSD = 1e-3         # final pose tolerance, Å


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


def check(batch, kn, gpu, orc, rel=REL):
    """Compare a GPU trace with the oracle's replay; returns a dict of counts, raises AssertionError on a mismatch."""
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
    stats = dict(sweeps=total, candidates=0, ambiguous=0, choice_differs=0)

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

    peeled = peeled_sweeps(batch, kn) if kn.get("enable_refinement", 0) else np.zeros(total, bool)
    for s in np.nonzero(live_sweep)[0]:
        evaluated = ost[s] != -2
        assert np.array_equal(evaluated, gst[s] != -2), f"sweep {s}: evaluated slots differ"
        for j in np.nonzero(evaluated)[0]:
            stats["candidates"] += 1
            amb = oamb[s, j]
            if amb:
                stats["ambiguous"] += 1
            feas_amb = amb & 6
            if not feas_amb:
                assert gst[s, j] == ost[s, j], f"sweep {s} slot {j}: status gpu {gst[s, j]} oracle {ost[s, j]}"
            if gst[s, j] == 1 and ost[s, j] == 1:
                lo, hi = olo[s, j], ohi[s, j]
                tol = rel * abs(oS[s, j])
                assert lo - tol <= gS[s, j] <= hi + tol, \
                    f"sweep {s} slot {j}: S gpu {gS[s, j]} oracle {oS[s, j]} [{lo}, {hi}]"
        # the GPU's choice is the first minimum of its own values
        k = gpu["chosen_k"][s]
        feas = np.nonzero(gst[s] == 1)[0]
        if len(feas):
            vals = gS[s, feas]
            own = feas[np.argmin(vals)]  # argmin returns the first minimum
            if peeled[s]:
                # with tile peeling only the incumbent and the tile's angles compete
                cut = 1 + 360 // oracle.peel_tile(kn["hp_step"])
                comp = np.array([j for j in feas if j == 0 or j >= cut])
                own = comp[np.argmin(gS[s, comp])]
            assert k == own, f"sweep {s}: committed {k}, first minimum {own}"
        # and agrees with the oracle's own choice unless ambiguous
        ko = orc["own_k"][s]
        if k != ko:
            stats["choice_differs"] += 1
            near = abs(oS[s, k] - oS[s, ko]) <= rel * abs(oS[s, ko])
            assert near or oamb[s, k] or oamb[s, ko], \
                f"sweep {s}: gpu chose {k} (S={oS[s, k]}), oracle {ko} (S={oS[s, ko]})"

    # final per-pose S is the GPU's own last committed value (each commit was
    # checked against the oracle above), and coordinates agree within RMSD
    gpS = gpu["pose_S"].astype(np.float64)
    start = 0
    for b in range(batch.n):
        for p in range(N):
            n = int(nsw[b])
            i = b * N + p
            if live[i]:
                last = gi[i]
                for s in range(start, start + n):
                    k = gpu["chosen_k"][s]
                    if k != 0:
                        last = gS[s, k]
                assert gpS[i] == np.float32(last), f"ligand {b} pose {p}: final S {gpS[i]} vs last commit {last}"
            start += n
    gx = gpu["pose_xyz"].reshape(-1, 3).astype(np.float64)
    ox = orc["pose_xyz"].reshape(-1, 3)
    natoms = int(batch.atom_off[-1])
    for b in range(batch.n):
        l = batch.atom_off[b + 1] - batch.atom_off[b]
        for p in range(N):
            if not live[b * N + p]:
                continue
            o = batch.atom_off[b] * N + p * l
            d = gx[o:o + l] - ox[o:o + l]
            rmsd = float(np.sqrt((d * d).sum(1).mean()))
            assert rmsd <= RMSD, f"ligand {b} pose {p}: RMSD {rmsd}"
    stats["natoms"] = natoms
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
