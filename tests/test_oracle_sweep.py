"""Pins of the oracle's rotation, bump check, poses and greedy sweep (Alg. 1/2, Eq. 2/3)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import indep
import oracle
import synth
import synth.configs as C
from conftest import GOLDEN


# ------------------------------------------------------------------ rotation

def test_rotate_matches_rotation_vector():
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = rng.normal(size=(7, 3)) * 3
        c, b = rng.normal(size=3), rng.normal(size=3)
        th = rng.uniform(-7, 7)
        k = (c - b) / np.linalg.norm(c - b)
        ref = Rotation.from_rotvec(k * th).apply(x - c) + c
        assert np.allclose(oracle.rotate(x, c, b, th), ref, atol=1e-12)


def test_full_turn_is_identity():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(5, 3))
    assert np.allclose(oracle.rotate(x, [0, 0, 1], [0, 0, 0], 2 * math.pi), x, atol=1e-12)


def _bond_geometry(x, bonds):
    lengths = np.linalg.norm(x[bonds[:, 0]] - x[bonds[:, 1]], axis=1)
    angles = []
    l = len(x)
    nb = [[] for _ in range(l)]
    for u, v in bonds:
        nb[u].append(v)
        nb[v].append(u)
    for a in range(l):
        for i in range(len(nb[a])):
            for j in range(i + 1, len(nb[a])):
                p, q = x[nb[a][i]] - x[a], x[nb[a][j]] - x[a]
                angles.append(math.acos(np.clip(p @ q / np.linalg.norm(p) / np.linalg.norm(q), -1, 1)))
    return lengths, np.array(angles)


def test_dock_preserves_bond_lengths_and_angles():
    pks, b, kn = C.single()
    r = oracle.dock(oracle.OraclePocket(pks[0]), b, kn, xyz_out=True)
    x0, bonds, _ = indep.ligand(b, 0)
    L0, A0 = _bond_geometry(x0, bonds)
    X = r["pose_xyz"].reshape(kn["n_poses"], -1, 3)
    moved = 0
    for p in range(kn["n_poses"]):
        L, A = _bond_geometry(X[p], bonds)
        assert np.allclose(L, L0, atol=1e-9) and np.allclose(A, A0, atol=1e-9)
        moved += r["pose_S"][p] != r["pose_init_S"][p]
    assert moved > 0  # the sweep did change some conformations


def test_initial_poses_rigid_and_centred():
    pks, b, kn = C.single()
    r = oracle.dock(oracle.OraclePocket(pks[0]), b, kn, xyz_out=True)
    x0, _, _ = indep.ligand(b, 0)
    D0 = np.linalg.norm(x0[:, None] - x0[None], axis=-1)
    X = r["init_xyz"].reshape(kn["n_poses"], -1, 3)
    for p in range(kn["n_poses"]):
        assert np.allclose(X[p].mean(0), pks[0].centre, atol=1e-9)
        assert np.allclose(np.linalg.norm(X[p][:, None] - X[p][None], axis=-1), D0, atol=1e-9)
    # pose 0 is the input conformer, only translated
    assert np.allclose(X[0] - X[0].mean(0), x0 - x0.mean(0), atol=1e-9)


# -------------------------------------------------------------------- poses

def test_splitmix_published_outputs():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.json")) as f:
        g = json.load(f)
    assert [oracle.splitmix(g["seed"], i) for i in range(len(g["outputs"]))] == [int(v) for v in g["outputs"]]


def test_pose_rotations_are_uniform_rotations():
    Rs = np.array([oracle.pose_rotation(11, lid, p) for lid in range(40) for p in range(1, 101)])
    assert np.allclose(np.einsum("nij,nkj->nik", Rs, Rs), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(Rs), 1.0, atol=1e-12)
    # Haar measure: E[R] = 0 and E[trace R] = 0 (4000 samples, std of a mean ~ 0.01)
    assert np.abs(Rs.mean(0)).max() < 0.05
    assert abs(np.trace(Rs, axis1=1, axis2=2).mean()) < 0.08
    assert np.array_equal(oracle.pose_rotation(11, 3, 0), np.eye(3))


# -------------------------------------------------------------------- sweep

def _small_problem(l=14, t=2, seed=21, n_grid=40, step=30.0, **kw):
    pk = synth.pocket(seed + 1, n_grid, 0.5, (6, 5, 4))
    b = synth.ligand_batch(seed, np.array([l]), np.array([t]))
    kn = C.knobs(hp_step=step, lp_step=step, n_poses=3, repetitions=1, seed=seed, **kw)
    return pk, b, kn


def _replay_conformations(b, kn, r, pose):
    """Sweep-start conformations rebuilt from the initial pose and the committed angles."""
    x0, bonds, rot = indep.ligand(b, 0)
    sides = indep.sides(len(x0), bonds, rot)
    X = r["init_xyz"].reshape(kn["n_poses"], -1, 3)[pose].copy()
    nsw = r["nsweep"][0]
    base = r["sweep_base"][0] + pose * nsw
    out = []
    for s in range(nsw):
        moving, c, bb = sides[s % len(sides)]
        out.append((X.copy(), moving, c, bb))
        k = r["chosen_k"][base + s]
        X = indep.rotate_side(X, moving, c, bb, math.radians(k * kn["hp_step"]))
    return out, X, bonds


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_each_sweep_is_the_argmax_over_its_angles(seed):
    pk, b, kn = _small_problem(seed=seed)
    opk = oracle.OraclePocket(pk)
    r = oracle.dock(opk, b, kn, trace=True, xyz_out=True)
    P = oracle.n_angles(kn["hp_step"])
    x0, bonds, _ = indep.ligand(b, 0)
    gd = indep.graph_distance(len(x0), bonds)
    for pose in range(kn["n_poses"]):
        if r["pose_status"][pose]:
            continue
        confs, final, _ = _replay_conformations(b, kn, r, pose)
        base = r["sweep_base"][0] + pose * r["nsweep"][0]
        for s, (X, moving, c, bb) in enumerate(confs):
            S0, _ = indep.nearest_S(opk.K, pk.origin, pk.h, X)
            best, best_k = S0, 0
            for k in range(P):
                ci = (base + s) * r["pmax"] + k
                if k == 0:
                    assert r["cand_S"][ci] == S0
                    continue
                Y = indep.rotate_side(X, moving, c, bb, math.radians(k * kn["hp_step"]))
                S, inside = indep.nearest_S(opk.K, pk.origin, pk.h, Y)
                feasible = inside and not indep.clashes(Y, gd, kn["bump_thr"])
                assert r["cand_status"][ci] == (1 if feasible else (0 if indep.clashes(Y, gd, 2.0) else -1))
                if feasible:
                    assert r["cand_S"][ci] == S
                    if S < best:
                        best, best_k = S, k
            assert r["chosen_k"][base + s] == best_k
        assert r["pose_S"][pose] == indep.nearest_S(opk.K, pk.origin, pk.h, final)[0]
        assert np.allclose(r["pose_xyz"].reshape(kn["n_poses"], -1, 3)[pose], final, atol=1e-9)


def test_greedy_not_better_than_exhaustive():
    # 2 rotatable bonds, 90 degree steps: all 4^4 angle combinations of the 4 sweeps
    import itertools
    pk, b, kn = _small_problem(l=12, t=2, seed=31, step=90.0)
    kn["n_poses"] = 1
    opk = oracle.OraclePocket(pk)
    r = oracle.dock(opk, b, kn, trace=True, xyz_out=True)
    x0, bonds, rot = indep.ligand(b, 0)
    gd = indep.graph_distance(len(x0), bonds)
    sides = indep.sides(len(x0), bonds, rot)
    X0 = r["init_xyz"].reshape(1, -1, 3)[0]
    best = math.inf
    for ks in itertools.product(range(4), repeat=len(sides)):
        X = X0.copy()
        ok = True
        for (moving, c, bb), k in zip(sides, ks):
            X = indep.rotate_side(X, moving, c, bb, math.radians(90.0 * k))
            ok = ok and not indep.clashes(X, gd, 2.0)
        S, inside = indep.nearest_S(opk.K, pk.origin, pk.h, X)
        if ok and inside:
            best = min(best, S)
    assert best <= r["pose_S"][0]


def test_step_360_and_no_rotamers_keep_the_initial_pose():
    pk, b, kn = _small_problem()
    opk = oracle.OraclePocket(pk)
    kn2 = dict(kn, hp_step=360.0, lp_step=360.0)
    r = oracle.dock(opk, b, kn2)
    assert np.array_equal(r["pose_S"], r["pose_init_S"])
    b0 = synth.ligand_batch(5, np.array([10]), np.array([0]))
    r = oracle.dock(opk, b0, kn)
    assert np.array_equal(r["pose_S"], r["pose_init_S"])
    kn3 = dict(kn, repetitions=0)
    r = oracle.dock(opk, b, kn3)
    assert np.array_equal(r["pose_S"], r["pose_init_S"])


def test_repetitions_continue_from_their_own_output():
    pk, b, kn = _small_problem(seed=41, step=20.0)
    opk = oracle.OraclePocket(pk)
    r1 = oracle.dock(opk, b, kn, trace=True)
    r2 = oracle.dock(opk, b, dict(kn, repetitions=2), trace=True)
    n1, n2 = r1["nsweep"][0], r2["nsweep"][0]
    for p in range(kn["n_poses"]):
        a = r1["chosen_k"][p * n1:(p + 1) * n1]
        c = r2["chosen_k"][p * n2:(p + 1) * n2]
        assert np.array_equal(a, c[:n1])  # the first repetition is the R = 1 run
        assert r2["pose_S"][p] <= r1["pose_S"][p]
        # the incumbent never gets worse along the sweeps
        inc = r2["cand_S"].reshape(-1, r2["pmax"])[p * n2:(p + 1) * n2, 0]
        assert np.all(np.diff(inc) <= 0)


@pytest.mark.parametrize("seed", [61, 62, 63])
def test_a_repetition_without_a_move_is_a_fixed_point(seed):
    """A repetition that commits no angle leaves the pose where it started, so every later repetition repeats
    it: the pose after R repetitions equals the pose after the first still one (what lets the GPU stop a pose
    there). Checked against runs with more repetitions, pose by pose."""
    pk, b, kn = _small_problem(l=18, t=3, seed=seed, step=20.0)
    kn = dict(kn, n_poses=6)
    opk = oracle.OraclePocket(pk)
    R = 6
    runs = {r: oracle.dock(opk, b, dict(kn, repetitions=r), trace=True, xyz_out=True) for r in range(1, R + 1)}
    full = runs[R]
    ns = full["nsweep"][0] // R
    still = 0
    for p in range(kn["n_poses"]):
        ck = full["chosen_k"][p * R * ns:(p + 1) * R * ns].reshape(R, ns)
        quiet = np.flatnonzero((ck == 0).all(axis=1))
        if not len(quiet):
            continue
        still += 1
        r0 = int(quiet[0]) + 1  # repetitions up to and including the first still one
        assert (ck[r0:] == 0).all()  # nothing moves afterwards
        for r in range(r0, R + 1):
            assert runs[r]["pose_S"][p] == full["pose_S"][p]
            xa = runs[r]["pose_xyz"].reshape(kn["n_poses"], -1, 3)[p]
            assert np.array_equal(xa, full["pose_xyz"].reshape(kn["n_poses"], -1, 3)[p])
    assert still > 0


def test_threshold_selects_the_coarse_step():
    pk, b, kn = _small_problem(seed=51)
    opk = oracle.OraclePocket(pk)
    for thr, step in ((1.0, 90.0), (0.0, 30.0)):
        r = oracle.dock(opk, b, dict(kn, threshold=thr, lp_step=90.0, hp_step=30.0), trace=True)
        st = r["cand_status"].reshape(-1, r["pmax"])
        assert np.all((st != -2).sum(1) == oracle.n_angles(step))


def test_analytic_single_point_optimum():
    """Exact mode, one probe point, no clash test: S(theta) = A + B cos(theta) + C sin(theta)."""
    for seed in range(5):
        p0 = np.array([40, 40, 40])

        class Pk:
            dims, h, origin = (80, 80, 80), 0.5, np.zeros(3)
            pts = p0[None].astype(np.int32)
            centre = np.array([12.0, 20.0, 21.0])
        b = synth.ligand_batch(60 + seed, np.array([12]), np.array([1]))
        step = 5.0
        kn = C.knobs(hp_step=step, lp_step=step, n_poses=1, bump_thr=0.0, clip_box=0, score_mode=2, seed=seed)
        opk = oracle.OraclePocket(Pk)
        r = oracle.dock(opk, b, kn, trace=True, xyz_out=True)
        X = r["init_xyz"].reshape(-1, 3) / Pk.h  # grid units
        x0, bonds, rot = indep.ligand(b, 0)
        moving, c, bb = indep.sides(len(x0), bonds, rot)[0]
        k = (X[c] - X[bb]) / np.linalg.norm(X[c] - X[bb])
        B = C_ = 0.0
        for i in np.nonzero(moving)[0]:
            v = X[i] - X[c]
            a = X[c] + k * (k @ v)
            u = v - k * (k @ v)
            w = np.cross(k, u)
            B += 2 * (a - p0) @ u
            C_ += 2 * (a - p0) @ w
        theta = math.degrees(math.atan2(-C_, -B)) % 360.0
        frac = theta / step - math.floor(theta / step)
        if abs(frac - 0.5) < 1e-6:
            continue
        kstar = int(round(theta / step)) % oracle.n_angles(step)
        assert r["chosen_k"][0] == kstar


def _rotate_problem(pk, b, Q):
    n = pk.dims[0]
    c = (n - 1) / 2.0
    pts2 = np.rint((pk.pts - c) @ Q.T + c).astype(np.int32)
    t = (b.xyz.astype(np.float64) - pk.origin) / pk.h
    xyz2 = pk.origin + pk.h * ((t - c) @ Q.T + c)
    centre2 = pk.origin + pk.h * (((pk.centre - pk.origin) / pk.h - c) @ Q.T + c)
    pk2 = synth.Pocket(pk.dims, pk.h, pk.origin, centre2, pts2)
    b2 = synth.LigandBatch(b.atom_off, b.bond_off, b.rot_off, xyz2, b.bonds, b.rot, b.id_base)
    return pk2, b2, xyz2


def test_dock_invariant_under_grid_rotation():
    from test_oracle_field_score import _proper_signed_permutations
    pk, b, kn = _small_problem(seed=71, step=15.0)
    kn["n_poses"] = 1
    kn["score_mode"] = 2  # exact point form: no rounding edges
    r = oracle.dock(oracle.OraclePocket(pk), b, kn, trace=True)
    for Q in _proper_signed_permutations()[:8]:
        pk2, b2, xyz2 = _rotate_problem(pk, b, Q)
        # the input is in float32 for both: compare against a run on the same rounded input
        b2r = synth.LigandBatch(b.atom_off, b.bond_off, b.rot_off, xyz2.astype(np.float32), b.bonds, b.rot)
        r2 = oracle.dock(oracle.OraclePocket(pk2), b2r, kn, trace=True)
        assert np.array_equal(r2["chosen_k"], r["chosen_k"])
        assert r2["pose_S"][0] == pytest.approx(r["pose_S"][0], rel=1e-6)


# ------------------------------------------------------------ tile peeling

def test_eq3_tile_and_eq2_evaluations():
    with open(os.path.join(GOLDEN, "eq2_eq3_tile_peeling.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        x = oracle.peel_tile(case["step"])
        assert x == case["tile"]
        assert 360 // x + int(round(x / case["step"])) == case["evaluations"]
    # Eq. 3 as printed, 6*sqrt(10)*sqrt(step), is the minimiser of Eq. 2
    for step in (1.0, 2.0, 5.0):
        xs = np.linspace(1, 360, 200001)
        y = 360 / xs + xs / step
        assert xs[np.argmin(y)] == pytest.approx(6 * math.sqrt(10) * math.sqrt(step), rel=1e-3)


def test_peeling_evaluates_eq2_candidates():
    pk, b, kn = _small_problem(seed=81, step=1.0)
    kn.update(enable_refinement=1, n_poses=2)
    opk = oracle.OraclePocket(pk)
    r = oracle.dock(opk, b, kn, trace=True)
    st = r["cand_status"].reshape(-1, r["pmax"])
    evaluated = (st[:, 1:] != -2).sum(1)
    # 20 peels, then 18 angles of the best tile (unless no peel is feasible)
    assert np.all((evaluated == 38) | (evaluated == 20))
    assert np.any(evaluated == 38)
    # the committed slot is the best feasible one among the incumbent and the tile angles
    S = r["cand_S"].reshape(-1, r["pmax"])
    for s in range(len(st)):
        k = r["chosen_k"][s]
        cands = [0] + [j for j in range(21, 39) if st[s, j] == 1]
        best = min(cands, key=lambda j: (S[s, j], j))
        assert k == best


def test_threshold_boundary_is_inclusive():
    # Alg. 2: a fragment whose relative size equals the threshold takes the coarse step
    pk, b, kn = _small_problem(l=14, t=2, seed=91)
    opk = oracle.OraclePocket(pk)
    x0, bonds, rot = indep.ligand(b, 0)
    sides = indep.sides(len(x0), bonds, rot)
    m = int(sides[0][0].sum())
    kn2 = dict(kn, threshold=m / len(x0), lp_step=90.0, hp_step=30.0)
    r = oracle.dock(opk, b, kn2, trace=True)
    st = r["cand_status"].reshape(-1, r["pmax"])
    nsw = r["nsweep"][0]
    for p in range(kn["n_poses"]):
        for s in range(nsw):
            ms = int(sides[s % len(sides)][0].sum())
            expect = oracle.n_angles(90.0) if ms <= m else oracle.n_angles(30.0)
            assert (st[p * nsw + s] != -2).sum() == expect


def test_peels_sit_at_tile_centres():
    pk, b, kn = _small_problem(seed=83, step=2.0)
    kn.update(enable_refinement=1, n_poses=1, clip_box=0, bump_thr=0.0)
    opk = oracle.OraclePocket(pk)
    r = oracle.dock(opk, b, kn, trace=True, xyz_out=True)
    x = oracle.peel_tile(2.0)  # 24 degrees
    X = r["init_xyz"].reshape(-1, 3)
    x0, bonds, rot = indep.ligand(b, 0)
    moving, c, bb = indep.sides(len(x0), bonds, rot)[0]
    S = r["cand_S"].reshape(-1, r["pmax"])[0]
    for t in range(360 // x):
        Y = indep.rotate_side(X, moving, c, bb, math.radians(t * x + x / 2))
        assert S[1 + t] == indep.nearest_S(opk.K, pk.origin, pk.h, Y, clip=False)[0] or \
            not indep.nearest_S(opk.K, pk.origin, pk.h, Y)[1]
