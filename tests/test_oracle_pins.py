"""Pins of the oracle parts every GPU parity check leans on: the candidate count of a sweep, the tile
of tile peeling, and the parity bands (the interval of a nearest-voxel term over its voxel-boundary
alternatives, the box band and the bump band). Each is checked against hand-computed values or a
brute-force count, not against the oracle's own formulas.
"""
import json
import math
import os

import numpy as np
import pytest

import indep
import oracle
import synth
from conftest import GOLDEN

DELTA = 1e-3  # voxel-boundary band of the parity checks, grid units


# ------------------------------------------------------------ candidate count (Alg. 1)

def test_n_angles_hand_values():
    with open(os.path.join(GOLDEN, "n_angles.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        assert oracle.n_angles(case["step"]) == case["count"], case


@pytest.mark.parametrize("step", [float(s) for s in range(1, 361)] + [1.5, 2.5, 3.7, 7.5, 22.5, 359.5])
def test_n_angles_brute_force(step):
    # count the angles k*step below one full turn by walking k upwards in exact rational steps
    num, den = (int(round(step * 10)), 10)
    k = 0
    while k * num < 360 * den:
        k += 1
    assert oracle.n_angles(step) == k


def test_peel_tile_hand_values_and_brute_force():
    with open(os.path.join(GOLDEN, "eq2_eq3_tile_peeling.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        assert oracle.peel_tile(case["step"]) == case["tile"], case
    for case in g["unsupported"]:
        assert oracle.peel_tile(case["step"]) == -1, case
    # brute force over integer steps: every divisor of 360 that is a multiple of the step, nearest to
    # sqrt(360 step), ties to the smaller
    for step in range(1, 361):
        divs = [x for x in range(1, 361) if 360 % x == 0 and x % step == 0]
        target = math.sqrt(360 * step)
        want = min(divs, key=lambda x: (abs(x - target), x)) if divs else -1
        assert oracle.peel_tile(float(step)) == want, step


# ------------------------------------------------------------ the parity bands

def _grid4():
    """4^3 grid, h = 1, origin 0, so the grid position of an atom is its coordinate. K(x, y, z) =
    1 + x + 4y + 16z, all distinct, so each voxel's value names it."""
    pk = synth.Pocket((4, 4, 4), 1.0, (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), np.array([[1, 1, 1]], np.int32))
    z, y, x = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
    K = (1 + x + 4 * y + 16 * z).astype(np.uint16)
    return oracle.OraclePocket(pk, K=K)


def _k(x, y, z):
    return 1 + x + 4 * y + 16 * z


def test_nearest_interval_two_alternatives():
    opk = _grid4()
    # x: t + 0.5 = 1.9995, voxel 1, 0.0005 below the edge to voxel 2; y, z at voxel centres
    D, lo, hi, fl = oracle.term(opk, (1.4995, 2.0, 2.0), delta=DELTA)
    assert (D, lo, hi) == (_k(1, 2, 2), _k(1, 2, 2), _k(2, 2, 2)) == (42, 42, 43)
    assert fl == 1 | 4  # inside, score interval, no box band


def test_nearest_interval_four_alternatives():
    opk = _grid4()
    # x within the band above voxel 1, y (t + 0.5 = 3.0005) within the band above the edge of voxels 2 and 3
    D, lo, hi, fl = oracle.term(opk, (1.4995, 2.5005, 2.0), delta=DELTA)
    alts = [_k(1, 3, 2), _k(2, 3, 2), _k(1, 2, 2), _k(2, 2, 2)]
    assert D == _k(1, 3, 2) == 46
    assert (lo, hi) == (min(alts), max(alts)) == (42, 47)
    assert fl == 1 | 4


def test_nearest_interval_outside_the_band_is_a_point():
    opk = _grid4()
    # 0.0015 from the edges on x and y: outside a 0.001 band (inside a doubled one)
    D, lo, hi, fl = oracle.term(opk, (1.4985, 2.5015, 2.0), delta=DELTA)
    assert D == lo == hi == _k(1, 3, 2)
    assert fl == 1
    # far from every edge
    D, lo, hi, fl = oracle.term(opk, (1.2, 2.7, 0.9), delta=DELTA)
    assert D == lo == hi == _k(1, 3, 1) and fl == 1
    # no band at all: a point
    D, lo, hi, fl = oracle.term(opk, (1.4995, 2.5005, 2.0), delta=0.0)
    assert D == lo == hi == _k(1, 3, 2) and fl == 1


def test_box_band_lower_edge():
    opk = _grid4()
    # t + 0.5 = 0.0005: voxel 0 (inside), its alternative -1 is outside the box
    for clip in (1, 0):
        D, lo, hi, fl = oracle.term(opk, (-0.4995, 1.0, 1.0), clip=clip, delta=DELTA)
        assert D == lo == hi == _k(0, 1, 1) == 21  # the outside alternative is dropped (clip) or clamps to 21 + 0
        assert fl == 1 | 2
    # just outside: t + 0.5 = -0.0005, voxel -1; 0.0005 beyond the box face at -0.5
    D, lo, hi, fl = oracle.term(opk, (-0.5005, 1.0, 1.0), clip=0, delta=DELTA)
    assert D == pytest.approx(21 + 0.0005 ** 2, abs=1e-15)
    assert lo == 21 and hi == D and fl == 2 | 4  # outside; the inside alternative 0 lies in the band
    D, lo, hi, fl = oracle.term(opk, (-0.5005, 1.0, 1.0), clip=1, delta=DELTA)
    assert D == lo == hi == 21 and fl == 2
    # outside the band: no box flag
    D, lo, hi, fl = oracle.term(opk, (-0.4985, 1.0, 1.0), clip=1, delta=DELTA)
    assert fl == 1


def test_box_band_upper_edge():
    opk = _grid4()
    # t + 0.5 = 3.9995: voxel 3, the alternative 4 lies outside the 4-voxel box
    D, lo, hi, fl = oracle.term(opk, (3.4995, 1.0, 1.0), clip=1, delta=DELTA)
    assert D == lo == hi == _k(3, 1, 1) and fl == 1 | 2
    D, lo, hi, fl = oracle.term(opk, (3.4985, 1.0, 1.0), clip=1, delta=DELTA)
    assert fl == 1


def test_box_band_trilinear_and_exact():
    opk = _grid4()
    # trilinear: inside iff 0 <= t <= n - 1; the band is delta around those faces
    assert oracle.term(opk, (0.0005, 1.0, 1.0), mode=1, delta=DELTA)[3] == 1 | 2
    assert oracle.term(opk, (0.0015, 1.0, 1.0), mode=1, delta=DELTA)[3] == 1
    assert oracle.term(opk, (2.9995, 1.0, 1.0), mode=1, delta=DELTA)[3] == 1 | 2
    assert oracle.term(opk, (3.0005, 1.0, 1.0), mode=1, delta=DELTA)[3] == 2
    # exact points: the box of the nearest-voxel lookup, the same band
    assert oracle.term(opk, (-0.4995, 1.0, 1.0), mode=2, delta=DELTA)[3] == 1 | 2
    assert oracle.term(opk, (-0.4985, 1.0, 1.0), mode=2, delta=DELTA)[3] == 1
    assert oracle.term(opk, (3.5005, 1.0, 1.0), mode=2, delta=DELTA)[3] == 2


def _rotor():
    """Four atoms in a chain, its middle bond rotatable, exactly representable coordinates:
    atom 0 (-0.5, 1.375, 0) on atom 1 (0, 0, 0), atom 3 (2, 1.375, 0) on atom 2 (1.5, 0, 0). Either side's
    sweep turns the one pair (0, 3); at angle theta its squared distance is 2.5^2 + 1.375^2 (2 - 2 cos theta):
    10.03125 at 90 and 270 degrees, 13.8125 at 180."""
    x = np.array([[-0.5, 1.375, 0.0], [0.0, 0.0, 0.0], [1.5, 0.0, 0.0], [2.0, 1.375, 0.0]], np.float32)
    return synth.LigandBatch([0, 4], [0, 3], [0, 1], x, np.array([[0, 1], [1, 2], [2, 3]], np.int32),
                             np.array([1], np.int32))


def _flat_pocket():
    """A constant field: every candidate ties with the incumbent, so no sweep moves the ligand."""
    pk = synth.Pocket((16, 16, 16), 1.0, (0.0, 0.0, 0.0), (8.0, 8.0, 8.0), np.array([[8, 8, 8]], np.int32))
    return oracle.OraclePocket(pk, K=np.full((16, 16, 16), 5, np.uint16))


@pytest.mark.parametrize("band", [4e-4, 2e-3])
def test_bump_band_hand_values(band):
    b = _rotor()
    opk = _flat_pocket()
    d90, d180 = 2.5 ** 2 + 1.375 ** 2 * 2, 2.5 ** 2 + 1.375 ** 2 * 4
    assert (d90, d180) == (10.03125, 13.8125)
    # (thr^2, expected status and band flag at slots 1, 2, 3 = 90, 180, 270 degrees)
    cases = [
        (d90 + 0.5 * band, [(0, 2), (1, 0), (0, 2)]),   # just infeasible, in the band
        (d90 + 2.0 * band, [(0, 0), (1, 0), (0, 0)]),   # infeasible, outside the band
        (d90 - 0.5 * band, [(1, 2), (1, 0), (1, 2)]),   # just feasible, in the band
        (d90 - 2.0 * band, [(1, 0), (1, 0), (1, 0)]),   # feasible, outside the band
        (d180 + 0.5 * band, [(0, 0), (0, 2), (0, 0)]),  # every candidate infeasible, 180 degrees in the band
        (d90, [(1, 2), (1, 0), (1, 2)]),                # equality is feasible
    ]
    for thr2, want in cases:
        kn = dict(hp_step=90.0, lp_step=90.0, threshold=0.0, repetitions=1, n_poses=1, enable_refinement=0,
                  clip_box=1, bump_thr=math.sqrt(thr2), score_mode=0, seed=0)
        r = oracle.dock(opk, b, kn, trace=True, amb_delta=DELTA, amb_bump=band)
        st = r["cand_status"].reshape(-1, r["pmax"])
        amb = r["cand_amb"].reshape(-1, r["pmax"])
        assert st.shape == (2, 4)  # left and right sweep; slots 0 (incumbent), 90, 180, 270
        for s in range(2):
            assert st[s, 0] == 1
            got = [(int(st[s, j]), int(amb[s, j]) & 2) for j in (1, 2, 3)]
            assert got == want, (thr2, s, got)
        assert np.all(r["chosen_k"] == 0)


def test_candidate_bands_are_the_sums_of_the_atom_bands():
    """The interval and the box flag of a traced candidate are the sum and the OR of its atoms' bands,
    recomputed here from an independent rotation of the candidate's atoms."""
    # a pocket small enough that some candidates reach the box edge
    pk = synth.pocket(31, 24, 0.5, (4.0, 3.5, 3.0))
    b = synth.ligand_batch(31, np.array([18]), np.array([3]))
    opk = oracle.OraclePocket(pk)
    kn = dict(hp_step=20.0, lp_step=20.0, threshold=0.0, repetitions=1, n_poses=6, enable_refinement=0,
              clip_box=1, bump_thr=2.0, score_mode=0, seed=3)
    delta = 0.05  # a wide band, so that plenty of atoms fall in it
    r = oracle.dock(opk, b, kn, trace=True, amb_delta=delta, xyz_out=True)
    x0, bonds, rot = indep.ligand(b, 0)
    sides = indep.sides(len(x0), bonds, rot)
    pmax, nsw = r["pmax"], int(r["nsweep"][0])
    lo = r["cand_lo"].reshape(-1, pmax)
    hi = r["cand_hi"].reshape(-1, pmax)
    amb = r["cand_amb"].reshape(-1, pmax)
    st = r["cand_status"].reshape(-1, pmax)
    X0 = r["init_xyz"].reshape(-1, 3)
    nbox = nscore = 0
    for p in range(kn["n_poses"]):
        if r["pose_status"][p]:
            continue
        X = X0[p * len(x0):(p + 1) * len(x0)].copy()
        for s in range(nsw):
            moving, c, bb = sides[s % len(sides)]
            row = p * nsw + s
            for j in range(1, pmax):
                if st[row, j] == -2:
                    continue
                Y = indep.rotate_side(X, moving, c, bb, math.radians(j * kn["hp_step"]))
                terms = [oracle.term(opk, y, delta=delta) for y in Y]
                box = any(t[3] & 2 for t in terms)
                assert bool(amb[row, j] & 4) == box
                if st[row, j] == 1:
                    assert lo[row, j] == pytest.approx(sum(t[1] for t in terms), abs=1e-9)
                    assert hi[row, j] == pytest.approx(sum(t[2] for t in terms), abs=1e-9)
                    assert bool(amb[row, j] & 1) == any(t[3] & 4 for t in terms)
                nbox += box
                nscore += bool(amb[row, j] & 1)
            k = r["chosen_k"][row]
            if k:
                X = indep.rotate_side(X, moving, c, bb, math.radians(k * kn["hp_step"]))
    assert nbox > 0 and nscore > 0
