"""Pins of the oracle's field (inner minimum of Eq. 1) and score (Eq. 1)."""
import json
import os

import numpy as np
import pytest
from scipy.ndimage import distance_transform_edt

import oracle
import synth
from conftest import GOLDEN


class _Pk:
    def __init__(self, dims, h, origin, pts, centre=(0, 0, 0)):
        self.dims, self.h = tuple(dims), h
        self.origin, self.centre = np.array(origin, float), np.array(centre, float)
        self.pts = np.array(pts, np.int32).reshape(-1, 3)


def _hand():
    with open(os.path.join(GOLDEN, "eq1_hand.json")) as f:
        return json.load(f)


def test_field_hand_values():
    g = _hand()
    K = oracle.field(g["grid"]["dims"], g["grid"]["points"])
    for s in g["field_samples"]:
        x, y, z = s["voxel"]
        assert K[z, y, x] == s["K"], s["why"]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_field_equals_euclidean_distance_transform(seed):
    # scipy's exact EDT gives the distance to the nearest probe voxel; squared and floored it is K
    rng = np.random.default_rng(seed)
    dims = (23, 17, 11)
    pts = np.stack([rng.integers(0, d, 9) for d in dims], 1)
    K = oracle.field(dims, pts)
    mask = np.ones(dims[::-1], bool)
    mask[pts[:, 2], pts[:, 1], pts[:, 0]] = False
    edt = distance_transform_edt(mask)
    ref = np.maximum(np.rint(edt ** 2), 1).astype(np.int64)
    assert np.array_equal(K.astype(np.int64), ref)


def test_field_of_synthetic_pocket():
    pk = synth.pocket(7, 48, 0.5, (8, 6, 5))
    K = oracle.field(pk.dims, pk.pts)
    assert K.min() == 1
    assert np.all(K[pk.pts[:, 2], pk.pts[:, 1], pk.pts[:, 0]] == 1)
    # probe lattice stride 3: inside the cavity every voxel is within 1+1+1 of a probe
    c = np.rint((pk.centre - pk.origin) / pk.h).astype(int)
    assert K[c[2], c[1], c[0]] <= 3


def test_eq1_hand_scores():
    g = _hand()
    pk = _Pk(g["grid"]["dims"], g["grid"]["h"], g["grid"]["origin"], g["grid"]["points"])
    opk = oracle.OraclePocket(pk)
    for s in g["scores"]:
        mode = {"nearest": 0, "trilinear": 1, "exact": 2}[s["mode"]]
        S, inside = oracle.score(opk, s["atoms_A"], mode=mode)
        assert S == pytest.approx(s["S"], abs=1e-12), s["why"]
        l = len(s["atoms_A"])
        assert l / (pk.h ** 2 * S) == pytest.approx(s["o"], rel=1e-12)
        assert inside


def test_nearest_on_voxel_centres_sums_the_field():
    pk = synth.pocket(7, 48, 0.5, (8, 6, 5))
    opk = oracle.OraclePocket(pk)
    rng = np.random.default_rng(3)
    v = rng.integers(0, 48, (20, 3))
    x = pk.origin + pk.h * v
    S, inside = oracle.score(opk, x, mode=0)
    assert inside
    assert S == float(opk.K[v[:, 2], v[:, 1], v[:, 0]].astype(np.int64).sum())


def test_trilinear_at_nodes_equals_nearest():
    pk = synth.pocket(7, 48, 0.5, (8, 6, 5))
    opk = oracle.OraclePocket(pk)
    rng = np.random.default_rng(4)
    v = rng.integers(1, 46, (30, 3))
    x = pk.origin + pk.h * v
    assert oracle.score(opk, x, mode=1)[0] == pytest.approx(oracle.score(opk, x, mode=0)[0], abs=1e-9)


def test_trilinear_error_bound_single_point():
    # f(t) = |t - p|^2 is a sum of 1-D parabolas; trilinear interpolation adds at most 1/4 per axis
    p = np.array([20, 21, 19])
    pk = _Pk((40, 40, 40), 0.5, (0, 0, 0), [p])
    opk = oracle.OraclePocket(pk)
    rng = np.random.default_rng(5)
    for _ in range(200):
        t = rng.uniform(2, 37, 3)
        if np.all(np.abs(t - p) < 2.5):
            continue  # keep the cell away from the floor at 1
        x = pk.h * t
        tri = oracle.score(opk, [x], mode=1)[0]
        exact = float(((t - p) ** 2).sum())
        assert exact - 1e-9 <= tri <= exact + 0.75 + 1e-9


def _proper_signed_permutations():
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            Q = np.zeros((3, 3))
            for i in range(3):
                Q[i, perm[i]] = signs[i]
            if round(np.linalg.det(Q)) == 1:
                out.append(Q)
    return out


def test_score_invariant_under_grid_symmetries():
    n = 32
    rng = np.random.default_rng(6)
    pts = rng.integers(4, n - 4, (15, 3))
    pk = _Pk((n, n, n), 0.5, (0, 0, 0), pts)
    opk = oracle.OraclePocket(pk)
    t = rng.uniform(3, n - 4, (25, 3))
    base = [oracle.score(opk, pk.h * t, mode=m)[0] for m in (0, 1, 2)]
    c = (n - 1) / 2.0
    for Q in _proper_signed_permutations():
        pts2 = np.rint((pts - c) @ Q.T + c).astype(np.int32)
        t2 = (t - c) @ Q.T + c
        opk2 = oracle.OraclePocket(_Pk((n, n, n), 0.5, (0, 0, 0), pts2))
        for m in (0, 1, 2):
            assert oracle.score(opk2, pk.h * t2, mode=m)[0] == pytest.approx(base[m], rel=1e-12)


def test_score_invariant_under_integer_voxel_shift():
    n = 32
    rng = np.random.default_rng(7)
    pts = rng.integers(4, 20, (10, 3))
    t = rng.uniform(4, 20, (12, 3))
    shift = np.array([5, 3, 7])
    a = oracle.OraclePocket(_Pk((n, n, n), 0.5, (0, 0, 0), pts))
    b = oracle.OraclePocket(_Pk((n, n, n), 0.5, (0, 0, 0), pts + shift))
    for m in (0, 1, 2):
        assert oracle.score(b, 0.5 * (t + shift), mode=m)[0] == pytest.approx(oracle.score(a, 0.5 * t, mode=m)[0],
                                                                                rel=1e-12)


def test_outside_box_clip_and_clamp():
    n = 10
    pk = _Pk((n, n, n), 1.0, (0, 0, 0), [[2, 2, 2]])
    opk = oracle.OraclePocket(pk)
    # nearest: inside iff -0.5 <= t < n - 0.5
    assert oracle.score(opk, [[-0.49, 0, 0]], mode=0)[1]
    assert not oracle.score(opk, [[-0.51, 0, 0]], mode=0)[1]
    assert not oracle.score(opk, [[9.5, 0, 0]], mode=0)[1]
    # clamped lookup plus the squared excess beyond the box edge
    S, inside = oracle.score(opk, [[12.0, 2.0, 2.0]], mode=0, clip=0)
    assert not inside
    assert S == pytest.approx(float(opk.K[2, 2, 9]) + (12.0 - 9.5) ** 2)
    # trilinear: inside iff 0 <= t <= n - 1
    assert oracle.score(opk, [[9.0, 0, 0]], mode=1)[1]
    assert not oracle.score(opk, [[9.01, 0, 0]], mode=1)[1]
    S, _ = oracle.score(opk, [[-1.0, 2.0, 2.0]], mode=1, clip=0)
    assert S == pytest.approx(float(opk.K[2, 2, 0]) + 1.0)
