"""Pins of the oracle's local refinement (trilinear score gradient, pose degrees of freedom, ascent loop).

The refinement is not in the paper (it only mentions steepest descent); what
fixes it is the mathematics: the trilinear interpolant reproduces linear
fields exactly, the analytic gradients must match central finite differences
of separately coded forward functions, rigid motions and torsions preserve
bond lengths and bond angles, each torsion delta changes exactly its own
dihedral, and accepted steps only ever lower S.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import indep
import oracle
import synth
import synth.configs as C


def _linear_pocket(n=20, h=0.5, slope=(3, 5, 7)):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    K = (slope[0] * x + slope[1] * y + slope[2] * z + 1).astype(np.uint16)
    pk = synth.Pocket((n, n, n), h, (0.25, -0.5, 1.0), (2.0, 2.0, 2.0), [[0, 0, 0]])
    return oracle.OraclePocket(pk, K=K), np.array(slope, np.float64)


def test_trilinear_linear_field_exact():
    opk, slope = _linear_pocket()
    rng = np.random.default_rng(1)
    t = rng.uniform(0.0, 19.0, (30, 3))
    x = t * opk.h + opk.origin
    S, dS, inside = oracle.trilinear_grad(opk, x)
    assert inside
    assert S == pytest.approx(float((t @ slope + 1).sum()), rel=1e-13)
    assert np.allclose(dS, slope / opk.h, rtol=0, atol=1e-9)


def test_trilinear_outside_penalty_gradient():
    # clip_box=0: the field at the clamped position plus the squared excess (grid units)
    opk, slope = _linear_pocket()
    t = np.array([[-2.0, 5.5, 7.25], [3.0, 21.5, 4.0], [1.0, 2.0, -0.5]])
    x = t * opk.h + opk.origin
    S, dS, inside = oracle.trilinear_grad(opk, x, clip=0)
    assert not inside
    tc = np.clip(t, 0, 19)
    assert S == pytest.approx(float((tc @ slope + 1).sum() + ((t - tc) ** 2).sum()), rel=1e-13)
    want = np.where(t != tc, 2 * (t - tc), slope) / opk.h
    assert np.allclose(dS, want, atol=1e-9)


def test_trilinear_gradient_matches_central_differences():
    pk = synth.pocket(8, 48, 0.5, C.ELLIPSOID)
    opk = oracle.OraclePocket(pk)
    rng = np.random.default_rng(2)
    t = rng.uniform(8.0, 40.0, (40, 3))
    frac = t - np.floor(t)
    t = np.where((frac < 1e-2) | (frac > 1 - 1e-2), t + 0.05, t)  # away from cell faces
    x = t * opk.h + opk.origin
    _, dS, _ = oracle.trilinear_grad(opk, x)
    eps = 1e-6
    for i in range(len(x)):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += eps
            xm[i, a] -= eps
            fd = (oracle.score(opk, xp, mode=1)[0] - oracle.score(opk, xm, mode=1)[0]) / (2 * eps)
            assert dS[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def _lig(seed=21, l=26, t=5):
    b = synth.ligand_batch(seed, np.array([l]), np.array([t]))
    x, bonds, rot = indep.ligand(b, 0)
    return b, x, bonds, rot


def _dihedral(p0, p1, p2, p3):
    b0, b1, b2 = p0 - p1, p2 - p1, p3 - p2
    b1 = b1 / np.linalg.norm(b1)
    v = b0 - (b0 @ b1) * b1
    w = b2 - (b2 @ b1) * b1
    return np.arctan2(np.cross(b1, v) @ w, v @ w)


def test_dof_apply_preserves_geometry_and_sets_each_dihedral():
    b, x, bonds, rot = _lig()
    T = len(rot)
    tor = oracle.torsions(b, 0)
    rng = np.random.default_rng(3)
    q = np.concatenate([rng.normal(0, 1, 3), rng.normal(0, 0.6, 3), rng.uniform(-np.pi, np.pi, T)])
    z = oracle.dof_apply(b, 0, x, q)
    # bond lengths and bond angles
    d0 = np.linalg.norm(x[bonds[:, 0]] - x[bonds[:, 1]], axis=1)
    d1 = np.linalg.norm(z[bonds[:, 0]] - z[bonds[:, 1]], axis=1)
    assert np.allclose(d0, d1, atol=1e-12)
    D = indep.graph_distance(len(x), bonds)
    i, j = np.nonzero(D == 2)
    assert np.allclose(np.linalg.norm(x[i] - x[j], axis=1), np.linalg.norm(z[i] - z[j], axis=1), atol=1e-12)
    # torsion k turns the dihedral (a, b_k, c_k, d) by exactly theta_k, whatever the other deltas
    adj = [set() for _ in range(len(x))]
    for u, v in bonds:
        adj[u].add(v)
        adj[v].add(u)
    for k in range(T):
        c, bb = tor["c"][k], tor["b"][k]
        a = min(adj[bb] - {c})
        d = min(adj[c] - {bb})
        turn = _dihedral(z[a], z[bb], z[c], z[d]) - _dihedral(x[a], x[bb], x[c], x[d])
        assert np.angle(np.exp(1j * (turn - q[6 + k]))) == pytest.approx(0.0, abs=1e-10)
        # the moving side of torsion k is the side without atom 0
        left, u, v = indep.sides(len(x), bonds, rot)[2 * k]
        side0 = left if left[0] else ~left
        assert np.array_equal(tor["mask"][k], ~side0)


def test_dof_apply_rigid_parts_and_full_turns():
    b, x, bonds, rot = _lig()
    T = len(rot)
    g = x.mean(0)
    t = np.array([0.3, -1.2, 2.0])
    w = np.array([0.4, -0.9, 0.2])
    z = oracle.dof_apply(b, 0, x, np.concatenate([t, w, np.zeros(T)]))
    assert np.allclose(z, Rotation.from_rotvec(w).apply(x - g) + g + t, atol=1e-12)
    z = oracle.dof_apply(b, 0, x, np.concatenate([np.zeros(3), w / np.linalg.norm(w) * 2 * np.pi,
                                                   np.full(T, 2 * np.pi)]))
    assert np.allclose(z, x, atol=1e-10)


def _smooth_objective(l, seed=4):
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(l, 3))
    wts = rng.uniform(0.5, 2.0, l)
    r = rng.normal(size=3)

    def f(z):
        return float((c * z).sum() + (wts * ((z - r) ** 2).sum(1)).sum())

    def df(z):
        return c + 2 * wts[:, None] * (z - r)

    return f, df


@pytest.mark.parametrize("at_zero", [True, False])
def test_dof_gradient_matches_central_differences(at_zero):
    b, x, bonds, rot = _lig(seed=22, l=30, t=6)
    n = 6 + len(rot)
    rng = np.random.default_rng(5)
    q = np.zeros(n) if at_zero else np.concatenate([rng.normal(0, 0.5, 3), rng.normal(0, 0.7, 3),
                                                    rng.uniform(-2, 2, n - 6)])
    f, df = _smooth_objective(len(x))
    z = oracle.dof_apply(b, 0, x, q)
    G = oracle.dof_grad(b, 0, x, q, df(z))
    eps = 1e-6
    for k in range(n):
        qp, qm = q.copy(), q.copy()
        qp[k] += eps
        qm[k] -= eps
        fd = (f(oracle.dof_apply(b, 0, x, qp)) - f(oracle.dof_apply(b, 0, x, qm))) / (2 * eps)
        assert G[k] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(G).max())


def test_score_dof_gradient_matches_central_differences():
    """d o / d q of the trilinear Eq. 1 at a docked pose against FP64 central differences at h = 1e-4."""
    pk = synth.pocket(8, 48, 0.5, C.ELLIPSOID)
    opk = oracle.OraclePocket(pk)
    b = synth.ligand_batch(23, np.array([24]), np.array([4]))
    kn = C.knobs(n_poses=4, score_mode=1, repetitions=1, seed=7)
    r = oracle.dock(opk, b, kn, xyz_out=True)
    p = int(r["best_pose"][0])
    z0 = r["pose_xyz"].reshape(4, 24, 3)[p]
    n = 6 + 4
    l = 24

    def o_of(z):
        S, _ = oracle.score(opk, z, mode=1)
        return l / (opk.h ** 2 * S)

    S, dS, inside = oracle.trilinear_grad(opk, z0)
    assert inside
    pz = -l / (opk.h ** 2 * S * S) * dS
    G = oracle.dof_grad(b, 0, z0, np.zeros(n), pz)
    eps = 1e-4
    checked = 0
    for k in range(n):
        e = np.zeros(n)
        e[k] = eps
        zp, zm = oracle.dof_apply(b, 0, z0, e), oracle.dof_apply(b, 0, z0, -e)
        # the finite difference is exact only when no atom crosses a cell face
        cells = [np.floor((zz - opk.origin) / opk.h) for zz in (zp, zm, z0)]
        if not (np.array_equal(cells[0], cells[2]) and np.array_equal(cells[1], cells[2])):
            continue
        fd = (o_of(zp) - o_of(zm)) / (2 * eps)
        assert G[k] == pytest.approx(fd, rel=1e-3, abs=1e-6 * np.abs(G).max())
        checked += 1
    assert checked >= 6


def _sampled(n=6, seed=24):
    pk = synth.pocket(8, 48, 0.5, C.ELLIPSOID)
    opk = oracle.OraclePocket(pk)
    l, t = synth.ligand_sizes(seed, n, 0, [16, 40, 0, 6])
    b = synth.ligand_batch(seed, l, t)
    kn = C.knobs(n_poses=4, score_mode=1, repetitions=1, seed=9)
    r = oracle.dock(opk, b, kn, xyz_out=True)
    xyz = np.zeros((int(b.atom_off[-1]), 3))
    px = r["pose_xyz"].reshape(-1, 3)
    for i in range(b.n):
        a0, a1 = b.atom_off[i], b.atom_off[i + 1]
        p = max(int(r["best_pose"][i]), 0)
        xyz[a0:a1] = px[a0 * 4 + p * (a1 - a0): a0 * 4 + (p + 1) * (a1 - a0)]
    return opk, b, xyz


def test_refine_descends_and_stays_feasible():
    opk, b, xyz = _sampled()
    steps = 20
    r = oracle.refine(opk, b, xyz, steps=steps)
    assert np.all(r["status"] == 0)
    assert np.all(r["S_final"] <= r["S_start"])
    assert np.any(r["S_final"] < r["S_start"])
    thr2 = 4.0
    for i in range(b.n):
        a0, a1 = b.atom_off[i], b.atom_off[i + 1]
        x, bonds, rot = indep.ligand(b, i)
        z = r["xyz"][a0:a1]
        # rigid geometry intact
        assert np.allclose(np.linalg.norm(z[bonds[:, 0]] - z[bonds[:, 1]], axis=1),
                           np.linalg.norm(xyz[a0:a1][bonds[:, 0]] - xyz[a0:a1][bonds[:, 1]], axis=1), atol=1e-9)
        # bump-free over every pair a torsion can move (Alg. 1 pair sets), restated from the graph
        for m, c, bb in indep.sides(len(x), bonds, rot):
            I = np.nonzero(m & (np.arange(len(x)) != c))[0]
            J = np.nonzero(~m & (np.arange(len(x)) != bb))[0]
            if len(I) and len(J):
                d2 = ((z[I][:, None] - z[J][None]) ** 2).sum(-1)
                assert d2.min() >= thr2
        # S never rises, and lambda follows the accept/reject rule
        S = r["S_start"][i]
        lam = oracle.LAMBDA0
        for s in range(steps):
            k = i * steps + s
            assert r["lam"][k] == pytest.approx(lam, rel=1e-15)
            if r["accept"][k]:
                assert r["S_new"][k] < S and (r["verdict"][k] & 7) == 7
                S = r["S_new"][k]
                lam = min(lam * oracle.GROW, oracle.LAMBDA_MAX)
            else:
                lam *= oracle.SHRINK
        assert r["S_final"][i] == S


def test_refine_replay_of_own_decisions_is_identical():
    opk, b, xyz = _sampled(n=4, seed=25)
    r = oracle.refine(opk, b, xyz, steps=10)
    r2 = oracle.refine(opk, b, xyz, steps=10, force_accept=r["accept"])
    assert np.array_equal(r["xyz"], r2["xyz"]) and np.array_equal(r["S_final"], r2["S_final"])
    # replaying all-reject keeps the start pose
    r3 = oracle.refine(opk, b, xyz, steps=10, force_accept=np.zeros_like(r["accept"]))
    assert np.array_equal(r3["xyz"], xyz) and np.array_equal(r3["S_final"], r3["S_start"])


def test_refine_rigid_ligand_moves_rigidly():
    opk, b, xyz = _sampled(n=3, seed=26)
    b0 = synth.ligand_batch(27, np.array([18]), np.array([0]))
    x = b0.xyz.astype(np.float64) - b0.xyz.mean(0) + opk.centre
    r = oracle.refine(opk, b0, x, steps=20)
    assert r["G"].shape == (1, 20, 6)
    z = r["xyz"]
    D0 = np.linalg.norm(x[:, None] - x[None], axis=-1)
    D1 = np.linalg.norm(z[:, None] - z[None], axis=-1)
    assert np.allclose(D0, D1, atol=1e-9)
    assert r["S_final"][0] <= r["S_start"][0]


def test_refine_bump_pairs_are_the_union_of_the_sweep_pair_sets():
    for seed, l, t in [(28, 30, 6), (29, 45, 10), (30, 16, 2)]:
        b = synth.ligand_batch(seed, np.array([l]), np.array([t]))
        x, bonds, rot = indep.ligand(b, 0)
        want = np.zeros((l, l), bool)
        for m, c, bb in indep.sides(l, bonds, rot):
            I = m & (np.arange(l) != c)
            J = ~m & (np.arange(l) != bb)
            want |= I[:, None] & J[None, :]
        want |= want.T
        assert np.array_equal(oracle.torsions(b, 0)["check"], want)
        # every such pair is at least 3 bonds apart
        assert indep.graph_distance(l, bonds)[want].min() >= 3
