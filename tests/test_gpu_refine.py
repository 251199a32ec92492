"""Parity of the refinement stage and the differentiable score (CUDA, through the C ABI) with the FP64 oracle.

Tolerances: every gradient entry within 1e-3 relative of the FP64 oracle
gradient and of FP64 central differences, |g_k - o_k| <= 1e-3 |o_k| + FLOOR *
max_k |o_k|, where the floor (2e-5 of the ligand's largest entry) only matters
for entries near zero: an entry is a sum of per-atom terms of up to the
largest entry's size, so the FP32 sum of a few dozen of them carries an
absolute rounding error of about 1e-6 of that size, whatever the entry's own
value. Scores within 1e-4 relative; poses within 1e-3 Å RMSD. The refinement
is compared by replay: the oracle commits the GPU's accept decisions and
every step's gradient, trial score and verdict are checked at the shared state.
"""
import numpy as np
import pytest

import oracle
import synth
import synth.configs as C

pytestmark = pytest.mark.gpu

REL_G = 1e-3
FLOOR = 2e-5  # absolute floor per gradient entry, as a fraction of the ligand's largest entry
REL_S = 1e-4
RMSD = 1e-3
AMB_BUMP = 4e-4  # Å^2 band around bump_thr^2, as in the sweep's replay
WORST = []  # worst entry ratio of every gradient comparison (<= 1 passes)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_06363_gb300 import Docker
    d = Docker(0)
    pk = synth.pocket(8, 48, 0.5, C.ELLIPSOID)
    pid = d.init_pocket(pk)
    opk = oracle.OraclePocket(pk)
    yield torch, d, pk, pid, opk
    d.close()


def _sampled_poses(torch, d, pid, b, seed=9, n_poses=8):
    """Best sampled pose per ligand from the GPU's own trilinear dock_run (the refinement's start)."""
    bid = d.upload_ligands(b)
    kn = C.knobs(n_poses=n_poses, score_mode=1, repetitions=1, seed=seed)
    res, xyz = d.run(bid, [pid], kn, b.n, int(b.atom_off[-1]))
    return bid, res, xyz[0].astype(np.float64)


def _batch(seed, n, lo=16, hi=40, tlo=0, thi=8):
    l, t = synth.ligand_sizes(seed, n, 0, [lo, hi, tlo, thi])
    return synth.ligand_batch(seed, l, t)


def _near_face(opk, x, delta=1e-3):
    t = (np.asarray(x, np.float64) - opk.origin) / opk.h
    return bool(np.any(np.abs(t - np.round(t)) <= delta))


def _elem(a, b):
    """Worst entry of |a_k - b_k| / (REL_G |b_k| + FLOOR max|b|): at most 1 when every entry agrees."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    tol = REL_G * np.abs(b) + FLOOR * max(np.abs(b).max(), 1e-30)
    r = float((np.abs(a - b) / tol).max())
    WORST.append(r)
    return r


def test_score_and_adjoint_match_oracle(env):
    torch, d, pk, pid, opk = env
    b = _batch(31, 12)
    bid, res, xyz = _sampled_poses(torch, d, pid, b)
    rng = np.random.default_rng(0)
    for clip in (1, 0):
        x = xyz + (rng.normal(0, 0.3, xyz.shape) if clip else rng.normal(0, 4.0, xyz.shape))
        xt = torch.tensor(x, dtype=torch.float32, device="cuda").reshape(-1)
        o = d.score_trilinear(bid, pid, xt, clip=clip).cpu().numpy()
        go = torch.tensor(rng.uniform(0.5, 2.0, b.n), dtype=torch.float32, device="cuda")
        g = d.score_trilinear_grad(bid, pid, xt, go, clip=clip).cpu().numpy().reshape(-1, 3)
        x32 = xt.cpu().numpy().astype(np.float64).reshape(-1, 3)
        for i in range(b.n):
            a0, a1 = b.atom_off[i], b.atom_off[i + 1]
            S, dS, _ = oracle.trilinear_grad(opk, x32[a0:a1], clip=clip)
            l = a1 - a0
            assert o[i] == pytest.approx(l / (pk.h ** 2 * S), rel=REL_S)
            if _near_face(opk, x32[a0:a1]):
                continue  # one-sided gradient on a cell face
            want = float(go[i]) * (-l / (pk.h ** 2 * S * S)) * dS
            assert _elem(g[a0:a1], want) <= 1, i


def test_dof_apply_and_adjoint_match_oracle(env):
    torch, d, pk, pid, opk = env
    b = _batch(32, 10, 16, 48, 0, 10)
    bid = d.upload_ligands(b)
    n, natoms, lmax, tmax = d.batch_info(bid)
    qs = 6 + tmax + 3  # a wider stride than needed
    rng = np.random.default_rng(1)
    q = np.zeros((n, qs))
    _, t = b.sizes()
    for i in range(n):
        q[i, :6] = np.concatenate([rng.normal(0, 0.5, 3), rng.normal(0, 0.8, 3)])
        q[i, 6:6 + t[i]] = rng.uniform(-2, 2, t[i])
    x = b.xyz.astype(np.float64)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda").reshape(-1)
    qt = torch.tensor(q, dtype=torch.float32, device="cuda")
    z = d.dof_apply(bid, xt, qt).cpu().numpy().reshape(-1, 3)
    p = rng.normal(size=(natoms, 3))
    G = d.dof_grad(bid, xt, qt, torch.tensor(p, dtype=torch.float32, device="cuda").reshape(-1)).cpu().numpy()
    for i in range(n):
        a0, a1 = b.atom_off[i], b.atom_off[i + 1]
        T = int(t[i])
        zo = oracle.dof_apply(b, i, x[a0:a1], q[i, :6 + T])
        assert np.abs(z[a0:a1] - zo).max() <= 1e-4
        Go = oracle.dof_grad(b, i, x[a0:a1], q[i, :6 + T], p[a0:a1])
        assert _elem(G[i, :6 + T], Go) <= 1, i
        assert np.all(G[i, 6 + T:] == 0)


def test_autograd_pose_score_gradient(env):
    """d o / d q through torch.autograd (both passes in the CUDA kernels) vs the FP64 oracle and FP64 FD."""
    torch, d, pk, pid, opk = env
    from paper_1901_06363_gb300.autograd import pose_score
    b = _batch(33, 8, 20, 40, 2, 6)
    bid, res, xyz = _sampled_poses(torch, d, pid, b)
    n, natoms, lmax, tmax = d.batch_info(bid)
    xt = torch.tensor(xyz, dtype=torch.float32, device="cuda").reshape(-1)
    q = torch.zeros((n, 6 + tmax), dtype=torch.float32, device="cuda", requires_grad=True)
    o = pose_score(d, bid, pid, xt, q)
    o.sum().backward()
    G = q.grad.cpu().numpy()
    _, t = b.sizes()
    x32 = xt.detach().cpu().numpy().astype(np.float64).reshape(-1, 3)
    checked = 0
    for i in range(n):
        a0, a1 = b.atom_off[i], b.atom_off[i + 1]
        l, T = a1 - a0, int(t[i])
        if _near_face(opk, x32[a0:a1]):
            continue  # one-sided gradient on a cell face
        S, dS, inside = oracle.trilinear_grad(opk, x32[a0:a1])
        Go = oracle.dof_grad(b, i, x32[a0:a1], np.zeros(6 + T), -l / (pk.h ** 2 * S * S) * dS)
        assert _elem(G[i, :6 + T], Go) <= 1, i
        # FP64 central differences (h = 1e-4) where no atom crosses a cell face
        eps = 1e-4
        fmax = np.abs(Go).max()
        for k in range(6 + T):
            e = np.zeros(6 + T)
            e[k] = eps
            zp = oracle.dof_apply(b, i, x32[a0:a1], e)
            zm = oracle.dof_apply(b, i, x32[a0:a1], -e)
            cells = [np.floor((zz - opk.origin) / opk.h) for zz in (zp, zm, x32[a0:a1])]
            if not (np.array_equal(cells[0], cells[2]) and np.array_equal(cells[1], cells[2])):
                continue
            fd = (l / (pk.h ** 2 * oracle.score(opk, zp, mode=1)[0]) -
                  l / (pk.h ** 2 * oracle.score(opk, zm, mode=1)[0])) / (2 * eps)
            assert abs(G[i, k] - fd) <= REL_G * abs(fd) + FLOOR * fmax, (i, k)
            WORST.append(abs(G[i, k] - fd) / (REL_G * abs(fd) + FLOOR * fmax))
            checked += 1
    assert checked >= 20


def _replay_check(b, kn, g, orc, xyz_start):
    steps = int(kn["refine_steps"])
    assert np.array_equal(g["status"], orc["status"])
    stats = dict(steps=0, accepted=0, face=0)
    for i in range(b.n):
        assert g["S_start"][i] == pytest.approx(orc["S_start"][i], rel=REL_S)
        if g["status"][i]:
            continue
        T = int(b.rot_off[i + 1] - b.rot_off[i])
        for s in range(steps):
            k = i * steps + s
            Gg, Go = g["G"][i, s, :6 + T], orc["G"][i, s, :6 + T]
            assert g["lam"][k] == orc["lam"][k]
            if orc["flags"][k] & 8:
                stats["face"] += 1  # one-sided gradient: the oracle took the GPU's direction
            else:
                assert _elem(Gg, Go) <= 1, (i, s)
                assert g["D"][k] == pytest.approx(orc["D"][k], rel=REL_G)
            if g["D"][k] > 0:
                assert g["S_new"][k] == pytest.approx(orc["S_new"][k], rel=REL_S)
                amb = orc["flags"][k]
                vg, vo = g["verdict"][k], orc["verdict"][k]
                if not amb & 1:
                    assert (vg & 1) == (vo & 1), (i, s)
                if not amb & 2:
                    assert (vg & 2) == (vo & 2), (i, s)
                if not amb & 4:
                    assert (vg & 4) == (vo & 4), (i, s)
            stats["steps"] += 1
            stats["accepted"] += int(g["accept"][k])
        assert g["S_final"][i] == pytest.approx(orc["S_final"][i], rel=REL_S)
        a0, a1 = b.atom_off[i], b.atom_off[i + 1]
        dd = g["xyz"][a0:a1] - orc["xyz"][a0:a1]
        assert np.sqrt((dd ** 2).sum(1).mean()) <= RMSD
    return stats


def test_refine_replay_parity(env):
    torch, d, pk, pid, opk = env
    b = _batch(34, 16, 16, 48, 0, 10)
    bid, res, xyz = _sampled_poses(torch, d, pid, b)
    kn = C.knobs(refine_steps=20)
    g = d.refine_trace(bid, pid, kn, xyz)
    orc = oracle.refine(opk, b, xyz.astype(np.float32).astype(np.float64), steps=20, force_accept=g["accept"], force_G=g["G"],
                        amb_delta=1e-3, amb_bump=AMB_BUMP, amb_rel=REL_S)
    st = _replay_check(b, kn, g, orc, xyz)
    assert st["accepted"] > 20
    # the device-memory form returns the same results
    xin = torch.tensor(xyz, dtype=torch.float32, device="cuda").reshape(-1)
    out, xo = d.refine(bid, [pid], kn, xin)
    assert np.array_equal(out.cpu().numpy().view(np.float32).reshape(-1, 4)[:, 0], g["result"]["score"])
    assert np.array_equal(xo.cpu().numpy().reshape(-1, 3), g["xyz"])
    # refined o is l / (h^2 S_final) and never below the sampled start
    l, _ = b.sizes()
    assert np.allclose(g["result"]["score"], l / (pk.h ** 2 * g["S_final"]), rtol=1e-6)
    assert np.all(g["S_final"] <= g["S_start"])


def test_refine_edge_cases(env):
    torch, d, pk, pid, opk = env
    # no rotatable bonds (6 DOF only), a single atom, zero steps, clip off, start pose outside the box
    one = synth.LigandBatch([0, 1], [0, 0], [0, 0], np.zeros((1, 3), np.float32), np.zeros((0, 2), np.int32),
                            np.zeros(0, np.int32))
    for b in (synth.ligand_batch(35, np.array([14, 20]), np.array([0, 3])), one):
        bid = d.upload_ligands(b)
        x = b.xyz.astype(np.float64) - b.xyz.mean(0) + pk.centre
        for kn in (C.knobs(refine_steps=12), C.knobs(refine_steps=0), C.knobs(refine_steps=12, clip_box=0)):
            g = d.refine_trace(bid, pid, kn, x)
            orc = oracle.refine(opk, b, x.astype(np.float32).astype(np.float64), steps=kn["refine_steps"],
                                clip=kn["clip_box"], force_accept=g["accept"], force_G=g["G"], amb_delta=1e-3, amb_bump=AMB_BUMP,
                                amb_rel=REL_S)
            _replay_check(b, kn, g, orc, x)
        far = x + np.array([100.0, 0, 0])
        g = d.refine_trace(bid, pid, C.knobs(refine_steps=5), far)
        assert np.all(g["status"] == 1) and np.all(g["result"]["status"] == 1)
        assert np.array_equal(g["xyz"], far.astype(np.float32))


def test_differentiation_workload_sampled(env):
    """4,096 ligands (20-60 atoms, 3-10 torsions), 64^3 trilinear field, 64 poses, 4 reps, then 20 refinement steps."""
    torch, d, _, _, _ = env
    pks, b, kn = C.differentiation()
    pid = d.init_pocket(pks[0])
    bid = d.upload_ligands(b)
    natoms = int(b.atom_off[-1])
    res, xyz = d.run(bid, [pid], kn, b.n, natoms)
    assert np.all(res["status"] == 0)
    xin = torch.tensor(xyz, dtype=torch.float32, device="cuda").reshape(-1)
    out, xo = d.refine(bid, [pid], kn, xin)
    out = out.cpu().numpy().view(np.float32).reshape(-1, 4)
    ref = out[:, 0]
    # the refined score is never below the trilinear score of the sampled pose
    o0 = d.score_trilinear(bid, pid, xin).cpu().numpy()
    assert np.all(ref >= o0 * (1 - 1e-6))
    assert np.mean(ref > o0) > 0.5
    # 256 sampled ligands replayed step by step against the oracle
    sample = np.sort(np.random.default_rng(4).choice(b.n, 256, replace=False))
    sub = b.subset(sample)
    opk = oracle.OraclePocket(pks[0])
    bs = d.upload_ligands(sub, ids=sample)
    xs = np.concatenate([xyz[0, b.atom_off[i]:b.atom_off[i + 1]] for i in sample]).astype(np.float64)
    g = d.refine_trace(bs, pid, kn, xs)
    orc = oracle.refine(opk, sub, xs, steps=20, force_accept=g["accept"], force_G=g["G"], amb_delta=1e-3,
                        amb_bump=AMB_BUMP, amb_rel=REL_S)
    st = _replay_check(sub, kn, g, orc, xs)
    assert st["steps"] == 256 * 20 and st["accepted"] > 256
    assert np.array_equal(g["result"]["score"], ref[sample])
    print(f"refinement replay: {st}; worst gradient entry ratio {max(WORST):.3f} over {len(WORST)} comparisons")
