"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import oracle
import parity
import synth
import synth.configs as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_06363_gb300 import Docker
    d = Docker(0)
    yield d
    d.close()


def _natoms(b):
    return int(b.atom_off[-1])


def trace_parity(dk, pk, batch, kn, opk=None, ids=None):
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(batch, ids=ids)
    g = dk.run_trace(bid, pid, kn, batch)
    orc = parity.replay(opk or oracle.OraclePocket(pk), batch, kn, g, ids=ids)
    stats = parity.check(batch, kn, g, orc)
    parity.check_best(batch, kn, g["result"], g["pose_S"], g["pose_status"])
    # the graph-captured batched run returns the trace run's results bit for bit
    res, xyz = dk.run(bid, [pid], kn, batch.n, _natoms(batch))
    assert np.array_equal(res.view(np.int32), g["result"].view(np.int32))
    # best-pose coordinates are that pose's final coordinates
    N = kn["n_poses"]
    px = g["pose_xyz"].reshape(-1, 3)
    for b in range(batch.n):
        if res[b]["status"]:
            continue
        l = batch.atom_off[b + 1] - batch.atom_off[b]
        o = batch.atom_off[b] * N + res[b]["pose"] * l
        assert np.array_equal(xyz[0, batch.atom_off[b]:batch.atom_off[b + 1]], px[o:o + l])
    dk.release_batch(bid)
    return stats, g, res


def test_field_bit_exact(dk):
    pks = [C.single()[0][0], synth.pocket(8, 64, 0.5, C.ELLIPSOID), synth.pocket(9, 96, 0.5, (11, 9, 7))]
    rng = np.random.default_rng(0)
    pks.append(synth.Pocket((37, 23, 19), 0.4, (1.0, -2.0, 0.5), (5.0, 3.0, 4.0),
                            np.stack([rng.integers(0, d, 50) for d in (37, 23, 19)], 1)))
    for pk in pks:
        pid = dk.init_pocket(pk)
        assert np.array_equal(dk.pocket_field(pid, pk.dims), oracle.field(pk.dims, pk.pts))


def test_single_ligand_config(dk):
    pks, b, kn = C.single()
    stats, g, res = trace_parity(dk, pks[0], b, kn)
    assert stats["candidates"] > 1000
    assert res[0]["status"] == 0 and res[0]["score"] > 0


@pytest.mark.parametrize("n_poses", [40, 7])
def test_small_batch_several_tiles(dk, n_poses):
    # 40 poses: a full warp plus a ragged 8-pose tail; 7 poses: a partial warp
    pk = synth.pocket(8, 64, 0.5, C.ELLIPSOID)
    l, t = synth.ligand_sizes(11, 16, 0, [16, 64, 2, 12])
    b = synth.ligand_batch(11, l, t)
    kn = C.knobs(n_poses=n_poses, hp_step=15.0, lp_step=15.0, repetitions=2, seed=5)
    stats, _, _ = trace_parity(dk, pk, b, kn)
    assert stats["candidates"] > 10000


def test_tile_shapes_bit_identical(dk):
    pk = synth.pocket(8, 64, 0.5, C.ELLIPSOID)
    l, t = synth.ligand_sizes(12, 24, 0, [16, 64, 2, 12])
    b = synth.ligand_batch(12, l, t)
    kn = C.knobs(n_poses=24, hp_step=10.0, lp_step=10.0, repetitions=1, seed=2)
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(b)
    ref = None
    for q, kc, w in [(1, 12, 4), (1, 36, 4), (2, 18, 2), (4, 8, 8), (8, 8, 4), (1, 8, 1)]:
        dk.set_tile(q, kc, w)
        res, xyz = dk.run(bid, [pid], kn, b.n, _natoms(b))
        if ref is None:
            ref = (res.copy(), xyz.copy())
        else:
            assert np.array_equal(res.view(np.int32), ref[0].view(np.int32)), (q, kc, w)
            assert np.array_equal(xyz, ref[1]), (q, kc, w)
    dk.set_tile(0, 0, 0)
    # plain one-launch-per-pair form: identical results
    res, xyz = dk.run(bid, [pid], dict(kn, plain_mode=1), b.n, _natoms(b))
    assert np.array_equal(res.view(np.int32), ref[0].view(np.int32))
    assert np.array_equal(xyz, ref[1])
    dk.release_batch(bid)


@pytest.mark.parametrize("variant", ["threshold", "noclip", "peel", "trilinear", "trilinear_noclip", "reps0",
                                     "step360", "exact", "exact_noclip", "exact_peel"])
def test_knob_variants(dk, variant):
    n_grid = 40 if variant in ("noclip", "trilinear_noclip", "exact_noclip") else 64
    pk = synth.pocket(13, n_grid, 0.5, (6, 5, 4))
    l, t = synth.ligand_sizes(13, 8, 0, [16, 48, 2, 8])
    b = synth.ligand_batch(13, l, t)
    kn = C.knobs(n_poses=12, hp_step=15.0, lp_step=15.0, repetitions=2, seed=3)
    kn.update({
        "threshold": dict(threshold=0.5, lp_step=45.0, hp_step=10.0),
        "noclip": dict(clip_box=0),
        "peel": dict(enable_refinement=1, hp_step=5.0, lp_step=30.0, threshold=0.3),
        "trilinear": dict(score_mode=1),
        "trilinear_noclip": dict(score_mode=1, clip_box=0),
        "reps0": dict(repetitions=0),
        "step360": dict(hp_step=360.0, lp_step=360.0),
        "exact": dict(score_mode=2),
        "exact_noclip": dict(score_mode=2, clip_box=0),
        "exact_peel": dict(score_mode=2, enable_refinement=1, hp_step=5.0, lp_step=30.0, threshold=0.3),
    }[variant])
    trace_parity(dk, pk, b, kn)


def test_heavy_ligand_split_keeps_results(dk):
    """With the nearest-voxel score a batch's plan may give a ligand more lanes per pose than the tile (the
    heaviest ligands of a batch, every ligand of a small one), and the poses still working take over the
    lanes of converged ones; neither changes a result: the default plan, a forced 2 lanes per pose and the
    traced run (which never remaps) agree bit for bit, as do the work counts that do not depend on which
    poses share a warp."""
    pk = synth.pocket(8, 64, 0.5, C.ELLIPSOID)
    l, t = synth.ligand_sizes(41, 12, 0, [16, 64, 2, 12])
    b = synth.ligand_batch(41, l, t)
    kn = C.knobs(n_poses=24, hp_step=15.0, lp_step=15.0, repetitions=4, seed=6)
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(b)
    res, xyz = dk.run(bid, [pid], kn, b.n, _natoms(b))
    st = dk.stats()
    dk.set_tile(2, 0, 0)
    res2, xyz2 = dk.run(bid, [pid], kn, b.n, _natoms(b))
    st2 = dk.stats()
    dk.set_tile(0, 0, 0)
    assert np.array_equal(res.view(np.int32), res2.view(np.int32))
    assert np.array_equal(xyz, xyz2)
    for key in ("candidates", "pair_bounds", "bump_pairs", "pose_reps_skipped"):
        assert st[key] == st2[key], key
    assert st["atom_updates"] + st["lookups_skipped"] == st2["atom_updates"] + st2["lookups_skipped"]
    g = dk.run_trace(bid, pid, kn, b)
    assert np.array_equal(res.view(np.int32), g["result"].view(np.int32))
    dk.release_batch(bid)


@pytest.mark.parametrize("clip", [1, 0])
def test_trilinear_non_cubic_grid(dk, clip):
    """Trilinear score on a 37 x 23 x 19 grid (h = 0.4 A, random probe points): the corner texture's three
    strides differ, and with clipping off every atom beyond an upper face is scored at the clamped
    position n - 1 exactly, where the texel's repeated corners take weight 0."""
    rng = np.random.default_rng(3)
    pk = synth.Pocket((37, 23, 19), 0.4, (1.0, -2.0, 0.5), (8.2, 2.4, 4.1),
                      np.stack([rng.integers(0, d, 80) for d in (37, 23, 19)], 1))
    l, t = synth.ligand_sizes(31, 8, 0, [12, 24, 2, 5])
    b = synth.ligand_batch(31, l, t)
    kn = C.knobs(n_poses=16, hp_step=20.0, lp_step=20.0, repetitions=2, seed=4, score_mode=1, clip_box=clip)
    stats, g, _ = trace_parity(dk, pk, b, kn)
    assert stats["candidates"] > 2000


def test_edge_cases(dk):
    pk = synth.pocket(14, 48, 0.5, C.ELLIPSOID)
    pid = dk.init_pocket(pk)
    kn = C.knobs(n_poses=5, repetitions=1, seed=1)
    # empty batch
    e = synth.LigandBatch(np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32),
                          np.zeros((0, 3), np.float32), np.zeros((0, 2), np.int32), np.zeros(0, np.int32))
    bid = dk.upload_ligands(e)
    res, xyz = dk.run(bid, [pid], kn, 0, 0)
    assert len(res) == 0
    # no rotatable bonds, a single atom, and a rotatable bond with a one-atom side
    b0 = synth.ligand_batch(3, np.array([12, 9]), np.array([0, 0]))
    one = synth.LigandBatch([0, 1], [0, 0], [0, 0], np.zeros((1, 3), np.float32), np.zeros((0, 2), np.int32),
                            np.zeros(0, np.int32))
    term = synth.ligand_batch(4, np.array([10]), np.array([0]))
    leaf = int(np.nonzero(np.bincount(term.bonds.ravel(), minlength=10) == 1)[0][0])
    e_leaf = int(np.nonzero((term.bonds == leaf).any(1))[0][0])
    term = synth.LigandBatch(term.atom_off, term.bond_off, [0, 1], term.xyz, term.bonds, [e_leaf])
    for batch in (b0, one, term):
        trace_parity(dk, pk, batch, kn)
    # every pose outside a tiny box: status 1
    tiny = synth.Pocket((6, 6, 6), 0.5, (-1.25, -1.25, -1.25), (0, 0, 0), [[3, 3, 3]])
    big = synth.ligand_batch(5, np.array([40]), np.array([4]))
    _, g, res = trace_parity(dk, tiny, big, kn)
    assert res[0]["status"] == 1 and res[0]["pose"] == -1 and res[0]["score"] == 0
    # one pose
    trace_parity(dk, pk, b0, dict(kn, n_poses=1))


def test_error_paths(dk):
    from paper_1901_06363_gb300 import DOCK_ERR_INVALID_ARG, DOCK_ERR_TOPOLOGY, DockError
    pk = synth.pocket(14, 48, 0.5, C.ELLIPSOID)
    pid = dk.init_pocket(pk)
    b = synth.ligand_batch(3, np.array([12]), np.array([2]))
    bid = dk.upload_ligands(b)
    for bad in (dict(hp_step=0.5), dict(n_poses=0), dict(n_poses=5000), dict(repetitions=-1), dict(bump_thr=-1.0),
                dict(score_mode=7)):
        with pytest.raises(DockError) as ei:
            dk.run(bid, [pid], C.knobs(**bad), b.n, _natoms(b))
        assert ei.value.code == DOCK_ERR_INVALID_ARG
    with pytest.raises(DockError) as ei:
        dk.run(bid, [pid + 100], C.knobs(), b.n, _natoms(b))
    assert ei.value.code == DOCK_ERR_INVALID_ARG
    # a ring: the closing bond does not split the ligand
    ring = synth.LigandBatch([0, 4], [0, 4], [0, 1], np.array([[0, 0, 0], [1.5, 0, 0], [1.5, 1.5, 0], [0, 1.5, 0]],
                                                               np.float32),
                             np.array([[0, 1], [1, 2], [2, 3], [3, 0]]), [1])
    with pytest.raises(DockError) as ei:
        dk.upload_ligands(ring)
    assert ei.value.code == DOCK_ERR_TOPOLOGY
    bad_atoms = synth.LigandBatch([0, 2], [0, 1], [0, 0], np.zeros((2, 3), np.float32), np.array([[0, 5]]),
                                  np.zeros(0, np.int32))
    with pytest.raises(DockError):
        dk.upload_ligands(bad_atoms)
    # a ligand larger than DOCK_MAX_ATOMS (255) is refused
    n = 256
    chain = synth.LigandBatch([0, n], [0, n - 1], [0, 0], np.stack([np.arange(n) * 1.5, np.zeros(n), np.zeros(n)], 1),
                              np.stack([np.arange(n - 1), np.arange(1, n)], 1), np.zeros(0, np.int32))
    with pytest.raises(DockError) as ei:
        dk.upload_ligands(chain)
    assert ei.value.code == DOCK_ERR_INVALID_ARG and "256 atoms" in str(ei.value)
    # non-finite and huge coordinates are refused before anything reaches the device, by both entry points
    for v in (np.nan, np.inf, -np.inf, 2e5):
        x = b.xyz.copy()
        x[3, 1] = v
        bad = synth.LigandBatch(b.atom_off, b.bond_off, b.rot_off, x, b.bonds, b.rot)
        with pytest.raises(DockError) as ei:
            dk.upload_ligands(bad)
        assert ei.value.code == DOCK_ERR_INVALID_ARG and "coordinate" in str(ei.value)
        with pytest.raises(DockError) as ei:
            dk.run_database(bad, [pid], C.knobs(), chunk=1)
        assert ei.value.code == DOCK_ERR_INVALID_ARG and "coordinate" in str(ei.value)


def test_bench_workload_sampled(dk):
    """1,024 ligands x 64^3 pocket, 64 poses, 10 degrees, 4 repetitions: the benchmark's launch, sampled."""
    pks, b, kn = C.batched()
    pid = dk.init_pocket(pks[0])
    bid = dk.upload_ligands(b)
    res, xyz = dk.run(bid, [pid], kn, b.n, _natoms(b))
    assert np.all(res["status"] == 0) and np.all(res["score"] > 0)
    # properties at full size: rigid geometry of every docked ligand is intact
    for i in range(b.n):
        a0, a1 = b.atom_off[i], b.atom_off[i + 1]
        bonds = b.bonds[b.bond_off[i]:b.bond_off[i + 1]]
        d0 = np.linalg.norm(b.xyz[a0:a1][bonds[:, 0]] - b.xyz[a0:a1][bonds[:, 1]], axis=1)
        d1 = np.linalg.norm(xyz[0, a0:a1][bonds[:, 0]] - xyz[0, a0:a1][bonds[:, 1]], axis=1)
        assert np.allclose(d0, d1, atol=2e-3)
    # 256 sampled ligands (a quarter of the batch, in four groups of 64): the same ligands (same ids) traced
    # alone give the same results as the full launch, and replay candidate by candidate against the oracle
    sample = np.sort(np.random.default_rng(2).choice(b.n, 256, replace=False))
    opk = oracle.OraclePocket(pks[0])
    tot = 0
    for part in np.split(sample, 4):
        sub = b.subset(part)
        stats, g, res_sub = trace_parity(dk, pks[0], sub, kn, opk=opk, ids=part)
        assert np.array_equal(res_sub.view(np.int32), res[part].view(np.int32))
        tot += stats["candidates"]
    assert tot > 10_000_000
    dk.release_batch(bid)


def test_exact_score_needs_probe_points(dk):
    from paper_1901_06363_gb300 import DOCK_ERR_UNSUPPORTED, DockError
    pk = synth.pocket(14, 48, 0.5, C.ELLIPSOID)
    K = oracle.field(pk.dims, pk.pts)
    bare = synth.Pocket(pk.dims, pk.h, pk.origin, pk.centre, np.zeros((0, 3), np.int32))
    pid = dk.init_pocket(bare, K=K)
    b = synth.ligand_batch(3, np.array([12]), np.array([2]))
    bid = dk.upload_ligands(b)
    with pytest.raises(DockError) as ei:
        dk.run(bid, [pid], C.knobs(score_mode=2), b.n, _natoms(b))
    assert ei.value.code == DOCK_ERR_UNSUPPORTED
    # the same pocket with its points gives the exact score, and nearest mode is unaffected by them
    pid2 = dk.init_pocket(pk)
    r0, _ = dk.run(bid, [pid], C.knobs(), b.n, _natoms(b))
    r1, _ = dk.run(bid, [pid2], C.knobs(), b.n, _natoms(b))
    assert np.array_equal(r0.view(np.int32), r1.view(np.int32))
    dk.release_batch(bid)


def test_autotune_picks_a_valid_shape_with_identical_results(dk):
    pk = synth.pocket(8, 64, 0.5, C.ELLIPSOID)
    l, t = synth.ligand_sizes(15, 96, 0, [16, 64, 2, 12])
    b = synth.ligand_batch(15, l, t)
    kn = C.knobs(n_poses=32, hp_step=10.0, lp_step=10.0, repetitions=1, seed=4)
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(b)
    ref, rx = dk.run(bid, [pid], kn, b.n, _natoms(b))
    q, kc, w = dk.autotune(bid, pid, kn)
    assert q in (1, 2, 4, 8) and kc in (8, 12, 18, 36) and w in (2, 4, 8)
    res, xyz = dk.run(bid, [pid], kn, b.n, _natoms(b))  # now with the tuned shape
    assert np.array_equal(res.view(np.int32), ref.view(np.int32)) and np.array_equal(xyz, rx)
    dk.release_batch(bid)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_run_to_run_bitwise_determinism(dk, mode):
    pk = synth.pocket(13, 48, 0.5, (6, 5, 4))
    l, t = synth.ligand_sizes(16, 24, 0, [16, 40, 1, 8])
    b = synth.ligand_batch(16, l, t)
    kn = C.knobs(n_poses=20, hp_step=20.0, lp_step=20.0, repetitions=2, seed=6, score_mode=mode)
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(b)
    outs = [dk.run(bid, [pid], kn, b.n, _natoms(b)) for _ in range(3)]
    for res, xyz in outs[1:]:
        assert np.array_equal(res.view(np.int32), outs[0][0].view(np.int32))
        assert np.array_equal(xyz, outs[0][1])
    dk.release_batch(bid)


def test_largest_ligands(dk):
    """Ligands up to DOCK_MAX_ATOMS (255): more lanes per pose so their poses fit a warp's slice."""
    pk = synth.pocket(8, 96, 0.5, (11, 9, 7))
    b = synth.ligand_batch(7, np.array([255, 200, 120, 33]), np.array([6, 5, 4, 3]))
    kn = C.knobs(n_poses=6, hp_step=30.0, lp_step=30.0, repetitions=1, seed=8, clip_box=0)
    stats, g, res = trace_parity(dk, pk, b, kn)
    assert stats["candidates"] > 500


@pytest.mark.parametrize("case", ["step1", "step1_peel", "step7", "thr0", "poses4096", "tiny_rotor"])
def test_stress_cases(dk, case):
    pk = synth.pocket(13, 64, 0.5, (6, 5, 4))
    if case == "tiny_rotor":
        # four atoms in a chain with its middle bond rotatable: one moving atom per side
        x = np.array([[0, 0, 0], [1.5, 0, 0], [2.0, 1.4, 0], [3.5, 1.4, 0.3]], np.float32)
        b = synth.LigandBatch([0, 4], [0, 3], [0, 1], x, np.array([[0, 1], [1, 2], [2, 3]], np.int32),
                              np.array([1], np.int32))
    else:
        l, t = synth.ligand_sizes(17, 3 if case == "poses4096" else 5, 0, [16, 40, 2, 6])
        b = synth.ligand_batch(17, l, t)
    kn = {
        "step1": C.knobs(n_poses=3, hp_step=1.0, lp_step=1.0, repetitions=1, seed=2),
        "step1_peel": C.knobs(n_poses=3, hp_step=1.0, lp_step=30.0, threshold=0.2, enable_refinement=1, seed=7),
        "step7": C.knobs(n_poses=5, hp_step=7.0, lp_step=20.0, threshold=0.3, seed=3),
        "thr0": C.knobs(n_poses=9, bump_thr=0.0, repetitions=2, seed=4),
        "poses4096": C.knobs(n_poses=4096, hp_step=45.0, lp_step=45.0, repetitions=1, seed=5),
        "tiny_rotor": C.knobs(n_poses=16, hp_step=10.0, lp_step=10.0, repetitions=2, seed=6),
    }[case]
    trace_parity(dk, pk, b, kn)


@pytest.mark.parametrize("n_grid", [64, 16])
def test_fixed_point_repetitions_are_counted_out(dk, n_grid):
    """Repetitions after one that committed no angle for a pose are not computed; the work counts
    exclude them and the results equal the traced run, which computes every repetition. On the 16^3
    grid many poses start outside the box and compute nothing."""
    pk = synth.pocket(8, n_grid, 0.5, C.ELLIPSOID)
    l, t = synth.ligand_sizes(18, 12, 0, [16, 40, 1, 6])
    b = synth.ligand_batch(18, l, t)
    kn = C.knobs(n_poses=16, hp_step=30.0, lp_step=30.0, repetitions=8, seed=9)
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(b)
    res, _ = dk.run(bid, [pid], kn, b.n, _natoms(b))
    st = dk.stats()
    full = 0
    for i in range(b.n):
        lb = int(b.atom_off[i + 1] - b.atom_off[i])
        tb = int(b.rot_off[i + 1] - b.rot_off[i])
        full += 2 * tb * (oracle.n_angles(30.0) - 1)
    full *= kn["n_poses"] * kn["repetitions"]
    assert st["pose_reps_skipped"] > 0
    assert 0 < st["candidates"] < full
    g = dk.run_trace(bid, pid, kn, b)
    assert np.array_equal(res.view(np.int32), g["result"].view(np.int32))
    # the traced run computes every repetition: from its chosen angles, a pose stops after its first
    # repetition that commits none (a pose outside the box computes none); count what is left out
    N, R = kn["n_poses"], kn["repetitions"]
    skipped, left_out, side_off = 0, 0, 0
    for i in range(b.n):
        ns = 2 * int(b.rot_off[i + 1] - b.rot_off[i])
        for p in range(N):
            if g["pose_status"][i * N + p] != 0:
                n = R
            else:
                ck = g["chosen_k"][N * R * side_off + p * R * ns:][:R * ns].reshape(R, ns)
                still = np.flatnonzero((ck == 0).all(axis=1))
                n = R - 1 - int(still[0]) if len(still) else 0
            skipped += n
            left_out += n * ns * (oracle.n_angles(30.0) - 1)
        side_off += ns
    assert st["pose_reps_skipped"] == skipped
    assert st["candidates"] == full - left_out
    if n_grid == 16:
        assert (g["pose_status"][:b.n * N] != 0).any()
    dk.release_batch(bid)


@pytest.mark.parametrize("score_mode", [0, 1])
def test_gated_lookups_are_counted_out(dk, score_mode):
    """Blocks of 6 candidates that the bump check rejected for every working pose of a warp are not scored; the
    count of lookups left out equals a replay of that rule on the traced run's candidate statuses (ligands of at
    most 32 atoms and 16 poses: one warp of 2 lanes per pose per ligand; 30 degrees: 11 candidates, blocks
    [0, 6) and [6, 11)), for the nearest-voxel and the trilinear score."""
    import indep
    pk = synth.pocket(8, 64, 0.5, C.ELLIPSOID)
    l, t = synth.ligand_sizes(23, 24, 0, [16, 32, 1, 6])
    b = synth.ligand_batch(23, l, t)
    kn = C.knobs(n_poses=16, hp_step=30.0, lp_step=30.0, repetitions=3, bump_thr=2.6, seed=2,
                 score_mode=score_mode)
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(b)
    dk.set_tile(2, 0, 0)  # forced: a small batch would otherwise spread each ligand's poses over more warps
    res, _ = dk.run(bid, [pid], kn, b.n, _natoms(b))
    st = dk.stats()
    dk.set_tile(0, 0, 0)
    g = dk.run_trace(bid, pid, kn, b)
    assert np.array_equal(res.view(np.int32), g["result"].view(np.int32))
    N, R, nc = kn["n_poses"], kn["repetitions"], oracle.n_angles(30.0) - 1
    pmax = len(g["cand_status"]) // len(g["chosen_k"])
    status = g["cand_status"].reshape(-1, pmax)
    expected, upd, side_off = 0, 0, 0
    for i in range(b.n):
        x, bonds, rot = indep.ligand(b, i)
        sides = indep.sides(len(x), bonds, rot)
        ns = len(sides)
        nmov = [int(m.sum()) - 1 for m, _, _ in sides]
        rows = lambda p, r: N * R * side_off + p * R * ns + r * ns  # noqa: E731
        working = [g["pose_status"][i * N + p] == 0 for p in range(N)]
        for r in range(R):
            for si in range(ns):
                cs = [status[rows(p, r) + si, 1:1 + nc] for p in range(N) if working[p]]
                for a, e in ((0, 6), (6, nc)):
                    if all((c[a:e] == 0).all() for c in cs):
                        expected += len(cs) * (e - a) * nmov[si]
                upd += len(cs) * nc * nmov[si]
            # a pose that committed nothing in this repetition computes no further one
            for p in range(N):
                if working[p] and not any(g["chosen_k"][rows(p, r) + si] for si in range(ns)):
                    working[p] = False
        side_off += ns
    assert expected > 0
    assert st["lookups_skipped"] == expected
    assert st["atom_updates"] == upd - expected
    dk.release_batch(bid)


def test_out_of_memory_is_an_error_and_the_context_recovers(dk):
    """A run whose scratch cannot fit the GPU (16 pockets x 30,000 ligands x 4,096 poses: about 0.8 TB of
    per-pose coordinates) fails with DOCK_ERR_OUT_OF_MEMORY before any launch; the same context then docks a
    small batch with the results of the module's context. It runs in a context of its own, so that the
    shared one keeps its small scratch."""
    from paper_1901_06363_gb300 import DOCK_ERR_OUT_OF_MEMORY, Docker, DockError
    pk = synth.pocket(14, 48, 0.5, C.ELLIPSOID)
    own = Docker(0)
    pid = own.init_pocket(pk)
    big = C.sweep_batch(30000)
    bid = own.upload_ligands(big)
    with pytest.raises(DockError) as ei:
        own.run(bid, [pid] * 16, C.knobs(n_poses=4096), big.n, _natoms(big), xyz=False)
    assert ei.value.code == DOCK_ERR_OUT_OF_MEMORY, str(ei.value)
    own.release_batch(bid)
    b = synth.ligand_batch(3, np.array([12, 30]), np.array([2, 4]))
    kn = C.knobs(n_poses=16, repetitions=2, seed=4)
    sb = own.upload_ligands(b)
    res, xyz = own.run(sb, [pid], kn, b.n, _natoms(b))
    own.close()
    fp = dk.init_pocket(pk)
    fb = dk.upload_ligands(b)
    res2, xyz2 = dk.run(fb, [fp], kn, b.n, _natoms(b))
    dk.release_batch(fb)
    assert np.array_equal(res.view(np.int32), res2.view(np.int32)) and np.array_equal(xyz, xyz2)
