"""dock_run_database: a host-memory ligand database docked chunk by chunk (host preparation of the next chunk
overlapping the device sweep) gives exactly the results, coordinates and work counts of one dock_run over the
whole database."""
import copy

import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def setup(dk):
    pks = [synth.pocket(8, 48, 0.5, C.ELLIPSOID), synth.pocket(9, 40, 0.5, (6, 5, 4))]
    pids = [dk.init_pocket(p) for p in pks]
    l, t = synth.ligand_sizes(31, 300, 0, [12, 60, 0, 8])
    b = synth.ligand_batch(31, l, t)
    kn = C.knobs(n_poses=16, hp_step=30.0, lp_step=30.0, repetitions=3, threshold=0.2, seed=5)
    return pids, b, kn


def _whole(dk, b, pids, kn, ids=None):
    bid = dk.upload_ligands(b, ids=ids)
    res, xyz = dk.run(bid, pids, kn, b.n, int(b.atom_off[-1]))
    st = dk.stats()
    dk.release_batch(bid)
    return res, xyz, st


@pytest.mark.parametrize("chunk", [64, 300, 1000, 1])
def test_database_matches_one_run(dk, setup, chunk):
    pids, b, kn = setup
    if chunk == 1:
        b = b.subset(np.arange(7))  # every ligand its own chunk
    res, xyz, st = _whole(dk, b, pids, kn)
    dres, dxyz = dk.run_database(b, pids, kn, chunk=chunk)
    dst = dk.stats()
    assert np.array_equal(dres.view(np.int32), res.view(np.int32))
    assert np.array_equal(dxyz, xyz)
    for key in ("candidates", "pair_bounds", "bump_pairs", "pose_reps_skipped"):
        assert dst[key] == st[key], key
    # lookups left out by the gate depend on which poses share a warp, which a chunk's own launch may
    # arrange differently (heavy ligands spread over more lanes); lookups made plus left out do not
    assert dst["atom_updates"] + dst["lookups_skipped"] == st["atom_updates"] + st["lookups_skipped"]
    assert dst["sweep_ms"] == -1.0


def test_database_ids_and_repeat_calls(dk, setup):
    """Explicit ids seed the poses as in dock_upload_ligands; a second call reuses the pipeline's buffers."""
    pids, b, kn = setup
    ids = np.arange(b.n, dtype=np.int64) * 7 + 1000
    res, xyz, _ = _whole(dk, b, pids[:1], kn, ids=ids)
    for _ in range(2):
        dres, dxyz = dk.run_database(b, pids[:1], kn, chunk=100, ids=ids)
        assert np.array_equal(dres.view(np.int32), res.view(np.int32))
        assert np.array_equal(dxyz, xyz)


def test_database_without_coordinates_and_empty(dk, setup):
    pids, b, kn = setup
    res, _, _ = _whole(dk, b, pids, kn)
    dres, dxyz = dk.run_database(b, pids, kn, chunk=128, xyz=False)
    assert dxyz is None and np.array_equal(dres.view(np.int32), res.view(np.int32))
    empty = b.subset(np.arange(0))
    dres, dxyz = dk.run_database(empty, pids, kn, chunk=16)
    assert len(dres) == 0 and dxyz.shape == (2, 0, 3)
    assert dk.stats()["candidates"] == 0


def test_database_errors(dk, setup):
    from paper_1901_06363_gb300.binding import DockError
    pids, b, kn = setup
    with pytest.raises(DockError, match="chunk"):
        dk.run_database(b, pids, kn, chunk=0)
    with pytest.raises(DockError, match="pocket"):
        dk.run_database(b, [99], kn, chunk=64)
    # a bond joining an atom to itself in ligand 130: reported with the chunk that holds it
    bad = copy.deepcopy(b)
    e0 = int(bad.bond_off[130])
    bad.bonds[e0, 1] = bad.bonds[e0, 0]
    with pytest.raises(DockError, match="ligands 128..191"):
        dk.run_database(bad, pids, kn, chunk=64)
    # the context stays usable
    res, xyz, _ = _whole(dk, b, pids, kn)
    dres, dxyz = dk.run_database(b, pids, kn, chunk=64)
    assert np.array_equal(dres.view(np.int32), res.view(np.int32))


@pytest.mark.parametrize("variant", ["peel", "trilinear", "noclip"])
def test_database_knob_variants(dk, setup, variant):
    """Tile peeling, the trilinear score and clipping off take the same path in chunks."""
    pids, b, kn = setup
    kn = dict(kn, **{"peel": dict(enable_refinement=1, hp_step=5.0, lp_step=30.0, n_poses=8),
                     "trilinear": dict(score_mode=1),
                     "noclip": dict(clip_box=0)}[variant])
    sub = b.subset(np.arange(90))
    res, xyz, st = _whole(dk, sub, pids, kn)
    dres, dxyz = dk.run_database(sub, pids, kn, chunk=40)
    assert np.array_equal(dres.view(np.int32), res.view(np.int32))
    assert np.array_equal(dxyz, xyz)
    assert dk.stats()["candidates"] == st["candidates"]
