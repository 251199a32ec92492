"""The knob-sweep and multi-pocket workloads on the GPU: full-size (or large-sample) runs checked by
properties, and sampled ligands replayed against the FP64 oracle."""
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


def _replay_sample(dk, pk, pid, batch, kn, sample, grouped_res):
    """Trace the sampled ligands alone (same ids), replay them in the oracle, and compare with the batch run."""
    sub = batch.subset(sample)
    bid = dk.upload_ligands(sub, ids=sample + batch.id_base)
    g = dk.run_trace(bid, pid, kn, sub)
    orc = parity.replay(oracle.OraclePocket(pk), sub, kn, g, ids=sample + batch.id_base)
    stats = parity.check(sub, kn, g, orc)
    parity.check_best(sub, kn, g["result"], g["pose_S"], g["pose_status"])
    assert np.array_equal(g["result"].view(np.int32), grouped_res.view(np.int32))
    dk.release_batch(bid)
    return stats


def test_multi_pocket_grouped_launch(dk):
    """16 pockets (48^3-128^3) x 50,000 lognormal ligands in one grouped launch; 32 poses, 15 degrees, 2 reps."""
    pks, b, kn = C.multi_pocket()
    pids = [dk.init_pocket(pk) for pk in pks]
    bid = dk.upload_ligands(b)
    natoms = int(b.atom_off[-1])
    res, _ = dk.run(bid, pids, kn, b.n, natoms, xyz=False)
    res = res.reshape(len(pks), b.n)
    ok = res["status"] == 0
    assert np.all(res["score"][ok] > 0) and np.all(res["score"][~ok] == 0)
    assert np.all((res["pose"][ok] >= 0) & (res["pose"][ok] < kn["n_poses"])) and np.all(res["pose"][~ok] == -1)
    assert ok.mean() > 0.9
    dk.release_batch(bid)
    # 16 sampled ligands of every pocket (256 pairs) replayed against the oracle; the grouped launch equals the
    # single-pocket one
    rng = np.random.default_rng(5)
    for i, (pk, pid) in enumerate(zip(pks, pids)):
        sample = np.sort(rng.choice(b.n, 16, replace=False))
        _replay_sample(dk, pk, pid, b, kn, sample, res[i][sample])


def test_knob_sweep_combinations(dk):
    """The 45 (step, poses, repetitions) combinations on the 100,000 lognormal ligands; 6 sampled ligands of
    every combination (270) replayed against the oracle."""
    pks, b, combos = C.knob_sweep()
    pid = dk.init_pocket(pks[0])
    bid = dk.upload_ligands(b)
    natoms = int(b.atom_off[-1])
    best = {}
    for kn in combos:
        res, _ = dk.run(bid, [pid], kn, b.n, natoms, xyz=False)
        ok = res["status"] == 0
        assert ok.mean() > 0.9 and np.all(res["score"][ok] > 0)
        best[(kn["hp_step"], kn["n_poses"], kn["repetitions"])] = res
    # more poses or more repetitions never make a ligand's result worse on average
    for s in C.SWEEP_STEPS:
        m = [np.mean(best[(s, p, 4)]["score"]) for p in C.SWEEP_POSES]
        assert m[0] <= m[1] <= m[2]
        m = [np.mean(best[(s, 32, r)]["score"]) for r in C.SWEEP_REPS]
        assert m[0] <= m[1] * (1 + 1e-6) and m[1] <= m[2] * (1 + 1e-6)
    rng = np.random.default_rng(3)
    for kn in combos:
        sample = np.sort(rng.choice(b.n, 6, replace=False))
        key = (kn["hp_step"], kn["n_poses"], kn["repetitions"])
        _replay_sample(dk, pks[0], pid, b, kn, sample, best[key][sample])
    dk.release_batch(bid)


@pytest.mark.parametrize("point", [(2.0, 45.0, 0.3, 2, 1), (5.0, 90.0, 0.8, 1, 1), (1.0, 45.0, 0.6, 3, 1),
                                   (3.0, 90.0, 0.3, 2, 0)])
def test_full_design_space_points(dk, point):
    """Points of the paper's full design space (Sec. 5.2: high-precision step, low-precision step, threshold,
    repetitions, tile peeling) with a threshold > 0, on 16 of the exploration's lognormal ligands and 8 poses:
    the launch of 2,000 ligands equals the sampled ligands traced alone, which replay against the oracle."""
    hp, lp, thr, reps, peel = point
    pks, _, _ = C.knob_sweep(n=1)
    b = C.sweep_batch(2000)
    kn = C.knobs(hp_step=hp, lp_step=lp, threshold=thr, repetitions=reps, enable_refinement=peel, n_poses=8, seed=3)
    pid = dk.init_pocket(pks[0])
    bid = dk.upload_ligands(b)
    res, _ = dk.run(bid, [pid], kn, b.n, int(b.atom_off[-1]), xyz=False)
    assert (res["status"] == 0).mean() > 0.9
    sample = np.sort(np.random.default_rng(int(hp * 100 + thr * 10)).choice(b.n, 16, replace=False))
    st = _replay_sample(dk, pks[0], pid, b, kn, sample, res[sample])
    assert st["candidates"] > 1000
    dk.release_batch(bid)
