"""The parity checker itself (tests/parity.py), on the CPU: the oracle's own trace, rounded to FP32
as the GPU reports it, passes; planted mistakes in that trace are caught."""
import numpy as np
import pytest

import oracle
import parity
import synth
import synth.configs as C


def _problem():
    pk = synth.pocket(8, 48, 0.5, C.ELLIPSOID)
    l, t = synth.ligand_sizes(41, 6, 0, [16, 40, 2, 6])
    b = synth.ligand_batch(41, l, t)
    kn = C.knobs(n_poses=8, hp_step=20.0, lp_step=20.0, repetitions=2, seed=4)
    return oracle.OraclePocket(pk), b, kn


def _as_gpu(r):
    """The oracle's own trace in the GPU trace's layout and precision."""
    return dict(pmax=r["pmax"], chosen_k=r["chosen_k"].copy(), cand_S=r["cand_S"].astype(np.float32),
                cand_status=r["cand_status"].copy(), pose_status=r["pose_status"].copy(),
                pose_init_S=r["pose_init_S"].astype(np.float32), pose_S=r["pose_S"].astype(np.float32),
                pose_xyz=r["pose_xyz"].astype(np.float32))


@pytest.fixture(scope="module")
def traced():
    opk, b, kn = _problem()
    own = oracle.dock(opk, b, kn, trace=True, xyz_out=True)
    g = _as_gpu(own)
    orc = parity.replay(opk, b, kn, g)
    return b, kn, g, orc


def test_oracle_trace_passes(traced):
    b, kn, g, orc = traced
    st = parity.check(b, kn, g, orc)
    assert st["candidates"] > 1000 and st["choice_differs"] == 0 and st["flips"] == 0
    assert st["max_dev_A"] < 1e-5


def _first_feasible(g, orc, want_band):
    st = g["cand_status"].reshape(-1, g["pmax"])
    amb = orc["cand_amb"].reshape(-1, g["pmax"])
    for s in range(st.shape[0]):
        for j in range(1, st.shape[1]):
            if st[s, j] == 1 and bool(amb[s, j] & 6) == want_band and g["chosen_k"][s] != j:
                return s, j
    raise AssertionError("no such candidate")


def test_planted_feasibility_flip_is_caught(traced):
    b, kn, g, orc = traced
    s, j = _first_feasible(g, orc, want_band=False)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    bad["cand_status"].reshape(-1, g["pmax"])[s, j] = 0
    with pytest.raises(AssertionError, match="feasibility differs"):
        parity.check(b, kn, bad, orc)


def test_planted_score_error_is_caught(traced):
    b, kn, g, orc = traced
    s, j = _first_feasible(g, orc, want_band=False)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    S = bad["cand_S"].reshape(-1, g["pmax"])
    S[s, j] = S[s, j] * np.float32(1.0 + 5e-4)
    with pytest.raises(AssertionError):
        parity.check(b, kn, bad, orc)


def test_planted_wrong_choice_is_caught(traced):
    b, kn, g, orc = traced
    # keep the incumbent at the last sweep of a pose where the oracle moved (no later sweep depends on it):
    # the committed slot is then not the first minimum of the reported values
    ends = np.cumsum(np.repeat(orc["nsweep"], kn["n_poses"])) - 1
    s = int([e for e in ends if g["chosen_k"][e] != 0][0])
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    bad["chosen_k"][s] = 0
    with pytest.raises(AssertionError, match="first minimum"):
        parity.check(b, kn, bad, parity.replay(oracle.OraclePocket(synth.pocket(8, 48, 0.5, C.ELLIPSOID)), b, kn,
                                                bad))


def test_planted_coordinate_error_is_caught(traced):
    b, kn, g, orc = traced
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    bad["pose_xyz"][:3] += np.float32(0.01)
    with pytest.raises(AssertionError, match="RMSD"):
        parity.check(b, kn, bad, orc)
