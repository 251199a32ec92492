"""The design spaces of the exploration (Sec. 5.2) and its Pareto front (host logic)."""
from paper_1901_06363_gb300 import knobsweep as ks


def _keys(name):
    pts, names, base = ks.space(name, poses=8)
    return [tuple(p[n] for n in names) for p in pts], names, base, pts


def test_paper_flat_space():
    keys, names, base, pts = _keys("flat")
    assert names == ("hp_step", "repetitions")
    assert len(keys) == len(set(keys)) == 8 * 3
    assert base == (1.0, 3) and base in keys
    assert sorted({k[0] for k in keys}) == [1.0, 2.0, 3.0, 5.0, 10.0, 15.0, 45.0, 60.0]
    assert all(p["threshold"] == 0 and p["enable_refinement"] == 0 and p["lp_step"] == p["hp_step"] for p in pts)
    assert all(p["n_poses"] == 8 for p in pts)


def test_paper_full_space():
    keys, names, base, pts = _keys("full")
    assert len(keys) == len(set(keys)) == 4 * 2 * 4 * 3 * 2 == 192
    assert base == (1.0, 45.0, 0.0, 3, 0) and base in keys
    assert sorted({k[2] for k in keys}) == [0.0, 0.3, 0.6, 0.8]
    assert sorted({k[1] for k in keys}) == [45.0, 90.0]
    assert {k[4] for k in keys} == {0, 1}


def test_grid_space():
    keys, names, base, _ = _keys("grid")
    assert len(keys) == 45 and base == (5.0, 128, 16) and base in keys


def test_pareto_front():
    rows = [dict(seconds=s, degradation_pct=d, id=i) for i, (s, d) in
            enumerate([(1.0, 0.0), (0.5, 3.0), (0.4, 3.0), (0.6, 1.0), (0.3, 10.0), (0.7, 2.0), (0.2, 10.0)])]
    front = [r["id"] for r in ks.pareto(rows)]
    # fastest first; each later point strictly less degraded; dominated points (0.5, 3), (0.7, 2), (0.3, 10) out
    assert front == [6, 2, 3, 0]


def test_summary_picks_the_peeling_only_point():
    names = ["hp_step", "lp_step", "threshold", "repetitions", "enable_refinement"]
    table = []
    for e in (0, 1):
        for r in (1, 3):
            table.append(dict(hp_step=1.0, lp_step=45.0, threshold=0.0, repetitions=r, enable_refinement=e,
                              seconds=1.0 / (1 + 6 * e) / (4 - r), speedup=(1 + 6 * e) * (4 - r) / 1.0,
                              degradation_pct=2.0 * e + (3 - r)))
    res = dict(space="full", knobs=names, baseline=[1.0, 45.0, 0.0, 3, 0], table=table, pareto=[], selection=[])
    s = ks.summary(res)
    assert s["peeling_only"] == dict(speedup=7.0, degradation_pct=2.0)
