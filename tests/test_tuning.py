"""Host logic of the time-to-solution model (Eq. 4), the overlap degradation (Eq. 5) and knob selection."""
import numpy as np
import pytest

from paper_1901_06363_gb300 import tuning


def test_features_are_the_paper_predictors():
    x = tuning.features(300, 32.5, 6.0)
    assert np.allclose(x, [300, 32.5, 6, 300 * 32.5, 300 * 6, 32.5 * 6, 300 * 32.5 * 6])


def test_fit_recovers_known_coefficients():
    rng = np.random.default_rng(0)
    alpha = np.array([1e-9, 2e-7, 3e-7, 4e-10, 5e-10, 6e-9, 7e-12])
    beta = 1.5e-6
    X = np.array([tuning.features(p, a, r) for p, a, r in
                  zip(rng.uniform(200, 2000, 40), rng.uniform(16, 64, 40), rng.uniform(1, 12, 40))])
    y = X @ alpha + beta
    m = tuning.fit(X, y)
    assert np.allclose(m.alpha, alpha, rtol=1e-6, atol=1e-15)
    assert m.beta == pytest.approx(beta, rel=1e-6)
    assert m.r2 == pytest.approx(1.0) and m.adj_r2 == pytest.approx(1.0)
    assert m.predict(X[3], 1000) == pytest.approx(1000 * y[3], rel=1e-9)


def test_adjusted_r2_textbook():
    # one predictor, y = x + noise: R^2 and adjusted R^2 by their definitions
    x = np.arange(10.0)
    e = np.array([0.5, -0.3, 0.2, -0.4, 0.1, 0.3, -0.2, 0.4, -0.5, 0.0])
    y = 2 * x + 1 + e
    m = tuning.fit(x[:, None], y)
    slope, icpt = np.polyfit(x, y, 1)
    res = y - (slope * x + icpt)
    r2 = 1 - (res ** 2).sum() / ((y - y.mean()) ** 2).sum()
    assert m.r2 == pytest.approx(r2, rel=1e-12)
    assert m.adj_r2 == pytest.approx(1 - (1 - r2) * 9 / 8, rel=1e-12)


def test_fit_models_groups_by_configuration():
    rows = []
    for cfg, s in (("fast", 1e-6), ("slow", 8e-6)):
        for p in (300, 600, 900):
            for a in (20, 40):
                for r in (2, 8):
                    t = s * (1 + a / 40 + r / 8) + 1e-12 * p * a * r
                    rows.append(dict(config=cfg, npts=p, mean_atoms=a, mean_rot=r, nu=1000, seconds=1000 * t))
    ms = tuning.fit_models(rows)
    assert set(ms) == {"fast", "slow"}
    for r in rows:
        x = tuning.features(r["npts"], r["mean_atoms"], r["mean_rot"])
        assert ms[r["config"]].predict(x, r["nu"]) == pytest.approx(r["seconds"], rel=1e-6)


def test_eq5_degradation_on_hand_values():
    orig = np.arange(1, 201, dtype=float)          # top 1% of 200 = 2 ligands: 200, 199 -> 199.5
    approx = orig * 0.9                            # -> 179.55
    assert tuning.top_mean(orig) == 199.5
    assert tuning.degradation(approx, orig) == pytest.approx(10.0)
    assert tuning.degradation(orig, orig) == 0.0
    assert tuning.top_mean([3.0, 1.0]) == 3.0       # at least one ligand


def test_select_under_budget():
    class M:
        def __init__(self, t):
            self.t = t

        def predict(self, x, nu):
            return self.t * nu

    models = {"A": M(1.0), "B": M(2.0), "C": M(4.0)}
    degr = {"A": 20.0, "B": 5.0, "C": 0.0}
    c = tuning.select(models, degr, None, 10, 25.0)
    assert c.config == "B" and c.completion == 1.0
    c = tuning.select(models, degr, None, 10, 100.0)
    assert c.config == "C"
    c = tuning.select(models, degr, None, 10, 5.0)
    assert c.config == "A" and c.completion == pytest.approx(0.5)


def test_select_ignores_models_outside_their_range():
    class M:
        def __init__(self, t):
            self.t = t

        def predict(self, x, nu):
            return self.t * nu

    c = tuning.select({"A": M(-1.0), "B": M(2.0)}, {"A": 0.0, "B": 5.0}, None, 10, 100.0)
    assert c.config == "B"
