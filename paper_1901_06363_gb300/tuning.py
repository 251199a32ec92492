"""Time-to-solution model and budget-driven knob selection (Sec. 3.4, Eq. 4 and Eq. 5).

Eq. 4 models the time to dock a database of nu ligands with knob
configuration k as nu times the time of the average ligand, a linear
regression with interactions over the data features

    x = (p, a, r, p a, p r, a r, p a r)

(p: probe points of the pocket, a: mean atoms per ligand, r: mean rotatable
bonds per ligand), with coefficients alpha(k) and intercept beta(k) fitted
per configuration:

    t = nu * (alpha(k) . x + beta(k)).

Eq. 5 measures the accuracy loss of a configuration as the overlap
degradation (1 - o_approx / o_original) * 100, where each o averages the
overlap scores of the best-scoring 1 % of the ligands.

Knob selection (the paper delegates it to its autotuner): among the
configurations whose predicted time fits the budget, take the one with the
lowest degradation; when none fits, take the fastest, which then docks the
fraction budget / t of the database. A configuration whose model predicts a
non-positive time (outside its training range) is left out.

Host-side arithmetic only: the times come from runs of the CUDA path.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FEATURES = ("p", "a", "r", "p*a", "p*r", "a*r", "p*a*r")


def features(npts: float, mean_atoms: float, mean_rot: float) -> np.ndarray:
    """The predictor vector of Eq. 4: the three data features and all their interactions."""
    p, a, r = float(npts), float(mean_atoms), float(mean_rot)
    return np.array([p, a, r, p * a, p * r, a * r, p * a * r])


@dataclass
class TimeModel:
    """t_la = alpha . x + beta for one knob configuration (seconds per ligand)."""
    alpha: np.ndarray
    beta: float
    r2: float
    adj_r2: float
    n: int = 0
    scale: np.ndarray = field(default_factory=lambda: np.ones(len(FEATURES)))

    def per_ligand(self, x) -> float:
        return float(np.asarray(x, np.float64) @ self.alpha + self.beta)

    def predict(self, x, nu) -> float:
        """Eq. 4: time to dock nu ligands with data features x."""
        return float(nu) * self.per_ligand(x)


def fit(X, y, ridge: float = 0.0) -> TimeModel:
    """Least-squares fit of y = X alpha + beta (rows of X are feature vectors, y seconds per ligand).

    The columns are scaled to unit maximum before solving (the interaction
    terms span orders of magnitude); ridge > 0 adds that much Tikhonov
    regularisation on the scaled coefficients (not on the intercept), for
    designs with fewer distinct feature rows than coefficients."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    m, q = X.shape
    scale = np.abs(X).max(0)
    scale[scale == 0] = 1.0
    A = np.hstack([X / scale, np.ones((m, 1))])
    if ridge > 0:
        R = np.sqrt(ridge) * np.eye(q + 1)[:q]
        A_ = np.vstack([A, R])
        y_ = np.concatenate([y, np.zeros(q)])
    else:
        A_, y_ = A, y
    coef, *_ = np.linalg.lstsq(A_, y_, rcond=None)
    alpha = coef[:q] / scale
    beta = float(coef[q])
    res = y - (X @ alpha + beta)
    ss_res = float(res @ res)
    ss_tot = float(((y - y.mean()) ** 2).sum())
    r2 = 1.0 - ss_res / ss_tot if ss_tot > 0 else 1.0
    # adjusted R^2 with q predictors and m observations
    adj = 1.0 - (1.0 - r2) * (m - 1) / (m - q - 1) if m > q + 1 else float("nan")
    return TimeModel(alpha=alpha, beta=beta, r2=r2, adj_r2=adj, n=m, scale=scale)


def fit_models(rows, ridge: float = 0.0):
    """One Eq. 4 model per configuration from measured rows.

    rows: iterable of dicts with keys config (hashable), npts, mean_atoms,
    mean_rot, nu (ligands docked) and seconds (time of that run)."""
    by = {}
    for r in rows:
        by.setdefault(r["config"], []).append(r)
    models = {}
    for k, rs in by.items():
        X = np.array([features(r["npts"], r["mean_atoms"], r["mean_rot"]) for r in rs])
        y = np.array([r["seconds"] / r["nu"] for r in rs])
        models[k] = fit(X, y, ridge)
    return models


def top_mean(scores, frac: float = 0.01) -> float:
    """Mean of the top `frac` of the scores (at least one)."""
    s = np.sort(np.asarray(scores, np.float64))[::-1]
    n = max(1, int(round(frac * len(s))))
    return float(s[:n].mean())


def degradation(scores_approx, scores_original, frac: float = 0.01) -> float:
    """Eq. 5: (1 - mean top-1% overlap of the configuration / that of the original) * 100."""
    return (1.0 - top_mean(scores_approx, frac) / top_mean(scores_original, frac)) * 100.0


@dataclass
class Choice:
    config: object
    predicted_s: float
    degradation: float
    completion: float  # fraction of the database docked within the budget


def select(models, degr, x, nu, budget_s) -> Choice:
    """The configuration of lowest degradation whose predicted time for nu ligands fits the budget;
    if none fits, the fastest one and the fraction of the database it docks in the budget."""
    # a model that predicts no time at all has left its training range: it gives no estimate
    t = {k: m.predict(x, nu) for k, m in models.items() if k in degr}
    t = {k: tk for k, tk in t.items() if tk > 0}
    fits = [k for k, tk in t.items() if tk <= budget_s]
    if fits:
        k = min(fits, key=lambda c: (degr[c], t[c]))
        return Choice(k, t[k], degr[k], 1.0)
    k = min(t, key=lambda c: (t[c], degr[c]))
    return Choice(k, t[k], degr[k], budget_s / t[k] if t[k] > 0 else 1.0)
