import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: longer CPU test")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_terminal_summary(terminalreporter):
    """Counts of the replay parity checks run in this session (candidates, band members, flips, differing
    choices and why, the largest final-coordinate deviation), so that a quiet run still shows them."""
    w = terminalreporter.write_line
    ref = sys.modules.get("test_gpu_refine")
    worst = getattr(ref, "WORST", None)
    if worst:
        w(f"gradient checks: {len(worst)} comparisons, worst entry at {max(worst):.3f} of its tolerance")
    parity = sys.modules.get("parity")
    rec = getattr(parity, "RECORD", None)
    if not rec:
        return
    keys = ("candidates", "amb_score", "amb_bump", "amb_box", "flips", "interval_used", "choice_differs",
            "choice_tie", "choice_overlap", "choice_flip")
    tot = {k: sum(s[k] for _, s in rec) for k in keys}
    w(f"parity replays: {len(rec)} checks")
    for label, s in rec:
        if label:
            w(f"  {label}: " + ", ".join(f"{k} {s[k]}" for k in keys) + f", max_dev_A {s['max_dev_A']:.2e}")
    band = tot["amb_bump"] + tot["amb_box"]
    w("  total: " + ", ".join(f"{k} {tot[k]}" for k in keys) +
      f"; feasibility-band fraction {band / max(tot['candidates'], 1):.2e}"
      f"; max_dev_A {max(s['max_dev_A'] for _, s in rec):.2e}")
