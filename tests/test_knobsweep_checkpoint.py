"""Checkpoint/resume of the knob sweep's result shards (host logic)."""
import os
import shutil

import numpy as np

from paper_1901_06363_gb300.knobsweep import Checkpoint

HERE = os.path.dirname(os.path.abspath(__file__))


def test_finished_shards_are_not_recomputed():
    d = os.path.join(HERE, f".ckpt_{os.getpid()}")
    try:
        calls = []

        def compute(v):
            calls.append(v)
            return dict(seconds=np.float64(v), scores=np.arange(3) * v)

        ck = Checkpoint(d)
        a = ck.get("sweep_5_10_1", lambda: compute(2.0))
        b = ck.get("sweep_5_10_4", lambda: compute(3.0))
        assert calls == [2.0, 3.0]
        # a restarted run (new object, same directory) loads both and computes only the new shard
        ck2 = Checkpoint(d)
        a2 = ck2.get("sweep_5_10_1", lambda: compute(99.0))
        b2 = ck2.get("sweep_5_10_4", lambda: compute(99.0))
        c2 = ck2.get("sweep_5_10_16", lambda: compute(4.0))
        assert calls == [2.0, 3.0, 4.0]
        assert float(a2["seconds"]) == 2.0 and np.array_equal(b2["scores"], b["scores"])
        assert np.array_equal(a2["scores"], a["scores"]) and float(c2["seconds"]) == 4.0
        # a shard left half-written by a stopped run is ignored
        open(os.path.join(d, "sweep_x.part.npz"), "wb").write(b"garbage")
        ck3 = Checkpoint(d)
        ck3.get("sweep_x", lambda: compute(5.0))
        assert calls[-1] == 5.0
        # no directory: always computed
        Checkpoint(None).get("k", lambda: compute(6.0))
        assert calls[-1] == 6.0
    finally:
        shutil.rmtree(d, ignore_errors=True)
