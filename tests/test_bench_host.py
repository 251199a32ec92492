"""Host helpers of bench.py: the repeated database of the end-to-end figure and the key of the ncu traffic
figure (kernel code without comments)."""
import importlib.util
import os

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_repeat_batch_concatenates_copies_with_continuing_ids():
    m = _bench()
    l, t = synth.ligand_sizes(5, 7, 0, [16, 30, 1, 5])
    b = synth.ligand_batch(5, l, t)
    r = m.repeat_batch(b, 3)
    assert r.n == 3 * b.n and r.id_base == b.id_base  # ligand k of copy c has id id_base + c * n + k
    for c in range(3):
        sub = r.subset(np.arange(c * b.n, (c + 1) * b.n))
        for name in ("atom_off", "bond_off", "rot_off", "xyz", "bonds", "rot"):
            assert np.array_equal(getattr(sub, name), getattr(b, name)), (c, name)
    assert m.input_bytes(r) == sum(getattr(r, a).nbytes for a in ("atom_off", "xyz", "bond_off", "bonds",
                                                                  "rot_off", "rot"))


def test_traffic_key_ignores_comments_only():
    m = _bench()
    text = open(os.path.join(ROOT, "paper_1901_06363_gb300", "csrc", "geodock_kernels.cuh")).read()
    base = m.kernel_code_sha()
    assert m.kernel_code_sha(text) == base
    assert m.kernel_code_sha("// a new comment\n" + text.replace("// ", "//  ", 3) + "\n/* x */\n\n") == base
    assert m.kernel_code_sha(text.replace("constexpr int IDX_FLOATS = 68;", "constexpr int IDX_FLOATS = 72;")) != base
