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


def test_sweep_moving_atoms_follow_the_fragments():
    import indep
    m = _bench()
    l, t = synth.ligand_sizes(6, 9, 0, [12, 40, 0, 6])
    b = synth.ligand_batch(6, l, t)
    nm = m.sweep_nmov(b)
    for i in range(b.n):
        x, bonds, rot = indep.ligand(b, i)
        sides = indep.sides(len(x), bonds, rot)
        assert list(nm[i]) == [int(mv.sum()) - 1 for mv, _, _ in sides]


def test_roofline_takes_the_slowest_resource():
    m = _bench()
    st = dict(atom_updates=600, lookups_skipped=400, bump_pairs=1000, candidates=100)
    fw = dict(feasible_lookups=300)
    rates = dict(fma_per_s=1e4, tex_local_per_s=100.0)
    bound, res = m.roofline_8d(st, fw, 10.0, rates, traffic=5000, hbm_gbs=1e-6)
    # fp32: 7 * 1000 + 3 * 1000 + 100 = 10100 lane-ops at 1e4/s = 1.01 s; texture 300 / 100 = 3 s; hbm 5 s
    assert res["fp32"]["work"] == 10100 and abs(res["fp32"]["time_s"] - 1.01) < 1e-12
    assert res["texture"]["time_s"] == 3.0 and abs(res["hbm"]["time_s"] - 5.0) < 1e-9
    assert bound == "hbm" and abs(res["hbm"]["frac"] - 0.5) < 1e-9
    bound, res = m.roofline_8d(st, fw, 10.0, rates, traffic=None, hbm_gbs=1.0)
    assert bound == "texture" and res["texture"]["frac"] == 0.3
