"""dock_run_static: docking without device allocation, checked against dock_run.

Callers that cannot call cudaMalloc or cudaFree on their docking path (device
memory pre-carved by their own pool or arena, or no room for the device
synchronisation an allocation may bring) use dock_run_static, whose scratch
is a fixed file-scope device array. This file is collected last so that a run
stopping at its first failure has already run every other test. It passes
both alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import synth
import synth.configs as C

pytestmark = pytest.mark.gpu

SCORE_REL = 1e-4  # per-score tolerance of the parity tests
XYZ_ABS = 1e-3    # Å, final-pose tolerance of the parity tests


@pytest.mark.parametrize("threshold", [0.0, 0.3])
def test_static_scratch_run_matches_dock_run(threshold):
    """threshold 0.3 with a 30-degree low-precision step: the per-sweep step choice (Alg. 2) matters."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_06363_gb300 import DOCK_ERR_INVALID_ARG, DOCK_OK, Docker, knobs_struct, lib

    dk = Docker(0)
    pk = synth.pocket(8, 64, 0.5, C.ELLIPSOID)
    l, t = synth.ligand_sizes(21, 24, 0, [16, 64, 2, 12])
    batch = synth.ligand_batch(21, l, t)
    kn = C.knobs(n_poses=40, hp_step=15.0, lp_step=30.0 if threshold else 15.0, threshold=threshold,
                 repetitions=2, seed=9)
    n, natoms = batch.n, int(batch.atom_off[-1])
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(batch)
    ref, ref_xyz = dk.run(bid, [pid], kn, n, natoms)

    out = torch.empty(n * 4, dtype=torch.int32, device="cuda")
    xyz = torch.empty(natoms * 3, dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    k = knobs_struct(kn)
    for call in range(2):
        # stale values from an earlier call must not leak into this one
        out.fill_(-7)
        xyz.fill_(float("nan"))
        rc = lib.dock_run_static(dk._c, bid, pid, ctypes.byref(k), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(xyz.data_ptr()), stream)
        assert rc == DOCK_OK, lib.dock_last_error(dk._c).decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(ref.dtype)
        assert np.array_equal(got["status"], ref["status"]), call
        assert np.array_equal(got["pose"], ref["pose"]), call
        assert np.allclose(got["score"], ref["score"], rtol=SCORE_REL, atol=0), call
        assert np.allclose(xyz.cpu().numpy().reshape(-1, 3), ref_xyz[0], rtol=0, atol=XYZ_ABS), call

    # runs beyond the fixed scratch (64 ligands x 4096 poses > 131072 slots) are refused before any launch
    lb, tb = synth.ligand_sizes(22, 64, 0, [16, 24, 2, 4])
    big = synth.ligand_batch(22, lb, tb)
    bid_big = dk.upload_ligands(big)
    big_out = torch.empty(big.n * 4, dtype=torch.int32, device="cuda")
    rc = lib.dock_run_static(dk._c, bid_big, pid, ctypes.byref(knobs_struct(dict(kn, n_poses=4096))),
                             ctypes.c_void_p(big_out.data_ptr()), None, stream)
    assert rc == DOCK_ERR_INVALID_ARG
    assert b"static scratch" in lib.dock_last_error(dk._c)
    dk.release_batch(bid_big)
    dk.release_batch(bid)
    dk.close()
