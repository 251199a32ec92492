"""dock_run_static: docking without device allocation, checked against dock_run.

Callers that cannot call cudaMalloc or cudaFree on their docking path (device
memory pre-carved by their own pool or arena, or no room for the device
synchronisation an allocation may bring) use dock_run_static, whose scratch
is a fixed file-scope device array. This file is collected last so that a run
stopping at its first failure has already run every other test. It passes
both alone in a fresh process and after the other tests.
"""
import ctypes
import time

import numpy as np
import pytest

import synth
import synth.configs as C

pytestmark = pytest.mark.gpu


def _env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_06363_gb300 import Docker
    return torch, Docker(0)


@pytest.mark.parametrize("score_mode,threshold", [(0, 0.0), (0, 0.3), (1, 0.0), (2, 0.3)])
def test_static_scratch_run_matches_dock_run(score_mode, threshold):
    """Bit-identical to dock_run in every score mode, on two calls in a row; threshold 0.3 with a 30-degree
    low-precision step makes the per-sweep step choice (Alg. 2) matter."""
    torch, dk = _env()
    from paper_1901_06363_gb300 import DOCK_ERR_INVALID_ARG, DOCK_OK, knobs_struct, lib

    pk = synth.pocket(8, 64, 0.5, C.ELLIPSOID)
    l, t = synth.ligand_sizes(21, 24, 0, [16, 64, 2, 12])
    batch = synth.ligand_batch(21, l, t)
    kn = C.knobs(n_poses=40, hp_step=15.0, lp_step=30.0 if threshold else 15.0, threshold=threshold,
                 repetitions=2, seed=9, score_mode=score_mode)
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
        assert np.array_equal(got.view(np.int32), ref.view(np.int32)), call
        assert np.array_equal(xyz.cpu().numpy().reshape(-1, 3), ref_xyz[0]), call

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


def test_static_scratch_run_does_not_wait():
    """The call only enqueues: behind a ~0.5 s device-side sleep on its stream it returns long before the sleep
    ends, and its results, read after the stream drains, equal dock_run's."""
    torch, dk = _env()
    from paper_1901_06363_gb300 import DOCK_OK, knobs_struct, lib

    pk = synth.pocket(8, 48, 0.5, C.ELLIPSOID)
    l, t = synth.ligand_sizes(24, 8, 0, [16, 40, 2, 6])
    batch = synth.ligand_batch(24, l, t)
    kn = C.knobs(n_poses=16, hp_step=20.0, lp_step=20.0, repetitions=1, seed=2)
    n, natoms = batch.n, int(batch.atom_off[-1])
    pid = dk.init_pocket(pk)
    bid = dk.upload_ligands(batch)
    ref, _ = dk.run(bid, [pid], kn, n, natoms)
    out = torch.empty(n * 4, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    stream = ctypes.c_void_p(s.cuda_stream)
    k = knobs_struct(kn)
    assert lib.dock_run_static(dk._c, bid, pid, ctypes.byref(k), ctypes.c_void_p(out.data_ptr()), None,
                               stream) == DOCK_OK  # first call on the device: the array's address is looked up
    torch.cuda.synchronize()
    out.fill_(-7)
    done = torch.cuda.Event()
    torch.cuda._sleep(1_000_000_000)  # about 0.5 s of clock cycles on this stream
    t0 = time.perf_counter()
    rc = lib.dock_run_static(dk._c, bid, pid, ctypes.byref(k), ctypes.c_void_p(out.data_ptr()), None, stream)
    dt = time.perf_counter() - t0
    done.record(s)
    still_running = not done.query()
    torch.cuda.synchronize()
    assert rc == DOCK_OK, lib.dock_last_error(dk._c).decode()
    assert dt < 0.05 and still_running, (dt, still_running)
    assert np.array_equal(out.cpu().numpy(), ref.view(np.int32).ravel())
    dk.release_batch(bid)
    dk.close()
