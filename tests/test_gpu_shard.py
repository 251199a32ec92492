"""Ligand sharding through the CUDA path: two gloo ranks each dock their LPT shard with dock_run (both on
cuda:0, whose launches do not wait on one another), and the results gathered to rank 0 equal one unsharded
dock_run bit for bit."""
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_rank_cuda_sharded_equals_unsharded():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mp = pytest.importorskip("torch.multiprocessing")
    import shard_worker
    q = mp.get_context("spawn").SimpleQueue()
    mp.spawn(shard_worker.gpu_worker, args=(2, _free_port(), q), nprocs=2, join=True)
    sharded, whole, idx0, share0 = q.get()
    assert np.array_equal(sharded.view(np.int32), whole.view(np.int32))
    assert 0 < len(idx0) < 300
    assert abs(share0 - 0.5) < 0.05  # the LPT split balances the modelled work
