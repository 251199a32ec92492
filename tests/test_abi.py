"""The C-ABI library loads without a GPU and exports every symbol the header declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "geodock.h")


def _declared():
    src = open(HEADER).read()
    return re.findall(r"^\s*(?:int|void|const char\*)\s+(dock_\w+)\s*\(", src, re.M)


@pytest.fixture(scope="module")
def lib():
    from paper_1901_06363_gb300 import build
    build.build()
    return ctypes.CDLL(build.OUT)


def test_header_declares_the_boundary():
    names = set(_declared())
    for n in ("dock_create", "dock_destroy", "dock_init_pocket", "dock_upload_ligands", "dock_run",
              "dock_last_error", "dock_run_trace", "dock_autotune"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls_without_gpu(lib):
    import paper_1901_06363_gb300 as g
    from paper_1901_06363_gb300.binding import knobs_struct
    import oracle
    import synth.configs as C
    # the trace layout agrees with the oracle's, for flat sweeps and for tile peeling
    for kn in (C.knobs(hp_step=10.0), C.knobs(hp_step=5.0, lp_step=45.0),
               C.knobs(hp_step=1.0, enable_refinement=1), C.knobs(hp_step=7.0, lp_step=2.0)):
        assert g.lib.dock_trace_pmax(ctypes.byref(knobs_struct(kn))) == oracle.pmax_of(kn)
    # no context: calls fail with an error code instead of crashing
    assert g.lib.dock_run(None, 0, None, 0, None, None, None, 0, None) == g.DOCK_ERR_INVALID_ARG
    assert g.lib.dock_last_error(None) == b"no context"


def test_refinement_calls_fail_cleanly_without_context(lib):
    import paper_1901_06363_gb300 as g
    assert g.lib.dock_batch_info(None, 0, None, None, None, None) == g.DOCK_ERR_INVALID_ARG
    assert g.lib.dock_score_trilinear(None, 0, 0, 1, None, None, None) == g.DOCK_ERR_INVALID_ARG
    assert g.lib.dock_dof_apply(None, 0, None, None, 6, None, None) == g.DOCK_ERR_INVALID_ARG
    assert g.lib.dock_dof_grad(None, 0, None, None, 6, None, None, None) == g.DOCK_ERR_INVALID_ARG
    assert g.lib.dock_refine(None, 0, None, 0, None, None, None, None, 0, None) == g.DOCK_ERR_INVALID_ARG
    assert g.lib.dock_refine_trace(None, 0, 0, None, None, None, None, None) == g.DOCK_ERR_INVALID_ARG


def test_database_and_rate_calls_fail_cleanly_without_context(lib):
    import paper_1901_06363_gb300 as g
    assert g.lib.dock_run_database(None, None, None, 0, None, 1, None, None, None) == g.DOCK_ERR_INVALID_ARG
    assert g.lib.dock_measure_peaks(None, 0, None, None) == g.DOCK_ERR_INVALID_ARG


def test_batch_ids_must_match_the_ligand_count(lib):
    import numpy as np
    import synth
    from paper_1901_06363_gb300 import Docker
    l, t = synth.ligand_sizes(3, 4, 0, [12, 20, 1, 3])
    b = synth.ligand_batch(3, l, t)
    s, keep = Docker._batch_struct(b, ids=np.arange(4))
    assert s.n == 4 and len(keep) == 7
    with pytest.raises(ValueError):
        Docker._batch_struct(b, ids=np.arange(3))
