"""dock_measure_peaks: the measured rates behind the sweep's rooflines are positive and of the device's order."""
import pytest

import synth
import synth.configs as C

pytestmark = pytest.mark.gpu


def test_measured_rates_are_plausible():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_06363_gb300 import Docker
    dk = Docker(0)
    pid = dk.init_pocket(synth.pocket(8, 64, 0.5, C.ELLIPSOID))
    r = dk.measure_peaks(pid)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # 128 FP32 lanes per SM at 1-2.5 GHz
    assert sms * 128 * 1.0e9 < r["fma_per_s"] < sms * 128 * 2.5e9
    assert r["ffma2_per_s"] > 0.9 * r["fma_per_s"]
    assert r["tex_field_per_s"] > 0 and r["tex_local_per_s"] > 0.5 * r["tex_field_per_s"]
    assert r["l2_sectors_per_s"] > 0
    dk.close()
