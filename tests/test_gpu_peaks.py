"""The library's own unit-rate probe (rbf_peak_probe), the denominator of the
benchmark's roofline fractions: each rate must be positive and below what the
device's unit counts allow at its highest clock (a rate above that would mean
the probe does not execute the work it counts)."""
import pytest

pytestmark = pytest.mark.gpu


def test_peak_probe_rates_are_physical():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_07652_gb300 import _lib
    _lib.load()
    props = torch.cuda.get_device_properties(0)
    n_sm = props.multi_processor_count
    clock_ghz = 2.2   # above every GB300 SM clock
    ffma = _lib.peak_probe(_lib.PROBE_FFMA, 0.2)
    dfma = _lib.peak_probe(_lib.PROBE_DFMA, 0.2)
    ex2 = _lib.peak_probe(_lib.PROBE_EX2, 0.2)
    rsq = _lib.peak_probe(_lib.PROBE_RSQRT, 0.2)
    print(f"FFMA {ffma / 1e12:.1f} TF/s  DFMA {dfma / 1e12:.2f} TF/s  "
          f"ex2 {ex2 / 1e12:.2f} T/s  rsqrt {rsq / 1e12:.2f} T/s")
    assert 0.3 * n_sm * 128 * 2 * clock_ghz * 1e9 < ffma <= n_sm * 128 * 2 * clock_ghz * 1e9
    assert 0 < dfma <= ffma
    for r in (ex2, rsq):
        assert 0 < r <= n_sm * 32 * clock_ghz * 1e9
