"""Energy accounting against a fake NVML (no GPU, no driver)."""
import ctypes

import pytest

from paper_2302_05662_gb300 import energy


class FakeNvml:
    """Counter that advances 500 mJ per read; records the calls made."""

    def __init__(self, fail=None):
        self.calls, self.mj, self.fail = [], 1000, fail

    def __getattr__(self, name):
        def f(*args):
            self.calls.append(name)
            if name == self.fail:
                return 999
            if name == "nvmlDeviceGetTotalEnergyConsumption":
                self.mj += 500
                ctypes.cast(args[1], ctypes.POINTER(ctypes.c_ulonglong))[0] = self.mj
            return 0
        return f


def test_energy_per_call_from_counter_difference():
    lib = FakeNvml()
    nv = energy.Nvml(3, lib=lib)
    ran = []
    out = energy.measure(nv, lambda: ran.append(1), lambda: None, flops_per_call=2e9, min_seconds=0.0)
    nv.close()
    assert out["calls"] == len(ran) == 64
    assert out["joules_per_call"] == pytest.approx(0.5 / 64)      # two reads, 500 mJ apart
    assert out["gflop_per_joule"] == pytest.approx(2.0 * 64 / 0.5, rel=1e-3)
    # only initialisation, handle lookup, counter reads and shutdown: no setter
    assert set(lib.calls) == {"nvmlInit_v2", "nvmlDeviceGetHandleByIndex_v2",
                              "nvmlDeviceGetTotalEnergyConsumption", "nvmlShutdown"}


def test_nvml_errors_raise():
    with pytest.raises(energy.NvmlError):
        energy.Nvml(0, lib=FakeNvml(fail="nvmlDeviceGetHandleByIndex_v2"))
