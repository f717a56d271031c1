"""Energy of repeated products from the GPU's cumulative energy counter.

Section 6.3 of the paper tunes for energy and power as well as latency,
reading NVML; here the counter is read (never any setting changed) around a
long loop of products, giving joules per product, average watts and
GFLOP/J.  The GPU is one of several in a shared machine, so the figures are
reported, not used to select.

NVML is reached through ctypes on the driver's libnvidia-ml.so.1; every call
goes through ``Nvml`` so tests can substitute a fake library object.
"""
from __future__ import annotations

import ctypes
import time


class NvmlError(RuntimeError):
    pass


class Nvml:
    """The cumulative energy counter (millijoules) of one GPU by NVML index."""

    def __init__(self, index: int, lib=None):
        self.lib = lib if lib is not None else ctypes.CDLL("libnvidia-ml.so.1")
        self._call("nvmlInit_v2")
        self.handle = ctypes.c_void_p()
        self._call("nvmlDeviceGetHandleByIndex_v2", ctypes.c_uint(index), ctypes.byref(self.handle))

    def _call(self, name, *args):
        rc = getattr(self.lib, name)(*args)
        if rc != 0:
            raise NvmlError(f"{name} returned {rc}")

    def energy_mj(self) -> int:
        v = ctypes.c_ulonglong()
        self._call("nvmlDeviceGetTotalEnergyConsumption", self.handle, ctypes.byref(v))
        return int(v.value)

    def close(self):
        self._call("nvmlShutdown")


def measure(nvml: Nvml, run, sync, flops_per_call: float, min_seconds: float = 1.0, max_calls: int = 1 << 20):
    """Call run() repeatedly for at least min_seconds (between two sync()s)
    and read the energy counter around the loop.  Returns joules per call,
    mean watts and GFLOP per joule."""
    calls = 0
    sync()
    e0 = nvml.energy_mj()
    t0 = time.perf_counter()
    while True:
        for _ in range(64):
            run()
        calls += 64
        sync()
        dt = time.perf_counter() - t0
        if dt >= min_seconds or calls >= max_calls:
            break
    e1 = nvml.energy_mj()
    joules = (e1 - e0) / 1e3
    if joules <= 0 or calls == 0:
        return None
    return {"calls": calls, "seconds": round(dt, 3), "joules_per_call": joules / calls,
            "watts": round(joules / dt, 1), "gflop_per_joule": round(flops_per_call * calls / joules / 1e9, 3)}
