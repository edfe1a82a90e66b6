"""GB300-native photon-packet Monte Carlo dust radiative transfer.

The transport itself runs in hand-written CUDA kernels behind a C ABI
(``include/rt.h``); :mod:`paper_1410_1629_gb300.rt` is the thin ctypes binding
with the same function names.  :mod:`paper_1410_1629_gb300.workloads` builds
seeded synthetic inputs.
"""
__all__ = ["rt", "workloads"]


def __getattr__(name):
    if name in ("rt", "workloads", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
