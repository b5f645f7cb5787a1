"""GB300-native dual price discovery for fungible resource allocation
(arXiv 2104.00282).

The compute path is the C-ABI library ``libra.so`` (hand-written sm_103a
CUDA); :mod:`paper_2104_00282_gb300.ra` is its thin ctypes binding.  The
binding is imported lazily so that :mod:`paper_2104_00282_gb300.workloads`
(seeded synthetic inputs) can be used without a GPU.
"""
import importlib

__all__ = ["workloads", "ra"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
