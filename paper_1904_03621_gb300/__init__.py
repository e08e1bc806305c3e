"""GB300-native exhaustive low-spectrum search for Ising spin glasses.

Imports are lazy: ``instances`` (seeded generators) can be used without
loading the CUDA library; ``low_spectrum`` and friends load ``libbf.so`` on
first use and raise if it is missing.
"""
import importlib

__all__ = ["instances", "low_spectrum", "low_spectrum_batched", "low_spectrum_backward", "low_spectrum_qubo",
           "low_spectrum_potts", "LowSpectrumFn", "autotune", "fit_spectrum", "search", "Solution", "lib"]

_API = ("low_spectrum", "low_spectrum_batched", "low_spectrum_backward", "low_spectrum_qubo", "low_spectrum_potts",
        "LowSpectrumFn", "autotune")


def __getattr__(name):
    if name == "instances":
        return importlib.import_module(__name__ + ".instances")
    if name == "lib":
        return importlib.import_module(__name__ + "._lib")
    if name == "fit_spectrum":
        return getattr(importlib.import_module(__name__ + ".fit"), name)
    if name in ("search", "Solution", "graph_to_dense"):
        return getattr(importlib.import_module(__name__ + ".graph"), name)
    if name in _API:
        return getattr(importlib.import_module(__name__ + ".api"), name)
    raise AttributeError(name)
