"""GB300 (sm_103a) FP64 implementation of the GENGA hybrid symplectic N-body step.

``paper_1404_2324_gb300.genga`` is the ctypes binding of the CUDA library (include/genga.h);
``paper_1404_2324_gb300.ics`` draws seeded synthetic initial conditions. The binding is imported
lazily so that the input generator works on machines without the CUDA library.
"""
import importlib

from . import ics  # noqa: F401


def __getattr__(name):
    if name in ("genga", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
