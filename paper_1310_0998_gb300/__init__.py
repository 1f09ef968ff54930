"""GB300 (sm_103a) simulator of self-propelled DPD dimers (arXiv:1310.0998).

The compute path is libdpd.so (CUDA, C ABI in include/dpd.h); this package
only marshals arguments.  Submodules load lazily so that importing the seeded
input generator (``synth``) does not load the CUDA library.
"""
import importlib

__all__ = ["Sim", "Sim3", "Ensemble", "Surrogate", "make_params", "synth"]


def __getattr__(name):
    if name in ("Sim", "Sim3", "make_params"):
        return getattr(importlib.import_module(__name__ + ".sim"), name)
    if name == "Surrogate":
        return importlib.import_module(__name__ + ".surrogate").Surrogate
    if name == "Ensemble":
        return importlib.import_module(__name__ + ".ensemble").Ensemble
    if name in ("synth", "sim", "build", "ensemble", "surrogate", "study", "tune"):
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
