"""tm: GB300-native evaluation of the temporal execution model and the task
reordering heuristic of Lazaro-Munoz et al. (arXiv 1806.10113).

The compute path is the C-ABI library ``libtm.so`` (hand-written CUDA for
sm_103a, declared in ``include/tm.h``).  ``paper_1806_10113_gb300.tm`` is its
thin ctypes binding; ``paper_1806_10113_gb300.inputs`` draws seeded synthetic
task groups.  Importing the package does not load the library; the binding
loads it on first use and raises if it is missing.
"""
import importlib

__all__ = ["inputs", "tm"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
