"""B300-native preconditioned Jacobian-free Newton-Krylov solver for steady
nonlinear free-surface flow past a submerged source (Pethiyagoda, McCue,
Moroney & Back, arXiv 1403.5044).

The compute path is the CUDA library ``libswj.so`` (C ABI declared in
``include/swj.h``); ``swj`` is its thin ctypes binding.  ``workloads`` holds
the seeded synthetic inputs.  Submodules load on first use so that importing
the input generators never loads the CUDA library.
"""
import importlib

__all__ = ["swj", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
