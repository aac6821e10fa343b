"""GB300 (sm_103a) forced D3Q19 MRT lattice Boltzmann with singular point
forces (Nash, Adhikari & Cates).

  build      -- compile the CUDA library in-tree (nvcc, sm_103a)
  lb         -- ctypes binding of include/lb.h (same names) + ``Lattice``
  workloads  -- seeded synthetic inputs of the benchmark configurations

Importing the package loads nothing; ``lb.load()`` loads the library and
raises if it has not been built.
"""
from . import build, workloads  # noqa: F401

__all__ = ["build", "workloads", "lb"]


def __getattr__(name):
    if name == "lb":
        import importlib
        return importlib.import_module(".lb", __name__)
    raise AttributeError(name)
