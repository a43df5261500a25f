"""GB300 (sm_103a) library for the two-site DMRG effective-Hamiltonian matvec.

The compute path is ``libheff.so`` (hand-written CUDA, C ABI in include/heff.h);
``heff`` is its Python binding.  Importing this package requires the library to be
built (``build.build()``); there is no CPU fallback.
"""
from . import heff  # noqa: F401  (raises ImportError when libheff.so is missing)
from .heff import Layout, Plan, HeffError, heff_layouts  # noqa: F401

__all__ = ["heff", "Layout", "Plan", "HeffError", "heff_layouts"]
