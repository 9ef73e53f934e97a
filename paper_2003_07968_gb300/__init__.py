"""GB300 (sm_103a) D2Q9 pseudopotential lattice Boltzmann step with the
nearest-neighbour force approach of arXiv 2003.07968.

The compute path is the CUDA library built from ``csrc/`` (see
:mod:`.build`) behind the C ABI of ``include/pplbm.h``; :mod:`.capi` is its
thin Python binding.  There is no CPU fallback: importing the binding
without the built library raises.
"""
from . import capi  # noqa: F401
from .capi import *  # noqa: F401,F403
