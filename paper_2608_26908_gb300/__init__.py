"""GB300-native Grand-Potential phase-field / lattice-Boltzmann coupled step.

The compute path is the CUDA library ``libgpflbm.so`` (sm_103a) behind the
C-ABI declared in ``include/gpflbm.h``; ``gpflbm.py`` is its thin ctypes
binding.  ``inputs.py`` builds seeded synthetic scenarios.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs"]
