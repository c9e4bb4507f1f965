"""GB300 (sm_103a) ADI isogeometric Maxwell time stepper.

The hot path (right-hand-side contractions, banded line solves, field update)
is CUDA in ``libadi_maxwell.so`` behind the C-ABI of ``include/adi_maxwell.h``;
``adi`` is its ctypes binding and ``inputs`` the seeded input generators.
"""
from . import inputs  # noqa: F401
