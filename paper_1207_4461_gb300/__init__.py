"""GB300 (sm_103a) implementation of the hot path of quadrature by expansion
(QBX) for 2D Helmholtz layer potentials: S, D and grad S with complex
wavenumber, in complex FP64 (Kloeckner, Barnett, Greengard, O'Neil,
arXiv:1207.4461).

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/qbx.h``); ``qbx`` is its thin Python binding.
"""
from .qbx import *  # noqa: F401,F403
from .qbx import Plan, Geometry, QBXError, lib, library_path  # noqa: F401
