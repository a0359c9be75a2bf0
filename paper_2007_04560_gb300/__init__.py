"""GB300 (sm_103a) Newton–Krylov–Schwarz time step of the energy-stable DVD scheme
for the coupled Allen–Cahn / Cahn–Hilliard system (arXiv 2007.04560).

The compute path is libacac.so (CUDA, C ABI in include/acac.h); acac.py is its
thin ctypes binding and build.py compiles it.
"""
from .acac import (AcacError, Solver, acac_params, acac_step_info, load,  # noqa: F401
                   to_c_params)
