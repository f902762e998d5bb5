"""GB300 (sm_103a) implementation of the primal-dual domain decomposition method for
dual total variation minimisation (Lee & Park, Algorithm 1).

The solver lives in the CUDA library ``libddtv.so`` behind the C ABI of
``include/dd_tv.h``; :mod:`._lib` is its ctypes binding and :class:`Solver` the
handle wrapper.  Build the library with ``python -m paper_1901_00682_gb300.build``.
"""
from ._lib import (L1, L2, PATH_FULLDIM, PATH_FUSED, PATH_PLAIN, SEG, DDTVError, Params, Solver, Stats,  # noqa: F401
                   load, make_params)
