"""GB300 (sm_103a) implementation of the D2Q9 lattice-Boltzmann step with
moving rigid disks and the Galilean-invariant momentum-exchange force of
Wen et al., arXiv:1303.0625.

The computation runs in the CUDA library ``_build/liblbm_gb300.so`` (sources
in ``csrc/``, C ABI in ``include/lbm.h``); ``lbm`` is its Python binding.
"""
from . import build  # noqa: F401
from .lbm import *  # noqa: F401,F403
from .lbm import Batch, Lattice, load  # noqa: F401
