"""GB300-native spacetime finite-element Dirac solver (hot path).

The compute path is the CUDA library ``lib/libdiracst.so`` built from
``csrc/`` for sm_103a; ``binding`` exposes its C ABI (``include/diracst.h``)
to Python with the same function names.  PyTorch supplies device memory and
streams only.
"""

from . import binding  # noqa: F401  (fails loudly if the library is not built)
from .binding import (DST_BC_DIRICHLET, DST_BC_OPEN, DST_BC_PERIODIC, DST_FP32, DST_FP64,  # noqa: F401
                      DstError, Mesh)
