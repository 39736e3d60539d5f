"""GB300-native randomized CP decomposition (Erichson, Manohar, Brunton & Kutz, arXiv 1703.09074).

The method's steps run in hand-written sm_103a CUDA kernels behind the C ABI of
``include/rcp.h`` (``librcp.so``); this package only marshals arguments.
"""

from .api import (BatchedPlan, Plan, WarmStartNet, decompose, measure_fma_rate,  # noqa: F401
                  synth_cp, test_normals, ws_canonicalize, ws_loss)
from ._lib import RcpError, load  # noqa: F401
