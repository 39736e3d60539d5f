"""Plain, slow FP64 CPU oracle for randomized CP decomposition (rCP-ALS).

TEST INFRASTRUCTURE ONLY.  This package states, step by step and in plain
numpy, what the randomized CP method of Erichson, Manohar, Brunton & Kutz
("Randomized CP Tensor Decomposition", arXiv 1703.09074) computes:

* Section 3.1 / Algorithm 1: randomized tensor compression (Gaussian test
  matrix, normalised power iterations, QR, mode-n projection),
* Section 3.2.1 / Algorithm 2: CP-ALS on the compressed tensor with the
  Khatri-Rao product pseudo-inverse, normalisation, the fit test of
  Section 3.3, and the back-projection of Eq. (qbs),
* the relative error of Section 4.

It shares no code with the CUDA path and never imports it.  Only the test
suite (``tests/``), ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path
never routes through it.

Library primitives (numpy matmul, LAPACK QR, SVD-based pinv) serve as single
steps; nothing is blocked, fused or reordered beyond what the paper states.
"""

from . import philox, tensor, rcp  # noqa: F401
