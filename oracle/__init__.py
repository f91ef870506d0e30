"""FP64 CPU oracle for the SV-LCOV truncated-SVD update step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library.

Three independent FP64 implementations of one update step:

* ``dense.define_*``  -- the definition itself ("maintaining an approximate
  rank-k truncated SVD", Section 3.3): materialise the updated dense matrix
  built from the current rank-k factors and take its truncated SVD.
* ``dense.zha_simon_*`` -- the Zha-Simon projection update of Section 2.1 with
  an explicit dense Householder QR of the augmented matrix.
* ``svlcov.State`` -- the paper's sparse method: Algorithm 2 (Gram-Schmidt in
  SV-LCOV space) with Algorithms 3, 4 and 11 acting on the extended
  decomposition U' U'' Sigma V''^T V'^T of Section 3.2.

``checks`` holds the error measures used to compare results; ``backward``
the reference gradient of one add-columns step (torch float64 autograd of
the dense formulation, and finite differences of the sparse method);
``scoring`` the pair scores of the downstream tasks.
"""
from . import dense, svlcov, checks, scoring  # noqa: F401
