"""Plain FP64 CPU oracle for randomized Tucker compression (Minster, Saibaba, Kilmer).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it. The product
path (the CUDA library and its Python binding) never imports, calls or links
anything here, and nothing here imports the product path.

Every function restates one passage of the paper in plain numpy, in the paper's
order of steps, with no blocking or fusion beyond what the passage states:

* ``rng``      -- the Gaussian test matrices Omega_j (Sec. 2.4, Sec. 3.1: entries
                  i.i.d. N(0,1), generated on the fly).  The paper fixes only the
                  distribution; the counter-based construction (Philox4x32-10 +
                  Box-Muller in FP32) is this library's own specification.
* ``tensor``   -- unfolding, mode product and Tucker reconstruction (Sec. 2.1, Eq. kron).
* ``tucker``   -- RandSVD (Alg. 1), R-HOSVD (Alg. 2), R-STHOSVD (Alg. 3),
                  HOSVD / STHOSVD (Sec. 2.2), adaptive variants (Alg. 4, Alg. 5),
                  SP-STHOSVD with strong RRQR (Alg. 6), error measures.

Pins: see ``tests/test_oracle_*.py``.  A function without an independent pin says
"parity unpinned" in its docstring.
"""

from . import rng, tensor, tucker  # noqa: F401
