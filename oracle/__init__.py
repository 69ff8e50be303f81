"""Oracle: a plain, slow, FP64 CPU restatement of the method of Sherman & Kolda,
"Estimating Higher-Order Moments Using Symmetric Tensor Decomposition" (arXiv 1911.03813).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it. The product path (the CUDA library and its
Python binding) never imports, calls or links anything here, and this package imports nothing
from the product: the two share no code.

Modules
-------
explicit    n^d arrays formed element by element: the moment tensor (eq. tensorX), symmetric
            outer products (eq. outer_product), inner products (eq. tensorIP), TTSV (eqs. ExpXbd,
            ExpXbdd), the objective (eq. optFunc) by brute force, and Alg. 1 (fg_explicit).
implicit    Alg. 2 (fg_implicit) in the paper's order, and ||X||^2 by Lemma 3.4 applied to X.
formats     decoding of the storage formats of V (bfloat16, OCP FP8 e4m3) from their bit-level
            definitions; the storage formats are not part of the paper.
lbfgs       limited-memory BFGS with a strong-Wolfe bracketing/zoom line search (Nocedal & Wright,
            Numerical Optimization, 2nd ed., Alg. 7.4 and Algs. 3.5/3.6), the optimiser of Sec. 4.
score       the similarity score of eq. Score (Sec. 4.2).
stochastic  Lemma 5.1's sampled Kruskal tensor and the Adam schedule of Sec. 5.
rrf         the randomized-range-finder start of eq. rrf (Sec. 4.2).
finite_diff central differences of a scalar function.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, brute force on tiny inputs, invariants, textbook
special cases). Functions without such a pin carry the words "parity unpinned" in their
docstring.
"""

from . import explicit, implicit, formats, lbfgs, score, finite_diff, stochastic, rrf  # noqa: F401
from .implicit import fg_implicit, norm_x  # noqa: F401
