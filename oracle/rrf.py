"""Randomized-range-finder start of eq. rrf (Sec. 4.2): A0 = V Omega with unit-norm columns.

Test infrastructure only (see the package docstring). The Gaussian test matrix Omega
(p x r_hat) is an input: the random numbers are drawn by the caller.
"""

import numpy as np


def rrf_start(V, Omega):
    """A0 = V Omega, columns normalised (V: n x p, Omega: p x r_hat)."""
    A0 = np.asarray(V, dtype=np.float64) @ np.asarray(Omega, dtype=np.float64)
    return A0 / np.linalg.norm(A0, axis=0, keepdims=True)
