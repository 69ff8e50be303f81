"""Similarity score of eq. Score (Sec. 4.2): the best one-to-one matching between computed and
true component directions, averaged |cosine|.

Test infrastructure only (see the package docstring).
"""

import itertools

import numpy as np
from scipy.optimize import linear_sum_assignment


def _unit_columns(A):
    A = np.asarray(A, dtype=np.float64)
    return A / np.linalg.norm(A, axis=0, keepdims=True)


def cosine_matrix(A_true, A):
    """|a_true_j^T a_k| for unit-normalised columns (r x r_hat)."""
    return np.abs(_unit_columns(A_true).T @ _unit_columns(A))


def score(A_true, A):
    """eq. Score: max over one-to-one maps from the smaller set of columns into the larger of the
    mean |cosine| over the smaller set. The maximising map is found by the Hungarian method
    (a library assignment routine serves as the step that searches the maps)."""
    C = cosine_matrix(A_true, A)
    rows, cols = linear_sum_assignment(C, maximize=True)
    return float(C[rows, cols].sum() / min(C.shape))


def score_bruteforce(A_true, A):
    """eq. Score by enumerating every one-to-one map (small r only)."""
    C = cosine_matrix(A_true, A)
    r, rh = C.shape
    best = -1.0
    if rh >= r:
        for perm in itertools.permutations(range(rh), r):
            best = max(best, sum(C[j, perm[j]] for j in range(r)) / r)
    else:
        for perm in itertools.permutations(range(r), rh):
            best = max(best, sum(C[perm[j], j] for j in range(rh)) / rh)
    return float(best)
