"""Run-only cross-check of the oracle's L-BFGS against SciPy's L-BFGS-B (the solver family the
paper used, Sec. 4) on the implicit objective: both reach the same optimum (CPU only)."""

import numpy as np
import pytest

import oracle
from oracle import lbfgs
from paper_1911_03813_gb300 import inputs


def test_oracle_lbfgs_matches_scipy_lbfgsb():
    scipy_opt = pytest.importorskip("scipy.optimize")
    n, p, r, d = 6, 300, 2, 3
    data = inputs.gmm(n, p, r, 0.0, seed=3, weights="equal")
    V = data["V"].T
    alpha = oracle.norm_x(None, V, d)
    # randomized-range-finder start (eq. rrf): with noiseless data it lies in the span of the means
    from oracle import rrf
    A0 = rrf.rrf_start(V, inputs.rng(4).standard_normal((p, r)))
    lam0 = np.full(r, 1.0 / r)

    def fg(x):
        f, gl, GA = oracle.fg_implicit(None, V, x[:r], x[r:].reshape(n, r, order="F"), d,
                                       alpha=alpha)
        return f, np.concatenate([gl, GA.reshape(-1, order="F")])

    x0 = np.concatenate([lam0, A0.reshape(-1, order="F")])
    ours = lbfgs.lbfgs(fg, x0, pgtol=1e-10, factr=0.0, max_iters=2000)
    ref = scipy_opt.minimize(fg, x0, jac=True, method="L-BFGS-B",
                             options=dict(maxcor=5, gtol=1e-10, ftol=0.0, maxiter=2000))
    assert abs(ours["f"] - ref.fun) <= 1e-12 * alpha
    assert abs(ours["f"]) <= 1e-12 * alpha
