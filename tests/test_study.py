"""The Gaussian-mixture study driver (Sec. 4.2): its score against the oracle's eq. Score, and one
scenario on the GPU (-m gpu)."""

import numpy as np
import pytest

from oracle import score as oscore
from paper_1911_03813_gb300 import inputs, study


@pytest.mark.parametrize("r,r_hat", [(3, 3), (5, 3), (3, 5), (7, 6), (6, 7), (1, 4), (4, 1),
                                     (10, 8), (12, 12)])
def test_score_matches_oracle(r, r_hat):
    """The study's own assignment search (dynamic programming over subsets) against the oracle's
    enumeration of every one-to-one map (up to 7 components), and against the oracle's Hungarian
    form above that."""
    g = inputs.rng(100 * r + r_hat)
    A_true = g.standard_normal((40, r))
    A = A_true[:, g.permutation(r)[: min(r, r_hat)]] * g.choice([-2.0, 3.0], min(r, r_hat))
    if r_hat > r:
        A = np.concatenate([A, g.standard_normal((40, r_hat - r))], axis=1)
    A = A + 0.1 * g.standard_normal(A.shape)
    if max(r, r_hat) <= 7:
        assert study.score(A_true, A) == pytest.approx(oscore.score_bruteforce(A_true, A),
                                                       abs=1e-14)
    else:
        assert study.score(A_true, A) == pytest.approx(oscore.score(A_true, A), abs=1e-14)


def test_score_is_one_for_a_permuted_rescaled_copy():
    g = inputs.rng(5)
    A_true = g.standard_normal((20, 6))
    A = A_true[:, [4, 2, 0, 5, 1, 3]] * np.array([-1.0, 2.0, 0.5, -3.0, 1.0, 7.0])
    assert study.score(A_true, A) == pytest.approx(1.0, abs=1e-14)


@pytest.mark.gpu
def test_study_scenario_on_gpu():
    """d = 3, r = 3, sigma = 1e-2, n = 500: every r_hat in 1..5 from 4 starts each. The reported
    f of each best fit equals the oracle's evaluation at the returned iterate, and r_hat = r
    recovers the means."""
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_1911_03813_gb300 import stmf
    torch.cuda.set_device(0)
    d, r, sigma = 3, 3, 1e-2
    with stmf.Server(max_fits=20, n_max=500, r_max=5, mem_budget=4 << 30) as srv:
        rows = study.scenario(srv, d, r, sigma, starts=4, seed=11)
    assert [row["r_hat"] for row in rows] == [1, 2, 3, 4, 5]
    data = inputs.gmm(500, 250 * r, r, sigma, seed=11, weights="equal", means="congruent",
                      equal_counts=True)
    V = np.asarray(inputs.to_storage(data["V"], "f32")["data"][:, :500], dtype=np.float64)
    alpha = oracle.norm_x(None, V.T, d)
    for row in rows:
        assert row["alpha"] == pytest.approx(alpha, rel=1e-5)
        f_o = oracle.fg_implicit(None, V.T, row["lam"], row["A"], d, alpha=alpha)[0]
        assert abs(row["f"] - f_o) <= 1e-5 * alpha
        assert row["stop"] in (1, 2)
    best = rows[2]
    assert best["score"] > 0.99 and best["rel_error"] < 0.2, best
    assert best["score"] == pytest.approx(oracle.score.score(data["means"], best["A"]), abs=1e-12)
