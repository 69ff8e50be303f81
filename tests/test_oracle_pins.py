"""Pins for the oracle against what the paper and the mathematics fix (CPU only).

Each test compares the oracle with something other than itself: hand-worked values, closed
forms, brute-force n^d sums, calculus (finite differences), invariants, and textbook special
cases. A plausible slip anywhere in Alg. 2 (a dropped term, a wrong power, a sign, a transposed
operand) breaks at least one of them.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import explicit as ex
from oracle import implicit as im
from oracle import finite_diff, formats, lbfgs, rrf, score, stochastic
from paper_1911_03813_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(np.linalg.norm(b), 1e-300)
    return float(np.linalg.norm(a - b) / den)


def small_problem(n, p, r, d, seed, uniform_nu=False):
    g = np.random.default_rng(seed)
    V = g.standard_normal((n, p))
    nu = np.full(p, 1.0 / p) if uniform_nu else g.random(p) + 0.1
    lam = g.standard_normal(r)
    A = g.standard_normal((n, r))
    return V, nu, lam, A


# ---------------------------------------------------------------- hand-worked golden values
def test_golden_hand_examples():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        V = np.array(c["V"])
        nu = np.array(c["nu"])
        lam = np.array(c["lambda"])
        A = np.array(c["A"])
        d = c["d"]
        X = ex.moment_tensor(nu, V, d)
        assert ex.inner(X, X) == pytest.approx(c["normX2"], rel=1e-14)
        assert im.norm_x(nu, V, d) == pytest.approx(c["normX2"], rel=1e-14)
        assert ex.f_bruteforce(X, lam, A) == pytest.approx(c["f"], rel=1e-14)
        gl, GA = ex.grad_bruteforce(X, lam, A)
        np.testing.assert_allclose(gl, c["g_lambda"], rtol=1e-14)
        np.testing.assert_allclose(GA, c["G_A"], rtol=1e-14, atol=1e-13)
        f, gl2, GA2 = im.fg_implicit(nu, V, lam, A, d, alpha=c["normX2"])
        assert f == pytest.approx(c["f"], rel=1e-14)
        np.testing.assert_allclose(gl2, c["g_lambda"], rtol=1e-14)
        np.testing.assert_allclose(GA2, c["G_A"], rtol=1e-14, atol=1e-13)
        f3, gl3, GA3 = ex.fg_explicit(X, lam, A, alpha=c["normX2"])
        assert f3 == pytest.approx(c["f"], rel=1e-14)
        np.testing.assert_allclose(GA3, c["G_A"], rtol=1e-14, atol=1e-13)


# ---------------------------------------------------------------- Lemmas 3.1 and 3.2
@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_lemma_3_1_inner_of_rank_one(d):
    g = np.random.default_rng(d)
    a, b = g.standard_normal(4), g.standard_normal(4)
    lhs = ex.inner(ex.outer_power(a, d), ex.outer_power(b, d))
    assert lhs == pytest.approx(float(a @ b) ** d, rel=1e-12)
    assert ex.outer_power(a, d).shape == (4,) * d
    # one explicit entry of the outer product (eq. outer_product)
    idx = tuple(range(d)) if d <= 4 else (0, 1, 2, 3, 0)
    assert ex.outer_power(a, d)[idx] == pytest.approx(np.prod([a[i] for i in idx]))


@pytest.mark.parametrize("d", [2, 3, 4])
def test_lemma_3_2_ttsv_of_rank_one(d):
    g = np.random.default_rng(10 + d)
    a, b = g.standard_normal(3), g.standard_normal(3)
    S = ex.outer_power(b, d)
    np.testing.assert_allclose(ex.ttsv_but_one(S, a), float(a @ b) ** (d - 1) * b, rtol=1e-12)
    assert ex.ttsv_all(S, a) == pytest.approx(float(a @ b) ** d, rel=1e-12)
    # X a^d = <X a^{d-1}, a> (Sec. 2.3)
    assert ex.ttsv_all(S, a) == pytest.approx(float(ex.ttsv_but_one(S, a) @ a), rel=1e-12)


# ---------------------------------------------------------------- closed form at r = p = 1
@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_closed_form_single_sample_single_component(d):
    g = np.random.default_rng(100 + d)
    v, a = g.standard_normal(5), g.standard_normal(5)
    nu, lam = 0.7, -1.3
    expect = nu**2 * (v @ v) ** d - 2 * nu * lam * (v @ a) ** d + lam**2 * (a @ a) ** d
    alpha = nu**2 * (v @ v) ** d
    f, gl, GA = im.fg_implicit(np.array([nu]), v[:, None], np.array([lam]), a[:, None], d,
                               alpha=alpha)
    assert f == pytest.approx(expect, rel=1e-12, abs=1e-12)
    # derivative of the closed form in lambda and in a
    assert gl[0] == pytest.approx(-2 * nu * (v @ a) ** d + 2 * lam * (a @ a) ** d, rel=1e-12)
    ga = -2 * nu * lam * d * (v @ a) ** (d - 1) * v + lam**2 * 2 * d * (a @ a) ** (d - 1) * a
    np.testing.assert_allclose(GA[:, 0], ga, rtol=1e-11, atol=1e-12)
    if d <= 4:
        X = ex.moment_tensor([nu], v[:, None], d)
        assert ex.f_bruteforce(X, [lam], a[:, None]) == pytest.approx(expect, rel=1e-12)


# ---------------------------------------------------------------- brute force on tiny inputs
@pytest.mark.parametrize("n,p,r,d", [(2, 1, 1, 3), (3, 4, 2, 3), (4, 7, 3, 4), (5, 6, 2, 2),
                                     (3, 5, 4, 5), (6, 9, 3, 3)])
def test_implicit_equals_bruteforce(n, p, r, d):
    V, nu, lam, A = small_problem(n, p, r, d, seed=n * 100 + p * 10 + r + d)
    X = ex.moment_tensor(nu, V, d)
    alpha = ex.inner(X, X)
    assert im.norm_x(nu, V, d) == pytest.approx(alpha, rel=1e-12)
    f_b = ex.f_bruteforce(X, lam, A)
    gl_b, GA_b = ex.grad_bruteforce(X, lam, A)
    f, gl, GA, parts = im.fg_implicit(nu, V, lam, A, d, alpha=alpha, return_parts=True)
    scale = alpha + abs(parts["u"] @ lam) + 2 * abs(parts["w"] @ lam)
    assert abs(f - f_b) <= 1e-13 * scale
    assert rel(gl, gl_b) < 1e-12
    assert rel(GA, GA_b) < 1e-12
    # the TTSV pieces: Y_j = X a_j^{d-1}, w_j = X a_j^d, ||M||^2 by brute force
    for j in range(r):
        np.testing.assert_allclose(parts["Y"][:, j], ex.ttsv_but_one(X, A[:, j]), rtol=1e-11,
                                   atol=1e-12 * np.abs(parts["Y"]).max())
        assert parts["w"][j] == pytest.approx(ex.ttsv_all(X, A[:, j]), rel=1e-11, abs=1e-13)
    M = ex.kruskal_full(lam, A, d)
    assert im.norm_m(lam, A, d) == pytest.approx(ex.inner(M, M), rel=1e-12)
    assert float(parts["u"] @ lam) == pytest.approx(ex.inner(M, M), rel=1e-12)
    assert float(parts["w"] @ lam) == pytest.approx(ex.inner(X, M), rel=1e-11, abs=1e-13)
    # Alg. 1 on the explicit tensor gives the same outputs (Sec. 3.4)
    f1, gl1, GA1 = ex.fg_explicit(X, lam, A, alpha=alpha)
    assert abs(f1 - f_b) <= 1e-13 * scale
    assert rel(gl1, gl_b) < 1e-12 and rel(GA1, GA_b) < 1e-12


def test_gradients_against_finite_differences():
    n, p, r, d = 3, 6, 2, 3
    V, nu, lam, A = small_problem(n, p, r, d, seed=7)
    X = ex.moment_tensor(nu, V, d)

    def f_of(x):
        return ex.f_bruteforce(X, x[:r], x[r:].reshape(n, r))

    x0 = np.concatenate([lam, A.reshape(-1)])
    g_fd = finite_diff.gradient(f_of, x0, rel_step=1e-5)
    gl, GA = ex.grad_bruteforce(X, lam, A)
    assert rel(np.concatenate([gl, GA.reshape(-1)]), g_fd) < 1e-8
    # and the implicit gradient, directionally
    f_i = lambda x: im.fg_implicit(nu, V, x[:r], x[r:].reshape(n, r), d)[0]
    _, gl2, GA2 = im.fg_implicit(nu, V, lam, A, d)
    gvec = np.concatenate([gl2, GA2.reshape(-1)])
    g = np.random.default_rng(3)
    for _ in range(5):
        delta = g.standard_normal(x0.size)
        delta /= np.linalg.norm(delta)
        fd = finite_diff.directional(f_i, x0, delta, 1e-5)
        assert fd == pytest.approx(float(gvec @ delta), rel=1e-7, abs=1e-10)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("d", [3, 4])
def test_zero_residual(d):
    """A = V, lambda = nu gives M = X (eq. tensorX), so f = 0 and the gradient vanishes."""
    n, p = 5, 4
    V, nu, _, _ = small_problem(n, p, 1, d, seed=11)
    alpha = im.norm_x(nu, V, d)
    f, gl, GA = im.fg_implicit(nu, V, nu, V, d, alpha=alpha)
    assert abs(f) <= 1e-13 * alpha
    gscale = np.abs(im.fg_implicit(nu, V, nu, 0.5 * V, d)[2]).max()
    assert np.abs(gl).max() <= 1e-12 * max(1.0, alpha)
    assert np.abs(GA).max() <= 1e-12 * gscale


def test_component_and_sample_permutation():
    n, p, r, d = 4, 9, 3, 3
    V, nu, lam, A = small_problem(n, p, r, d, seed=5)
    f, gl, GA = im.fg_implicit(nu, V, lam, A, d)
    perm = np.array([2, 0, 1])
    f2, gl2, GA2 = im.fg_implicit(nu, V, lam[perm], A[:, perm], d)
    assert f2 == pytest.approx(f, rel=1e-13, abs=1e-14)
    np.testing.assert_allclose(gl2, gl[perm], rtol=1e-12)
    np.testing.assert_allclose(GA2, GA[:, perm], rtol=1e-12)
    sp = np.random.default_rng(1).permutation(p)
    f3, gl3, GA3 = im.fg_implicit(nu[sp], V[:, sp], lam, A, d)
    assert f3 == pytest.approx(f, rel=1e-13, abs=1e-14)
    np.testing.assert_allclose(GA3, GA, rtol=1e-12)


@pytest.mark.parametrize("d", [3, 4])
def test_scale_and_sign_invariance(d):
    n, p, r = 4, 7, 2
    V, nu, lam, A = small_problem(n, p, r, d, seed=21)
    f = im.fg_implicit(nu, V, lam, A, d)[0]
    c = 1.7
    lam2 = lam.copy()
    A2 = A.copy()
    lam2[0] *= c ** (-d)
    A2[:, 0] *= c
    assert im.fg_implicit(nu, V, lam2, A2, d)[0] == pytest.approx(f, rel=1e-12)
    A3 = A.copy()
    A3[:, 1] *= -1
    lam3 = lam.copy()
    if d % 2 == 1:
        lam3[1] *= -1
    assert im.fg_implicit(nu, V, lam3, A3, d)[0] == pytest.approx(f, rel=1e-12)


def test_d2_is_the_matrix_problem():
    """d = 2: X = V D_nu V^T and M = A D_lambda A^T are matrices; the objective is the squared
    Frobenius distance and its gradient is plain matrix calculus."""
    n, p, r = 6, 10, 3
    V, nu, lam, A = small_problem(n, p, r, 2, seed=31)
    Xm = V @ np.diag(nu) @ V.T
    Mm = A @ np.diag(lam) @ A.T
    R = Xm - Mm
    alpha = float(np.sum(np.linalg.eigvalsh(Xm) ** 2))
    assert im.norm_x(nu, V, 2) == pytest.approx(alpha, rel=1e-12)
    f, gl, GA = im.fg_implicit(nu, V, lam, A, 2, alpha=alpha)
    assert f == pytest.approx(float(np.sum(R * R)), rel=1e-12)
    np.testing.assert_allclose(gl, [-2 * A[:, j] @ R @ A[:, j] for j in range(r)], rtol=1e-11)
    np.testing.assert_allclose(GA, -4 * R @ A @ np.diag(lam), rtol=1e-11, atol=1e-13)


def test_chunking_and_callable_columns():
    n, p, r, d = 5, 37, 3, 4
    V, nu, lam, A = small_problem(n, p, r, d, seed=41)
    ref = im.fg_implicit(nu, V, lam, A, d)
    for chunk in (1, 4, 16, 100):
        out = im.fg_implicit(nu, V, lam, A, d, chunk=chunk)
        assert out[0] == pytest.approx(ref[0], rel=1e-13)
        assert rel(out[2], ref[2]) < 1e-13
    out = im.fg_implicit(nu, lambda a, b: V[:, a:b], lam, A, d, p=p, chunk=8)
    assert rel(out[2], ref[2]) < 1e-13
    assert im.norm_x(nu, V, d, chunk=5) == pytest.approx(im.norm_x(nu, V, d), rel=1e-13)
    # nu=None is the paper's default 1/p
    a = im.fg_implicit(None, V, lam, A, d)
    b = im.fg_implicit(np.full(p, 1.0 / p), V, lam, A, d)
    assert rel(a[2], b[2]) < 1e-15


def test_relative_error_reading():
    n, p, r, d = 4, 8, 2, 3
    V, nu, lam, A = small_problem(n, p, r, d, seed=51)
    X = ex.moment_tensor(nu, V, d)
    M = ex.kruskal_full(lam, A, d)
    alpha = im.norm_x(nu, V, d)
    f = im.fg_implicit(nu, V, lam, A, d, alpha=alpha)[0]
    assert im.relative_error(f, alpha) == pytest.approx(
        math.sqrt(ex.inner(X - M, X - M)) / math.sqrt(ex.inner(X, X)), rel=1e-10)


# ---------------------------------------------------------------- storage formats
def test_e4m3_decoder():
    torch = pytest.importorskip("torch")
    codes = np.arange(256, dtype=np.uint8)
    ours = formats.decode_e4m3(codes)
    lib = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    both_nan = np.isnan(ours) & np.isnan(lib)
    assert np.all(both_nan | (ours == lib))
    assert formats.decode_e4m3(np.uint8(0x7E)) == 448.0          # largest finite
    assert formats.decode_e4m3(np.uint8(0x08)) == 2.0 ** -6      # smallest normal
    assert formats.decode_e4m3(np.uint8(0x01)) == 2.0 ** -9      # smallest subnormal
    assert formats.decode_e4m3(np.uint8(0xB8)) == -1.0


def test_bf16_decoder():
    torch = pytest.importorskip("torch")
    x = torch.tensor([1.0, -2.5, 3.14159, 1e-30, 65504.0]).to(torch.bfloat16)
    bits = x.view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(formats.decode_bf16(bits), x.to(torch.float64).numpy())
    assert formats.decode_bf16(np.uint16(0x3F80)) == 1.0


# ---------------------------------------------------------------- score (eq. Score)
def test_score_matches_bruteforce_and_special_cases():
    g = np.random.default_rng(61)
    for r, rh in [(3, 3), (3, 5), (5, 3), (4, 4)]:
        At = g.standard_normal((8, r))
        Ah = g.standard_normal((8, rh))
        assert score.score(At, Ah) == pytest.approx(score.score_bruteforce(At, Ah), rel=1e-12)
    At = g.standard_normal((8, 4))
    perm = [2, 3, 0, 1]
    assert score.score(At, -3.0 * At[:, perm]) == pytest.approx(1.0, rel=1e-12)
    # one extra column in the estimate changes nothing
    assert score.score(At, np.hstack([At, g.standard_normal((8, 1))])) == pytest.approx(1.0)


# ---------------------------------------------------------------- L-BFGS
def test_lbfgs_rosenbrock():
    def fg(x):
        a, b = x
        f = (1 - a) ** 2 + 100 * (b - a * a) ** 2
        return f, np.array([-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)])
    out = lbfgs.lbfgs(fg, [-1.2, 1.0], pgtol=1e-8, factr=0.0, max_iters=500)
    np.testing.assert_allclose(out["x"], [1.0, 1.0], atol=1e-6)
    assert out["stop"] == lbfgs.STOP_PGTOL


def test_lbfgs_quadratic():
    g = np.random.default_rng(71)
    Q = g.standard_normal((12, 12))
    H = Q @ Q.T + 12 * np.eye(12)
    b = g.standard_normal(12)
    out = lbfgs.lbfgs(lambda x: (0.5 * x @ H @ x - b @ x, H @ x - b), np.zeros(12),
                      pgtol=1e-10, factr=0.0)
    np.testing.assert_allclose(out["x"], np.linalg.solve(H, b), rtol=1e-8, atol=1e-10)


def test_lbfgs_eckart_young_d2():
    """d = 2: the best symmetric rank-r approximation of the PSD matrix X leaves the sum of
    squares of its n - r smallest eigenvalues (Eckart-Young)."""
    n, p, r = 8, 40, 3
    g = np.random.default_rng(81)
    V = g.standard_normal((n, p))
    nu = np.full(p, 1.0 / p)
    eig = np.linalg.eigvalsh(V @ np.diag(nu) @ V.T)
    fstar = float(np.sum(eig[: n - r] ** 2))
    alpha = im.norm_x(nu, V, 2)
    lam0, A0 = inputs.random_model(n, r, seed=3, lam="equal")

    def fg(x):
        f, gl, GA = im.fg_implicit(nu, V, x[:r], x[r:].reshape(n, r, order="F"), 2, alpha=alpha)
        return f, np.concatenate([gl, GA.reshape(-1, order="F")])

    out = lbfgs.lbfgs(fg, np.concatenate([lam0, A0.reshape(-1, order="F")]), pgtol=1e-9,
                      factr=0.0, max_iters=2000)
    assert out["f"] == pytest.approx(fstar, rel=1e-6, abs=1e-10)


# ---------------------------------------------------------------- Sec. 5 and eq. rrf
def test_lemma_5_1_unbiased_by_enumeration():
    """E[X_tilde a^{d-1}] = X a^{d-1} with X = (1/p) sum v_l^{(x)d}: average over every one of the
    p^s equally likely index tuples (sampling with replacement)."""
    n, p, s, d = 3, 4, 2, 3
    g = np.random.default_rng(91)
    V = g.standard_normal((n, p))
    a = g.standard_normal((n, 1))
    X = ex.moment_tensor(np.full(p, 1.0 / p), V, d)
    target = ex.ttsv_but_one(X, a[:, 0])
    acc = np.zeros(n)
    for tup in itertools.product(range(p), repeat=s):
        parts = im.fg_implicit(np.full(s, 1.0 / s), V[:, list(tup)], [1.0], a, d,
                               return_parts=True)[3]
        acc += parts["Y"][:, 0]
    np.testing.assert_allclose(acc / p**s, target, rtol=1e-12)


def test_adam_first_step_and_schedule():
    n, p, r, d = 6, 300, 2, 3
    data = inputs.gmm(n, p, r, 0.05, seed=5, weights="equal")
    V = data["V"].T
    lam0, A0 = inputs.random_model(n, r, seed=9, lam="equal")
    g = np.random.default_rng(2)
    sample_idx = g.integers(0, p, size=(400, 50))
    est_idx = g.integers(0, p, size=200)
    # one Adam step moves every coordinate by lr * g / (|g| + eps) (bias-corrected first step)
    out1 = stochastic.adam(V, lam0, A0, d, sample_idx[:1], est_idx, epoch=1, max_epochs=1)
    _, gl, GA = stochastic.fg_sampled(V, sample_idx[0], lam0, A0, d)
    gv = np.concatenate([gl, GA.reshape(-1, order="F")])
    x0 = np.concatenate([lam0, A0.reshape(-1, order="F")])
    x1 = np.concatenate([out1["lam"], out1["A"].reshape(-1, order="F")])
    if out1["epochs"] == 1 and out1["f_est"] < stochastic.fg_sampled(V, est_idx, lam0, A0, d)[0]:
        np.testing.assert_allclose(x1 - x0, -1e-2 * gv / (np.abs(gv) + 1e-8), rtol=1e-9)
    out = stochastic.adam(V, lam0, A0, d, sample_idx, est_idx, epoch=100)
    assert out["f_est"] <= out["trace"][0]
    assert out["epochs"] >= 1


class _ScriptedSampledObjective:
    """Stand-in for the oracle's fg_sampled with everything known in advance. The estimation
    rows are marked by the index -1: the k-th estimate returns script[k] (the last entry once the
    script runs out, so a method that fails to stop runs on and fails the checks). A step row [t] returns
    the gradient +1 in every coordinate, or -1 for t in `reverse`. With a constant gradient g,
    every bias-corrected Adam step moves each coordinate by exactly -lr g / (|g| + eps), whatever
    the step count (m_t / (1 - beta1^t) = g and v_t / (1 - beta2^t) = g^2); a history that mixes
    -1 and +1 does not give that step, so a moment that was not rolled back shows."""

    def __init__(self, script, reverse=()):
        self.script = list(script)
        self.reverse = set(reverse)
        self.estimates = 0
        self.steps = []

    def __call__(self, V, idx, lam, A, d, alpha=0.0):
        idx = np.asarray(idx)
        r = len(lam)
        if idx[0] == -1:
            f = self.script[min(self.estimates, len(self.script) - 1)]
            self.estimates += 1
            return f, np.zeros(r), np.zeros(np.shape(A))
        t = int(idx[0])
        self.steps.append(t)
        sgn = -1.0 if t in self.reverse else 1.0
        return 0.0, np.full(r, sgn), np.full(np.shape(A), sgn)


@pytest.mark.parametrize("case", ["drop_then_stop", "drop_at_first_epoch"])
def test_adam_schedule_pinned(monkeypatch, case):
    """Sec. 5's schedule on scripted estimates: the learning rate drops from 1e-2 to 1e-3 exactly
    at the first non-decrease of the epoch estimate, the iterate, both Adam moments and the step
    count return to the end of the prior epoch, and the second non-decrease stops the method with
    the prior epoch's iterate and estimate. The step rows keep advancing through a rollback (each
    iteration draws fresh samples)."""
    n, r, d, epoch = 3, 2, 3, 100
    lam0 = np.array([0.5, 0.25])
    A0 = np.arange(n * r, dtype=np.float64).reshape(n, r) / 7.0
    x0 = np.concatenate([lam0, A0.reshape(-1, order="F")])
    step0 = 1e-2 / (1.0 + 1e-8)
    step1 = 1e-3 / (1.0 + 1e-8)
    if case == "drop_then_stop":
        # estimates: start 10; epochs 1, 2 decrease; epoch 3 does not (its gradient is reversed,
        # and it is rolled back); epoch 4 decreases at the lower rate; epoch 5 does not: stop
        stub = _ScriptedSampledObjective([10.0, 9.0, 8.0, 8.5, 7.0, 7.5],
                                         reverse=range(2 * epoch, 3 * epoch))
        x_expected = x0 - 2 * epoch * step0 - epoch * step1
        f_expected, epochs_expected = 7.0, 5
        trace_expected = [10.0, 9.0, 8.0, 8.5, 7.0, 7.5]
    else:
        # the first epoch's estimate does not decrease: back to the start (zero moments, t = 0)
        # at the lower rate; epoch 2 decreases; epoch 3 does not: stop with epoch 2's iterate
        stub = _ScriptedSampledObjective([5.0, 5.0, 4.0, 4.0], reverse=range(0, epoch))
        x_expected = x0 - epoch * step1
        f_expected, epochs_expected = 4.0, 3
        trace_expected = [5.0, 5.0, 4.0, 4.0]
    monkeypatch.setattr(stochastic, "fg_sampled", stub)
    sample_idx = np.arange(10 * epoch).reshape(-1, 1)
    est_idx = np.array([-1])
    out = stochastic.adam(None, lam0, A0, d, sample_idx, est_idx, epoch=epoch)
    x = np.concatenate([out["lam"], out["A"].reshape(-1, order="F")])
    np.testing.assert_allclose(x, x_expected, rtol=1e-12, atol=1e-14)
    assert out["f_est"] == f_expected
    assert out["epochs"] == epochs_expected
    assert out["trace"] == trace_expected
    assert stub.steps == list(range(epochs_expected * epoch))


def test_rrf_start_in_range_of_samples():
    g = np.random.default_rng(5)
    V = g.standard_normal((10, 4)) @ g.standard_normal((4, 50))     # rank-4 sample matrix
    Om = g.standard_normal((50, 3))
    A0 = rrf.rrf_start(V, Om)
    np.testing.assert_allclose(np.linalg.norm(A0, axis=0), 1.0, rtol=1e-14)
    Q, _ = np.linalg.qr(V[:, :4])
    assert np.linalg.norm(A0 - Q @ (Q.T @ A0)) < 1e-12
    B = V @ Om
    np.testing.assert_allclose(A0 * np.linalg.norm(B, axis=0), B, rtol=1e-13)


@pytest.mark.parametrize("n,p,d", [(3, 7, 2), (4, 9, 3), (3, 11, 4), (5, 40, 3), (6, 25, 4)])
def test_norm_x_explicit_pins(n, p, d):
    """||X||^2 from the explicitly formed X (chunked) equals brute force <X, X> and the Gram form
    of Lemma 3.4 (two routes that share no arithmetic)."""
    g = np.random.default_rng(1000 * n + p + d)
    V = g.standard_normal((n, p))
    nu = g.uniform(0.1, 1.0, p)
    Xb = ex.moment_tensor(nu, V, d)
    ref = ex.inner(Xb, Xb)
    assert ex.norm_x_explicit(nu, V, d, chunk=4) == pytest.approx(ref, rel=1e-12)
    assert im.norm_x(nu, V, d) == pytest.approx(ref, rel=1e-12)
