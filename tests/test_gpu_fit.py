"""On-device L-BFGS (stmf_fit) against the oracle's L-BFGS and against known optima (-m gpu).

Optimisation paths are not compared step by step: the paper notes that round-off alone changes
the path (Sec. 4.1). What is pinned: the stopping rule holds at the returned iterate when the
oracle re-evaluates it, the final objective lies within the paper's band of the oracle's own
fit from the same start (paired runs differ by at most 2e-5 in Sec. 4.1; measured here relative
to alpha), recovery scores, exact recovery from noiseless data, and the d = 2 optimum.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import lbfgs as olbfgs  # noqa: E402
from oracle import formats  # noqa: E402
from oracle import score  # noqa: E402
from paper_1911_03813_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stmf():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_03813_gb300 import stmf as s
    torch.cuda.set_device(0)
    return s


def gpu_fit(stmf, st, nu, lam0, A0, d, **kw):
    lam = torch.tensor(lam0, dtype=torch.float64, device="cuda")
    A = torch.tensor(np.ascontiguousarray(A0.T), dtype=torch.float64, device="cuda").T
    nu_t = None if nu is None else torch.tensor(nu, dtype=torch.float64, device="cuda")
    res = stmf.fit(st, nu_t, d, lam, A, **kw)
    torch.cuda.synchronize()
    return res, lam.cpu().numpy(), A.cpu().numpy()


def oracle_fit(V, nu, lam0, A0, d, alpha, **kw):
    n, r = A0.shape

    def fg(x):
        f, gl, GA = oracle.fg_implicit(nu, V.T, x[:r], x[r:].reshape(n, r, order="F"), d,
                                       alpha=alpha)
        return f, np.concatenate([gl, GA.reshape(-1, order="F")])

    out = olbfgs.lbfgs(fg, np.concatenate([lam0, A0.reshape(-1, order="F")]), **kw)
    return out, out["x"][:r], out["x"][r:].reshape(n, r, order="F")


def test_fit_small_fp64_config(stmf):
    """n=10, d=3, r=2, p=1000 FP64 Gaussian mixture (weights 0.6/0.4, sigma=0.01), seeded random
    start, alpha = ||X||^2: full fit against the oracle's fit from the same start."""
    n, p, r, d = 10, 1000, 2, 3
    data = inputs.gmm(n, p, r, 0.01, seed=1, weights=[0.6, 0.4])
    lam0, A0 = inputs.random_model(n, r, seed=2, lam="equal")
    st = inputs.to_storage(data["V"], "f64", device="cuda")
    pgtol = 1e-9
    res, lam, A = gpu_fit(stmf, st, None, lam0, A0, d, pgtol=pgtol)
    alpha = oracle.norm_x(None, data["V"].T, d)
    assert res["status"] == 0
    assert res["alpha"] == pytest.approx(alpha, rel=1e-12)
    assert res["stop"] in (1, 2), res
    # the returned iterate, re-evaluated by the oracle
    f_o, gl_o, GA_o = oracle.fg_implicit(None, data["V"].T, lam, A, d, alpha=alpha)
    assert f_o == pytest.approx(res["f"], rel=1e-10, abs=1e-14)
    ginf = max(np.abs(gl_o).max(), np.abs(GA_o).max())
    if res["stop"] == 1:
        assert ginf <= pgtol * (1 + 1e-6)
    out, lam_r, A_r = oracle_fit(data["V"], None, lam0, A0, d, alpha, pgtol=pgtol)
    assert abs(res["f"] - out["f"]) <= 2e-5 * alpha
    assert score.score(data["means"], A) >= score.score(data["means"], A_r) - 0.01
    assert oracle.implicit.relative_error(res["f"], alpha) < 0.05


def test_fit_exact_recovery_noiseless(stmf):
    """sigma = 0: X has rank r exactly and the fit reaches f ~ 0 with score 1."""
    n, p, r, d = 12, 600, 3, 3
    # (a seed whose randomized-range-finder start the oracle's own fit takes to f = 0; from other
    # starts both optimisers can stall at the same spurious stationary point)
    data = inputs.gmm(n, p, r, 0.0, seed=17, weights="equal")
    # randomized-range-finder start (eq. rrf), computed on the host as an input to the fit
    A0 = oracle.rrf.rrf_start(data["V"].T, inputs.rng(18).standard_normal((p, r)))
    lam0 = np.full(r, 1.0 / r)
    st = inputs.to_storage(data["V"], "f64", device="cuda")
    res, lam, A = gpu_fit(stmf, st, None, lam0, A0, d, pgtol=1e-12, factr=0.0, max_evals=5000)
    assert res["status"] == 0
    assert oracle.implicit.relative_error(res["f"], res["alpha"]) < 1e-6, res
    assert score.score(data["means"], A) > 1 - 1e-6


def test_fit_d2_eckart_young(stmf):
    """d = 2: the optimum leaves the squares of the n - r smallest eigenvalues of X."""
    n, p, r, d = 8, 400, 3, 2
    V = inputs.rng(21).standard_normal((p, n))
    eig = np.linalg.eigvalsh(V.T @ V / p)
    fstar = float(np.sum(eig[: n - r] ** 2))
    lam0, A0 = inputs.random_model(n, r, seed=22, lam="equal")
    st = inputs.to_storage(V, "f64", device="cuda")
    res, _, _ = gpu_fit(stmf, st, None, lam0, A0, d, pgtol=1e-10, factr=0.0, max_evals=20000)
    assert res["f"] == pytest.approx(fstar, rel=1e-6, abs=1e-12), res


def test_fit_bf16_and_budget(stmf):
    """BF16 samples through the tensor-core pass; max_evals stops the method."""
    n, p, r, d = 32, 20000, 4, 4
    data = inputs.gmm(n, p, r, 0.05, seed=31, weights="equal")
    st = inputs.to_storage(data["V"], "bf16", device="cuda")
    from oracle import formats
    Vb = formats.decode_bf16(inputs.storage_bits(st))
    A0 = oracle.rrf.rrf_start(Vb.T, inputs.rng(32).standard_normal((p, r)))
    lam0 = np.full(r, 1.0 / r)
    res, lam, A = gpu_fit(stmf, st, None, lam0, A0, d, pgtol=1e-7, max_evals=40)
    assert res["evals"] <= 40 and res["stop"] in (1, 2, 4)
    # Path-level parity while the objective still drops fast: at equal evaluation budgets the
    # device optimiser has taken the same iterations as the oracle's (same iterate count, f equal
    # to the evaluation's precision).
    alpha = oracle.norm_x(None, Vb.T, d)
    for me in (3, 5, 10):
        res_k, _, _ = gpu_fit(stmf, st, None, lam0, A0, d, pgtol=1e-8, max_evals=me)
        out_k, _, _ = oracle_fit(Vb, None, lam0, A0, d, alpha, pgtol=1e-8, max_evals=me)
        assert res_k["iters"] == out_k["iters"], (me, res_k, out_k["iters"])
        assert abs(res_k["f"] - out_k["f"]) <= 1e-5 * alpha, (me, res_k["f"], out_k["f"])
    # A full run ends at a near-stationary point (re-evaluated by the oracle). factr = 0: a BF16
    # evaluation carries ~1e-7 noise in f, more than the default relative-decrease test
    # (factr * eps = 2.2e-9) can tell from progress.
    res2, lam2, A2 = gpu_fit(stmf, st, None, lam0, A0, d, pgtol=1e-6, factr=0.0, max_evals=3000)
    assert res2["stop"] in (1, 5), res2
    _, gl0, GA0 = oracle.fg_implicit(None, Vb.T, lam0, A0, d)
    _, gl2, GA2 = oracle.fg_implicit(None, Vb.T, lam2, A2, d)
    g0 = max(np.abs(gl0).max(), np.abs(GA0).max())
    g2 = max(np.abs(gl2).max(), np.abs(GA2).max())
    assert g2 <= 1e-3 * g0, (g2, g0)
    assert res2["f"] < oracle.fg_implicit(None, Vb.T, lam0, A0, d, alpha=alpha)[0]
    bad = stmf.fit_options(m=0)
    with pytest.raises(stmf.StmfError):
        gpu_fit(stmf, st, None, lam0, A0, d, opts=bad)


@pytest.mark.parametrize("sigma", [1e-3, 1e-1])
def test_fit_full_size_bf16(stmf, sigma):
    """n=256, d=4, r=16, p=2^24 BF16 Gaussian mixture: a full fit from the randomized range
    finder start (eq. rrf), run to convergence. The model floor set by the sigma^2 terms (Sec. 4.2)
    keeps the relative error from reaching 1e-6 at these sigma, so what is checked is the
    accuracy of the evaluation at the fit: the device's f at the returned iterate equals the
    FP64 oracle's to 1e-6 of the cancellation scale S = alpha + |lambda^T u| + 2 |w^T lambda|, and
    the stopping rule holds there. The attained
    relative error is printed."""
    n, p, r, d = 256, 1 << 24, 16, 4
    st = inputs.gmm_device(n, p, r, sigma, seed=4096, device="cuda", out_dtype="bf16")
    A0 = stmf.rrf_start(st, r, seed=4097)
    lam = torch.full((r,), 1.0 / r, dtype=torch.float64, device="cuda")
    A = torch.empty((r, n), dtype=torch.float64, device="cuda").T
    A.copy_(A0)
    res = stmf.fit(st, None, d, lam, A, pgtol=1e-6, factr=1e9, max_evals=3000)
    torch.cuda.synchronize()
    assert res["status"] == 0 and res["stop"] in (1, 2, 5), res
    alpha = res["alpha"]
    lam_h, A_h = lam.cpu().numpy(), A.cpu().numpy()
    data = st["data"]

    def cols(c0, c1):
        return formats.decode_bf16(inputs.storage_bits(dict(st, data=data[c0:c1]))).T

    f_o, gl_o, GA_o, parts = oracle.fg_implicit(None, cols, lam_h, A_h, d, p=p, chunk=1 << 16,
                                                return_parts=True)
    # the device's f includes alpha; the oracle's here is the shifted one. The evaluation at the
    # fit is accurate to 1e-6 of the scale of the terms that cancel in f (alpha is about a third
    # of that scale here).
    S = alpha + abs(parts["u"] @ lam_h) + 2 * abs(parts["w"] @ lam_h)
    err = abs((res["f"] - alpha) - f_o)
    print(f"\nfull-size fit sigma={sigma}: |f - f_oracle| = {err:.2e} = {err / alpha:.2e} alpha "
          f"= {err / S:.2e} S")
    assert err <= 1e-6 * S, (res["f"] - alpha, f_o, alpha, S)
    if res["stop"] == 1:
        assert max(np.abs(gl_o).max(), np.abs(GA_o).max()) <= 1e-6 * 1.01 + 1e-7
    rel_err = oracle.implicit.relative_error(res["f"], alpha)
    print(f"\nfull-size BF16 fit, sigma={sigma}: relative error {rel_err:.3e}, "
          f"{res['iters']} iterations, {res['evals']} evaluations, stop {res['stop']}")
    assert rel_err < 1.0
    del st
    torch.cuda.empty_cache()
