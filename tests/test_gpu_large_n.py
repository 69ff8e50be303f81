"""Samples with up to 512 features (-m gpu): the Gaussian-mixture study of Sec. 4.2 fixes n = 500.

BF16 and E4M3 samples with 256 < n <= 512 (r <= 16) take the sub-stage tensor-core pass
(128-feature sub-stages); FP32 and FP64 samples past n = 256 run on the CUDA cores: 64-sample
tiles (32 for FP64 samples, whose 64-sample tile does not fit in shared memory); the Gram pass is
staged in feature chunks, and the range finder runs in FP32 when its FP64 tile does not fit.
Tolerances: FP64 1e-12; FP32 (FP32 arithmetic) 1e-5 normwise and entry by entry with a floor of
0.01 of the largest entry; BF16/E4M3 on the tensor cores 5e-6 normwise and 1e-5 entry by entry
with a floor of 0.1 of the largest entry (as for the whole-tile pass); the FP32 range finder is
compared at 1e-5.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import formats, score  # noqa: E402
from oracle import lbfgs as olbfgs  # noqa: E402
from paper_1911_03813_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 5e-6, "e4m3": 5e-6}
TOL_EL = {"f64": (1e-12, 0.01), "f32": (1e-5, 0.01), "bf16": (1e-5, 0.1), "e4m3": (1e-5, 0.1)}


@pytest.fixture(scope="module")
def stmf():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_03813_gb300 import stmf as s
    torch.cuda.set_device(0)
    return s


def decoded(st):
    bits = inputs.storage_bits(st)
    if st["dtype"] == "bf16":
        return formats.decode_bf16(bits)
    if st["dtype"] == "e4m3":
        return formats.dequantize_e4m3(bits, st["scale"].cpu().numpy())
    return np.asarray(bits, dtype=np.float64)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def elementwise(a, b, c):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.max(np.abs(a - b) / (np.abs(b) + c * np.max(np.abs(b)) + 1e-300)))


def dev_model(lam, A):
    lam_t = torch.tensor(lam, dtype=torch.float64, device="cuda")
    A_t = torch.tensor(np.ascontiguousarray(A.T), dtype=torch.float64, device="cuda").T
    return lam_t, A_t


@pytest.mark.parametrize("dtype,n,p,r,d", [
    ("f32", 500, 20001, 16, 3), ("bf16", 500, 20001, 16, 4), ("e4m3", 500, 9001, 10, 3),
    ("f32", 512, 5000, 32, 4), ("bf16", 300, 7001, 5, 4),
    ("f64", 500, 3001, 12, 3),   # 32-sample FP64 tiles
    ("f64", 300, 7001, 4, 4),
    # the sub-stage tensor-core pass: both sides of each 128-feature boundary, r on both sides
    # of 8, the largest n, ragged tails and enough tiles per block for the ring to wrap
    ("bf16", 257, 300001, 16, 3), ("e4m3", 257, 30001, 8, 4), ("bf16", 384, 100003, 12, 4),
    ("e4m3", 385, 50001, 16, 3), ("bf16", 512, 200001, 16, 4), ("e4m3", 512, 70001, 9, 4),
    ("bf16", 500, 1000, 20, 3),  # r > 16: the CUDA-core pass
])
def test_fg_parity_large_n(stmf, dtype, n, p, r, d):
    data = inputs.gmm(n, p, 5, 0.1, seed=n + p, means="congruent")
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    lam, A = inputs.random_model(n, r, seed=r + n)
    f_ref, gl_ref, GA_ref, parts = oracle.fg_implicit(None, decoded(st).T, lam, A, d,
                                                      return_parts=True)
    f, gl, GA = stmf.fg(st, None, d, *dev_model(lam, A))
    torch.cuda.synchronize()
    assert stmf.default_context().device_status() == 0
    S = abs(parts["u"] @ lam) + 2 * abs(parts["w"] @ lam)
    tol = TOL[dtype] if r <= 16 else max(TOL[dtype], 1e-5)
    assert abs(f.item() - f_ref) <= tol * S
    assert rel(gl.cpu().numpy(), gl_ref) <= tol
    assert rel(GA.cpu().numpy(), GA_ref) <= tol
    tol_el, c = TOL_EL[dtype] if r <= 16 else (1e-5, 0.01)
    assert elementwise(gl.cpu().numpy(), gl_ref, c) <= tol_el
    assert elementwise(GA.cpu().numpy(), GA_ref, c) <= tol_el


@pytest.mark.parametrize("dtype,n,r", [("f64", 512, 32), ("f32", 512, 64)])
def test_fg_large_n_limits(stmf, dtype, n, r):
    """n x r past what the CUDA-core pass holds is refused before any work."""
    data = inputs.gmm(n, 100, 3, 0.1, seed=1)
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    lam, A = inputs.random_model(n, r, seed=2)
    with pytest.raises(stmf.StmfError):
        stmf.fg(st, None, 3, *dev_model(lam, A))


@pytest.mark.parametrize("dtype,n,p,d", [("f64", 500, 3001, 3), ("f32", 512, 2500, 4),
                                         ("bf16", 500, 3001, 4), ("e4m3", 300, 2000, 3)])
def test_norm_x_large_n(stmf, dtype, n, p, d):
    """||X||^2 with the Gram pass staged in chunks of 128 features."""
    data = inputs.gmm(n, p, 5, 0.1, seed=p)
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    ref = oracle.norm_x(None, decoded(st).T, d)
    got = stmf.norm_x(st, None, d).item()
    torch.cuda.synchronize()
    tol = 1e-12 if dtype == "f64" else 1e-5
    assert abs(got - ref) <= tol * abs(ref), (got, ref)


@pytest.mark.parametrize("dtype,n,p,r_hat", [("bf16", 500, 4000, 10), ("f32", 500, 3000, 12),
                                             ("f64", 500, 2000, 8), ("bf16", 512, 3000, 32),
                                             ("f32", 512, 2000, 28)])
def test_rrf_start_large_n(stmf, dtype, n, p, r_hat):
    """eq. rrf at n = 500 and 512: FP64 samples draw and accumulate in FP64 (32-sample tiles);
    the other types draw and multiply in FP32 and fold the FP32 sums into FP64."""
    from oracle import philox, rrf
    data = inputs.gmm(n, p, 5, 0.1, seed=p, means="congruent")
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    seed = 0x5EED0000 + n
    ref = rrf.rrf_start(decoded(st).T, philox.gaussian_test_matrix(p, r_hat, seed))
    A0 = stmf.rrf_start(st, r_hat, seed).cpu().numpy()
    tol = 1e-12 if dtype == "f64" else 1e-5
    assert rel(A0, ref) < tol, rel(A0, ref)


@pytest.mark.parametrize("d", [3, 4])
def test_fit_gmm_study_shape(stmf, d):
    """One scenario of the Gaussian-mixture study (Sec. 4.2): n = 500, r = 5 congruent means
    (pairwise cosine 0.5), sigma = 1e-2, p = 250 r samples with equal counts, r_hat = r, pgtol =
    1e-4, randomized range finder start; FP32 samples. The device fit stops by the paper's rule,
    its f lies within the paper's 2e-5 band (relative to alpha) of the FP64 oracle's fit from the
    same start, and its score is within 0.01 of the oracle's."""
    n, r, sigma = 500, 5, 1e-2
    p = 250 * r
    data = inputs.gmm(n, p, r, sigma, seed=500 + d, weights="equal", means="congruent",
                      equal_counts=True)
    st = inputs.to_storage(data["V"], "f32", device="cuda")
    Vd = decoded(st)
    from oracle import philox, rrf
    seed = 9000 + d
    A0 = rrf.rrf_start(Vd.T, philox.gaussian_test_matrix(p, r, seed))
    lam0 = np.full(r, 1.0 / r)
    lam_t, A_t = dev_model(lam0, A0)
    res = stmf.fit(st, None, d, lam_t, A_t, pgtol=1e-4, max_evals=5000)
    torch.cuda.synchronize()
    assert res["status"] == 0 and res["stop"] in (1, 2), res
    alpha = oracle.norm_x(None, Vd.T, d)
    assert res["alpha"] == pytest.approx(alpha, rel=1e-5)

    def fg(x):
        f, gl, GA = oracle.fg_implicit(None, Vd.T, x[:r], x[r:].reshape(n, r, order="F"), d,
                                       alpha=alpha)
        return f, np.concatenate([gl, GA.reshape(-1, order="F")])

    out = olbfgs.lbfgs(fg, np.concatenate([lam0, A0.reshape(-1, order="F")]), pgtol=1e-4,
                       max_evals=5000)
    A_o = out["x"][r:].reshape(n, r, order="F")
    assert abs(res["f"] - out["f"]) <= 2e-5 * alpha, (res["f"], out["f"], alpha)
    s_dev = score.score(data["means"], A_t.cpu().numpy())
    s_orc = score.score(data["means"], A_o)
    assert s_dev >= s_orc - 0.01, (s_dev, s_orc)
