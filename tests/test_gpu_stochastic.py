"""Sec. 5 on the device: sampled evaluation (Lemma 5.1) and the Adam schedule (-m gpu).

The sampled rows are inputs shared by the device and the oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import formats, stochastic  # noqa: E402
from paper_1911_03813_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-5, "e4m3": 1e-5}


@pytest.fixture(scope="module")
def stmf():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_03813_gb300 import stmf as s
    torch.cuda.set_device(0)
    return s


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("s", [1, 10, 100, 1000])
def test_fg_sampled_parity(stmf, dtype, s):
    n, p, r, d = 50, 20000, 6, 3
    data = inputs.gmm(n, p, 6, 0.1, seed=s + 3)
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    bits = inputs.storage_bits(st)
    Vd = formats.decode_bf16(bits) if dtype == "bf16" else np.asarray(bits, dtype=np.float64)
    idx = np.random.default_rng(s).integers(0, p, size=s)
    lam, A = inputs.random_model(n, r, seed=s)
    f_ref, gl_ref, GA_ref = stochastic.fg_sampled(Vd.T, idx, lam, A, d)
    f, gl, GA = stmf.fg_sampled(st, torch.tensor(idx, device="cuda"), d,
                                torch.tensor(lam, device="cuda"),
                                torch.tensor(A.T.copy(), device="cuda").T)
    torch.cuda.synchronize()
    assert stmf.default_context().device_status() == 0
    scale = abs(f_ref) + 1e-300
    assert abs(f.item() - f_ref) <= TOL[dtype] * max(scale, np.abs(gl_ref).max())
    assert rel(gl.cpu().numpy(), gl_ref) <= TOL[dtype]
    assert rel(GA.cpu().numpy(), GA_ref) <= TOL[dtype]


def test_fg_sampled_out_of_range_index_is_reported(stmf):
    st = inputs.to_storage(np.ones((100, 8)), "f32", device="cuda")
    idx = torch.tensor([0, 5, 100], device="cuda")   # 100 is outside [0, p)
    stmf.fg_sampled(st, idx, 3, torch.ones(2, dtype=torch.float64, device="cuda"),
                    torch.ones((2, 8), dtype=torch.float64, device="cuda").T)
    assert stmf.default_context().device_status() == 1   # STMF_EINVAL


@pytest.mark.parametrize("dtype", ["bf16", "f32", "e4m3"])
@pytest.mark.parametrize("n,s,r", [(256, 30001, 16), (100, 5000, 10), (37, 129, 3)])
def test_fg_sampled_tensor_cores(stmf, dtype, n, s, r):
    """Rows gathered by the tensor-core passes (BF16: gather warps of the whole-tile pass; E4M3:
    its converter warps fetch the code rows before widening them, each sample's scale taken
    through the index; FP32: the converter warps of the sub-stage pass fetch the rows before
    splitting them): several tiles and a ragged last one, n = 100 and 37 ending inside a 16-byte
    chunk, rows drawn with repeats; against the oracle on the stored values, normwise and entry
    by entry."""
    p, d = 60000, 4
    data = inputs.gmm(n, p, 8, 0.1, seed=n + s)
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    bits = inputs.storage_bits(st)
    if dtype == "bf16":
        Vd = formats.decode_bf16(bits)
    elif dtype == "e4m3":
        Vd = formats.dequantize_e4m3(bits, st["scale"].cpu().numpy())
    else:
        Vd = np.asarray(bits, dtype=np.float64)
    idx = np.random.default_rng(s).integers(0, p, size=s)
    lam, A = inputs.random_model(n, r, seed=s)
    f_ref, gl_ref, GA_ref = stochastic.fg_sampled(Vd.T, idx, lam, A, d)
    f, gl, GA = stmf.fg_sampled(st, torch.tensor(idx, device="cuda"), d,
                                torch.tensor(lam, device="cuda"),
                                torch.tensor(A.T.copy(), device="cuda").T)
    torch.cuda.synchronize()
    assert stmf.default_context().device_status() == 0
    tol = TOL[dtype]
    assert abs(f.item() - f_ref) <= tol * max(abs(f_ref), np.abs(gl_ref).max())
    gl_h, GA_h = gl.cpu().numpy(), GA.cpu().numpy()
    assert rel(gl_h, gl_ref) <= tol and rel(GA_h, GA_ref) <= tol
    assert np.max(np.abs(GA_h - GA_ref)) <= 10 * tol * np.max(np.abs(GA_ref))


def test_fg_sampled_tensor_cores_out_of_range_index(stmf):
    """A sampled BF16 row outside the storage reads as zero and is reported (STMF_EINVAL)."""
    st = inputs.to_storage(np.ones((300, 64)), "bf16", device="cuda")
    idx = torch.tensor([0, 5, 300, 7], device="cuda")   # 300 is outside [0, p)
    f, _, _ = stmf.fg_sampled(st, idx, 3, torch.ones(2, dtype=torch.float64, device="cuda"),
                              torch.ones((2, 64), dtype=torch.float64, device="cuda").T)
    torch.cuda.synchronize()
    assert stmf.default_context().device_status() == 1   # STMF_EINVAL
    assert np.isfinite(f.item())


def test_adam_matches_oracle_schedule(stmf):
    """FP64 samples: the device Adam takes the oracle's steps (same sampled rows), through the
    learning-rate drop and the stop."""
    n, p, r, d = 20, 5000, 3, 3
    data = inputs.gmm(n, p, r, 0.1, seed=41, weights="equal")
    st = inputs.to_storage(data["V"], "f64", device="cuda")
    V = data["V"].T
    lam0, A0 = inputs.random_model(n, r, seed=42, lam="equal")
    g = np.random.default_rng(43)
    sample_idx = g.integers(0, p, size=(3000, 50))
    est_idx = g.integers(0, p, size=500)
    ref = stochastic.adam(V, lam0, A0, d, sample_idx, est_idx, epoch=20)
    lam = torch.tensor(lam0, device="cuda")
    A = torch.tensor(A0.T.copy(), device="cuda").T
    out = stmf.adam(st, d, lam, A, torch.tensor(sample_idx, device="cuda"),
                    torch.tensor(est_idx, device="cuda"), epoch=20)
    assert out["status"] == 0
    assert out["epochs"] == ref["epochs"]
    assert out["f_est"] == pytest.approx(ref["f_est"], rel=1e-9, abs=1e-14)
    x = np.concatenate([lam.cpu().numpy(), A.cpu().numpy().reshape(-1, order="F")])
    xr = np.concatenate([ref["lam"], ref["A"].reshape(-1, order="F")])
    assert rel(x, xr) < 1e-8


@pytest.mark.parametrize("dtype,n,p,r_hat", [("f64", 30, 7000, 5), ("f32", 100, 20000, 10),
                                             ("bf16", 256, 9000, 16), ("e4m3", 64, 3000, 3),
                                             ("bf16", 200, 30001, 12), ("e4m3", 256, 20000, 16),
                                             ("bf16", 40, 130, 1)])
def test_rrf_start_parity(stmf, dtype, n, p, r_hat):
    """eq. rrf with the test matrix drawn on the device from Philox4x32-10 (same draws as the
    oracle's generator). FP64 samples: FP64 draws and sums (1e-12). Other samples: the draws in
    FP32 (BF16/E4M3 with n <= 256 and r_hat <= 16 on the tensor cores, W = the drawn rows as a
    BF16 hi/lo pair; the rest on the CUDA cores with FP64 folds), within 1e-5 of the oracle's
    FP64 start; ragged tiles and a single column included."""
    from oracle import philox, rrf
    data = inputs.gmm(n, p, 4, 0.1, seed=p)
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    bits = inputs.storage_bits(st)
    if dtype == "bf16":
        Vd = formats.decode_bf16(bits)
    elif dtype == "e4m3":
        Vd = formats.dequantize_e4m3(bits, st["scale"].cpu().numpy())
    else:
        Vd = np.asarray(bits, dtype=np.float64)
    seed = 0x1234ABCD5678 + p
    ref = rrf.rrf_start(Vd.T, philox.gaussian_test_matrix(p, r_hat, seed))
    A0 = stmf.rrf_start(st, r_hat, seed).cpu().numpy()
    tol = 1e-12 if dtype == "f64" else 1e-5
    assert rel(A0, ref) < tol, rel(A0, ref)
    assert np.allclose(np.linalg.norm(A0, axis=0), 1.0, atol=1e-13)
