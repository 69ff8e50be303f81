"""stmf_fg_noalloc against stmf_fg and the oracle (run with -m gpu; collected last on purpose).

stmf_fg_noalloc serves callers that cannot allocate device memory (for example code that runs
inside another runtime's memory arena); it keeps its scratch in a fixed array of the library's
device globals instead of a context workspace. These checks call it through the C ABI twice in
a row on the same inputs and compare both results with stmf_fg within the parity tolerances of
the other GPU tests, so they also show that a call leaves nothing behind that spoils the next;
one result per case is also compared with the FP64 oracle on the values the GPU reads. A
non-finite model must reach the caller's status word and make every output NaN.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import formats  # noqa: E402
from paper_1911_03813_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16": 5e-6, "e4m3": 5e-6}


@pytest.fixture(scope="module")
def stmf():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_03813_gb300 import stmf as s
    torch.cuda.set_device(0)
    return s


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def decoded(st):
    bits = inputs.storage_bits(st)
    if st["dtype"] == "bf16":
        return formats.decode_bf16(bits)
    if st["dtype"] == "e4m3":
        return formats.dequantize_e4m3(bits, st["scale"].cpu().numpy())
    return np.asarray(bits, dtype=np.float64)


@pytest.mark.parametrize("dtype,n,p,r,d", [("bf16", 256, 70000, 16, 4), ("f32", 100, 20000, 10, 3),
                                           ("bf16", 33, 130, 5, 3), ("f32", 256, 9000, 64, 2),
                                           ("e4m3", 128, 40000, 12, 4)])
def test_noalloc_matches_fg_twice(stmf, dtype, n, p, r, d):
    data = inputs.gmm(n, p, min(r, 8), 0.1, seed=7 * n + r)
    lam, A = inputs.random_model(n, r, seed=r + d)
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    lam_t = torch.tensor(lam, device="cuda")
    A_t = torch.tensor(np.ascontiguousarray(A.T), device="cuda").T
    alpha = torch.tensor([0.25], dtype=torch.float64, device="cuda")
    f0, g0, G0 = stmf.fg(st, None, d, lam_t, A_t, alpha=alpha)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    tol = TOL[dtype]
    for _ in range(2):
        f1, g1, G1 = stmf.fg_noalloc(st, None, d, lam_t, A_t, alpha=alpha, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert abs(f1.item() - f0.item()) <= tol * max(1.0, abs(f0.item()))
        assert rel(g1, g0) <= tol
        assert rel(G1, G0) <= tol
    # the FP64 oracle on the values the GPU reads (BF16 codes widened, E4M3 codes times scales)
    f_o, g_o, G_o, parts = oracle.fg_implicit(None, decoded(st).T, lam, A, d, alpha=0.25,
                                              return_parts=True)
    S = 0.25 + abs(parts["u"] @ lam) + 2 * abs(parts["w"] @ lam)
    assert abs(f1.item() - f_o) <= tol * S
    assert np.linalg.norm(g1.cpu().numpy() - g_o) <= tol * np.linalg.norm(g_o)
    assert np.linalg.norm(G1.cpu().numpy() - G_o) <= tol * np.linalg.norm(G_o)


def test_noalloc_reports_device_errors(stmf):
    """A NaN in lambda is a host-side input that makes f non-finite: the caller's status word
    receives STMF_ENONFINITE and every output is NaN; with no status word the outputs are NaN
    too, and the next call (whose internal word starts clear) is unaffected."""
    n, p, r, d = 40, 3000, 4, 3
    data = inputs.gmm(n, p, 4, 0.1, seed=12)
    lam, A = inputs.random_model(n, r, seed=13)
    st = inputs.to_storage(data["V"], "bf16", device="cuda")
    A_t = torch.tensor(np.ascontiguousarray(A.T), device="cuda").T
    bad = lam.copy()
    bad[1] = np.nan
    bad_t = torch.tensor(bad, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    f, g, G = stmf.fg_noalloc(st, None, d, bad_t, A_t, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 5           # STMF_ENONFINITE
    assert torch.isnan(f).all()
    # the word is the caller's: while it still holds the error, outputs stay NaN
    f, g, G = stmf.fg_noalloc(st, None, d, torch.tensor(lam, device="cuda"), A_t, status=status)
    torch.cuda.synchronize()
    assert torch.isnan(f).all() and torch.isnan(g).all() and torch.isnan(G).all()
    status.zero_()
    f, g, G = stmf.fg_noalloc(st, None, d, torch.tensor(lam, device="cuda"), A_t, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and torch.isfinite(G).all()
    # internal status word: NaN outputs for the bad model, a clean result for the next call
    f, g, G = stmf.fg_noalloc(st, None, d, bad_t, A_t)
    torch.cuda.synchronize()
    assert torch.isnan(f).all() and torch.isnan(G).all()
    f, g, G = stmf.fg_noalloc(st, None, d, torch.tensor(lam, device="cuda"), A_t)
    torch.cuda.synchronize()
    assert torch.isfinite(f).all() and torch.isfinite(G).all()
    # a row-major A is refused by the binding before any call
    with pytest.raises(ValueError):
        stmf.fg_noalloc(st, None, d, torch.tensor(lam, device="cuda"),
                        torch.tensor(A, device="cuda"))


def test_noalloc_internal_status_and_limits(stmf):
    n, p, r, d = 64, 5000, 8, 3
    data = inputs.gmm(n, p, 8, 0.1, seed=3)
    lam, A = inputs.random_model(n, r, seed=4)
    st = inputs.to_storage(data["V"], "bf16", device="cuda")
    lam_t = torch.tensor(lam, device="cuda")
    A_t = torch.tensor(np.ascontiguousarray(A.T), device="cuda").T
    f0, g0, G0 = stmf.fg(st, None, d, lam_t, A_t)
    f1, g1, G1 = stmf.fg_noalloc(st, None, d, lam_t, A_t)      # status=NULL: internal word
    f2, g2, G2 = stmf.fg_noalloc(st, None, d, lam_t, A_t)
    torch.cuda.synchronize()
    assert rel(G1, G0) <= TOL["bf16"] and rel(G2, G0) <= TOL["bf16"]
    assert torch.equal(G1, G2)
    # requests beyond the limits are refused before any work
    desc, keep = stmf.as_samples(st)
    L = stmf.lib()
    big = torch.ones(65, dtype=torch.float64, device="cuda")
    Abig = torch.ones((65, n), dtype=torch.float64, device="cuda")
    out = [torch.empty(k, dtype=torch.float64, device="cuda") for k in (1, 65, 65 * n)]
    rc = L.stmf_fg_noalloc(ctypes.byref(desc), None, 3, 65, ctypes.c_void_p(big.data_ptr()),
                           ctypes.c_void_p(Abig.data_ptr()), None,
                           *[ctypes.c_void_p(t.data_ptr()) for t in out], None, None)
    assert rc == 1  # STMF_EINVAL
    rc = L.stmf_fg_noalloc(ctypes.byref(desc), None, 9, r, ctypes.c_void_p(lam_t.data_ptr()),
                           ctypes.c_void_p(A_t.data_ptr()), None,
                           *[ctypes.c_void_p(t.data_ptr()) for t in out], None, None)
    assert rc == 1
