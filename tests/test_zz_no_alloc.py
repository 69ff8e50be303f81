"""stmf_fg_noalloc against stmf_fg (run with -m gpu; collected last on purpose).

stmf_fg_noalloc serves callers that cannot allocate device memory (for example code that runs
inside another runtime's memory arena); it keeps its scratch in a fixed array of the library's
device globals instead of a context workspace. These checks call it through the C ABI twice in
a row on the same inputs and compare both results with stmf_fg within the parity tolerances of
the other GPU tests, so they also show that a call leaves nothing behind that spoils the next.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1911_03813_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16": 4e-5}


@pytest.fixture(scope="module")
def stmf():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_03813_gb300 import stmf as s
    torch.cuda.set_device(0)
    return s


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("dtype,n,p,r,d", [("bf16", 256, 70000, 16, 4), ("f32", 100, 20000, 10, 3),
                                           ("bf16", 33, 130, 5, 3), ("f32", 256, 9000, 64, 2)])
def test_noalloc_matches_fg_twice(stmf, dtype, n, p, r, d):
    data = inputs.gmm(n, p, min(r, 8), 0.1, seed=7 * n + r)
    lam, A = inputs.random_model(n, r, seed=r + d)
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    lam_t = torch.tensor(lam, device="cuda")
    A_t = torch.tensor(np.ascontiguousarray(A.T), device="cuda").T
    alpha = torch.tensor([0.25], dtype=torch.float64, device="cuda")
    f0, g0, G0 = stmf.fg(st, None, d, lam_t, A_t, alpha=alpha)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        f1, g1, G1 = stmf.fg_noalloc(st, None, d, lam_t, A_t, alpha=alpha, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        tol = TOL[dtype]
        assert abs(f1.item() - f0.item()) <= tol * max(1.0, abs(f0.item()))
        assert rel(g1, g0) <= tol
        assert rel(G1, G0) <= tol


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
