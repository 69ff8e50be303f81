"""Continuously batched fits through stmf_server_* (-m gpu).

Checks: a request's result is bitwise the same alone and in a mix of concurrent requests of
uneven (n, p, r, d); it also equals stmf_fit from the same start; admission keeps the admitted
footprint within the budget while requests queue; cancellation; invalid and non-finite requests
report per ticket; fits overlap on the device.
"""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1911_03813_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stmf():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_03813_gb300 import stmf as s
    torch.cuda.set_device(0)
    return s


def host_request(n, p, r, d, sigma, seed, starts, dtype="bf16"):
    data = inputs.gmm(n, p, r, sigma, seed=seed, weights="dirichlet")
    st = inputs.to_storage(data["V"], dtype, device="cpu")
    arr = st["data"]
    if dtype == "bf16":
        arr = arr.view(torch.int16).numpy()
    else:
        arr = arr.numpy()
    V = dict(data=arr, n=n, dtype=dtype)
    x0 = []
    for k in range(starts):
        lam0, A0 = inputs.random_model(n, r, seed=seed * 10 + k, lam="equal")
        x0.append(np.concatenate([lam0, A0.reshape(-1, order="F")]))
    return V, np.array(x0), data


def test_alone_equals_mix_and_stmf_fit(stmf):
    n, p, r, d = 48, 30000, 4, 3
    V0, x0, _ = host_request(n, p, r, d, 0.05, seed=1, starts=2)
    opts = dict(pgtol=1e-7, factr=0.0, max_evals=300, alpha_mode=0, chunk=8)
    lam_a = torch.empty(r, dtype=torch.float64, device="cuda")
    A_a = torch.empty(n * r, dtype=torch.float64, device="cuda")
    with stmf.Server(max_fits=8, n_max=128, r_max=16) as srv:
        t = srv.submit(V0, d, x0, lam_out=lam_a, A_out=A_a, **opts)
        alone = srv.poll(t)
    assert alone["state"] == 0, alone
    lam_m = torch.empty_like(lam_a)
    A_m = torch.empty_like(A_a)
    rng = np.random.default_rng(5)
    with stmf.Server(max_fits=12, n_max=128, r_max=16) as srv:
        others = []
        for k in range(6):   # a burst of uneven requests first
            nk = int(rng.integers(8, 129))
            Vk, xk, _ = host_request(nk, int(rng.integers(1000, 60000)), int(rng.integers(1, 9)),
                                     int(rng.integers(3, 5)), 0.05, seed=100 + k, starts=2)
            others.append(srv.submit(Vk, 3, xk, **opts))
        t = srv.submit(V0, d, x0, lam_out=lam_m, A_out=A_m, **opts)
        time.sleep(0.01)
        for k in range(4):   # more arrive while the mix runs
            nk = int(rng.integers(8, 129))
            Vk, xk, _ = host_request(nk, int(rng.integers(1000, 60000)), int(rng.integers(1, 9)),
                                     4, 0.05, seed=200 + k, starts=1)
            others.append(srv.submit(Vk, 4, xk, **opts))
        mix = srv.poll(t)
        for o in others:
            assert srv.poll(o)["state"] == 0
        st = srv.stats()
    assert mix["state"] == 0
    assert mix["f"] == alone["f"] and mix["best_start"] == alone["best_start"]
    assert torch.equal(lam_m, lam_a) and torch.equal(A_m, A_a)
    assert st["completed"] == 11
    # the same start through stmf_fit (its own context, with the slots' launch shape) gives the
    # same iterate, bit for bit
    b = alone["best_start"]
    st_dev = inputs.to_storage(_decode(V0), "bf16", device="cuda")
    lam = torch.tensor(x0[b][:r], device="cuda")
    A = torch.tensor(x0[b][r:], device="cuda").reshape(r, n).T   # column-major n x r view
    ctx = stmf.Context()
    ctx.set_pass_tiles(stmf.SERVER_PASS_TILES)
    res = stmf.fit(st_dev, None, d, lam, A, ctx=ctx, **opts)
    ctx.close()
    assert res["f"] == alone["f"]
    assert torch.equal(lam, lam_a)


def _decode(V):
    from oracle import formats
    return formats.decode_bf16(V["data"].view(np.uint16))[:, : V["n"]]


def test_admission_by_memory_and_overlap(stmf):
    n, p, r, d = 64, 200000, 4, 3
    reqs = [host_request(n, p, r, d, 0.05, seed=300 + k, starts=1) for k in range(8)]
    opts = dict(pgtol=1e-7, factr=0.0, max_evals=120, alpha_mode=0, chunk=8)
    one = p * n * 2 + 2048      # samples copy + start vector (rounded up)
    with _server_with_room(stmf, 3 * one) as srv:
        tickets = [srv.submit(V, d, x0, **opts) for V, x0, _ in reqs]
        results = [srv.poll(t) for t in tickets]
        s = srv.stats()
    assert all(r_["state"] == 0 for r_ in results)
    assert s["peak_bytes_in_use"] <= 3 * one + 4096   # the budget admitted at most 3 at once
    assert s["peak_active_fits"] >= 2                  # fits ran side by side
    assert s["peak_active_fits"] <= 3
    assert max(r_["t_admit"] for r_ in results) > min(r_["t_done"] for r_ in results)  # queued


def _server_with_room(stmf, room):
    probe = stmf.Server(max_fits=8, n_max=64, r_max=4, mem_budget=64 << 30)
    slot_bytes = probe.stats()["slot_bytes"]
    probe.close()
    return stmf.Server(max_fits=8, n_max=64, r_max=4, mem_budget=slot_bytes + room)


def test_cancel_invalid_and_nonfinite(stmf):
    n, p, r, d = 32, 50000, 3, 3
    V, x0, _ = host_request(n, p, r, d, 0.05, seed=7, starts=1)
    with stmf.Server(max_fits=4, n_max=64, r_max=8) as srv:
        # a blocker holds every slot; the request behind it is cancelled while queued
        Vb, xb, _ = host_request(n, 400000, r, d, 0.05, seed=8, starts=4)
        blocker = srv.submit(Vb, d, xb, pgtol=0.0, factr=0.0, max_evals=50000, alpha_mode=0)
        t = srv.submit(V, d, x0, pgtol=1e-6, max_evals=200, alpha_mode=0)
        srv.cancel(t)
        assert srv.poll(t)["state"] == 7          # STMF_ECANCELLED before admission
        srv.cancel(blocker)
        assert srv.poll(blocker)["state"] in (0, 7)   # cancelled while running (or finished)
        with pytest.raises(stmf.StmfError):
            srv.submit(V, 9, x0)                   # d out of range
        bad = dict(V)
        arr = V["data"].copy()
        arr[5, 0] = 0x7FC0                         # a BF16 NaN in one sample
        bad["data"] = arr
        t2 = srv.submit(bad, d, x0, pgtol=1e-7, max_evals=200, alpha_mode=0)
        res = srv.poll(t2)
        assert res["state"] == 0 and res["stop"] == 6   # finished: non-finite objective
        t3 = srv.submit(V, d, x0, pgtol=1e-6, max_evals=200, alpha_mode=0)
        assert srv.poll(t3)["state"] == 0               # the server keeps serving
        with pytest.raises(stmf.StmfError):
            srv.poll(t3)                                # a delivered result releases its ticket
