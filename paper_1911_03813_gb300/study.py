"""The Gaussian-mixture study of Sec. 4.2 on the GPU.

For each scenario (d, r, sigma): n = 500 features, r congruent unit means (pairwise cosine 0.5),
p = 250 r samples with equal counts, sigma^2 I noise. For every r_hat in r-2 .. r+2 the fit runs
from `starts` randomized-range-finder starts (eq. rrf, lambda_0 = 1/r_hat) with pgtol = 1e-4, and
the start with the lowest final f is kept (the paper's best-of-ten). Reported per (scenario,
r_hat): the relative error sqrt(max(f, 0) / alpha) of the best fit (Sec. 4.2, from the implicit
terms with alpha = ||X||^2) and its score (eq. Score) against the true means. All fits of a
scenario are submitted at once to the continuously batched server, so they share the GPU.
"""

import time

import numpy as np

from . import inputs, stmf


def score(A_true, A):
    """eq. Score: the best one-to-one matching between the computed and the true component
    directions (unit-normalised columns), averaged |cosine| over the smaller set.

    The matching is found exactly by dynamic programming over subsets: with k columns on the
    smaller side and m on the larger (k <= m), best[S] is the largest sum of |cosines| that
    matches the first |S| small-side columns to the large-side set S, and
    best[S | {c}] = max(best[S] + C[|S|, c]) over c not in S. That is O(m 2^m) work, which suits
    the ranks of the study (m <= 16)."""
    U = np.asarray(A_true, dtype=np.float64)
    W = np.asarray(A, dtype=np.float64)
    U = U / np.linalg.norm(U, axis=0, keepdims=True)
    W = W / np.linalg.norm(W, axis=0, keepdims=True)
    C = np.abs(U.T @ W)
    if C.shape[0] > C.shape[1]:
        C = C.T                       # rows: the smaller set
    k, m = C.shape
    if m > 20:
        raise ValueError("score: at most 20 components per side")
    best = np.full(1 << m, -np.inf)
    best[0] = 0.0
    popcount = np.array([bin(S).count("1") for S in range(1 << m)])
    for S in range(1 << m):
        i = popcount[S]
        if i >= k or best[S] == -np.inf:
            continue
        for c in range(m):
            if not S & (1 << c):
                T = S | (1 << c)
                v = best[S] + C[i, c]
                if v > best[T]:
                    best[T] = v
    return float(best[popcount == k].max() / k)


def scenario(server, d, r, sigma, n=500, starts=10, dtype="f32", pgtol=1e-4, max_evals=20000,
             seed=0):
    """Submit every fit of one scenario and collect the best start per r_hat. Returns a list of
    dicts (d, r, sigma, r_hat, f, alpha, rel_error, score, evals, stop, seconds, and the best
    start's lam and A)."""
    import torch
    p = 250 * r
    data = inputs.gmm(n, p, r, sigma, seed=seed, weights="equal", means="congruent",
                      equal_counts=True)
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    tickets = []
    for r_hat in range(max(1, r - 2), r + 3):
        x0 = np.empty((starts, r_hat + n * r_hat))
        for k in range(starts):
            A0 = stmf.rrf_start(st, r_hat, seed=(seed << 20) + 97 * r_hat + k).cpu().numpy()
            x0[k, :r_hat] = 1.0 / r_hat
            x0[k, r_hat:] = A0.reshape(-1, order="F")
        lam = torch.empty(r_hat, dtype=torch.float64, device="cuda")
        A = torch.empty((r_hat, n), dtype=torch.float64, device="cuda").T
        t = server.submit(st, d, x0, lam_out=lam, A_out=A, pgtol=pgtol, max_evals=max_evals)
        tickets.append((r_hat, t, lam, A))
    rows = []
    for r_hat, t, lam, A in tickets:
        res = server.poll(t)
        torch.cuda.synchronize()
        if res["state"] != 0:
            raise stmf.StmfError(res["state"], "fit of the study scenario")
        rows.append(dict(d=d, r=r, sigma=sigma, r_hat=r_hat, f=res["f"], alpha=res["alpha"],
                         rel_error=float(np.sqrt(max(res["f"], 0.0) / res["alpha"])),
                         score=score(data["means"], A.cpu().numpy()),
                         evals=res["total_evals"], stop=res["stop"],
                         seconds=res["t_done"] - res["t_submit"],
                         lam=lam.cpu().numpy(), A=A.cpu().numpy()))
    return rows


def run(d_values=(3, 4), r_values=(3, 5, 10), sigmas=(1e-4, 1e-3, 1e-2, 1e-1), starts=10,
        dtype="f32", seed=0, max_fits=32, mem_budget=16 << 30):
    """The whole grid of the study; returns (rows, wall seconds)."""
    t0 = time.perf_counter()
    rows = []
    with stmf.Server(max_fits=max(max_fits, starts), n_max=500, r_max=max(r_values) + 2,
                     mem_budget=mem_budget) as srv:
        for d in d_values:
            for r in r_values:
                for k, sigma in enumerate(sigmas):
                    rows += scenario(srv, d, r, sigma, starts=starts, dtype=dtype,
                                     seed=seed + 1000 * d + 10 * r + k)
    return rows, time.perf_counter() - t0
