"""Sec. 5: stochastic evaluation from sampled columns (Lemma 5.1) and the Adam schedule used
with it.

Test infrastructure only (see the package docstring). Every random draw (the sampled column
indices of each iteration) is an input, drawn by the caller.
"""

import numpy as np

from .implicit import fg_implicit


def fg_sampled(V, idx, lam, A, d, alpha=0.0):
    """Alg. 2 on the stochastic Kruskal tensor of Lemma 5.1: the s columns V[:, idx] (drawn with
    replacement) with weights nu_tilde = 1/s."""
    Vs = np.asarray(V, dtype=np.float64)[:, np.asarray(idx)]
    s = Vs.shape[1]
    return fg_implicit(np.full(s, 1.0 / s), Vs, lam, A, d, alpha=alpha)


def adam(V, lam0, A0, d, sample_idx, est_idx, lr0=1e-2, lr1=1e-3, epoch=100,
         beta1=0.9, beta2=0.999, eps=1e-8, max_epochs=None):
    """Adam (Kingma & Ba, 2015) on x = (lambda, A) with the schedule of Sec. 5:

    * each iteration draws its own column sample (row t of `sample_idx`, s indices) and steps
      on Lemma 5.1's stochastic gradient;
    * after every `epoch` iterations the (shifted) objective is estimated on the fixed columns
      `est_idx` (Sec. 5 uses 1,000);
    * the first time the estimate fails to decrease, the learning rate drops from lr0 to lr1 and
      the state returns to the end of the prior epoch; the second time, the method stops and
      returns the prior epoch's iterate.

    Reading where Sec. 5 is silent: going back to the prior epoch's iterate restores that
    epoch's Adam moments and step counter as well as (lambda, A).

    Returns dict(lam, A, f_est, epochs, trace)."""
    lam = np.array(lam0, dtype=np.float64)
    A = np.array(A0, dtype=np.float64)
    n, r = A.shape
    x = np.concatenate([lam, A.reshape(-1, order="F")])
    mom1 = np.zeros_like(x)
    mom2 = np.zeros_like(x)
    t = 0

    def unpack(z):
        return z[:r], z[r:].reshape(n, r, order="F")

    def estimate(z):
        lz, Az = unpack(z)
        return fg_sampled(V, est_idx, lz, Az, d)[0]

    f_prev = estimate(x)
    saved = (x.copy(), mom1.copy(), mom2.copy(), t)
    lr = lr0
    drops = 0
    trace = [f_prev]
    it = 0
    epochs = 0
    total = sample_idx.shape[0]
    while it + epoch <= total:
        for _ in range(epoch):
            lz, Az = unpack(x)
            _, gl, gA = fg_sampled(V, sample_idx[it], lz, Az, d)
            g = np.concatenate([gl, gA.reshape(-1, order="F")])
            t += 1
            mom1 = beta1 * mom1 + (1.0 - beta1) * g
            mom2 = beta2 * mom2 + (1.0 - beta2) * g * g
            mhat = mom1 / (1.0 - beta1 ** t)
            vhat = mom2 / (1.0 - beta2 ** t)
            x = x - lr * mhat / (np.sqrt(vhat) + eps)
            it += 1
        epochs += 1
        f_now = estimate(x)
        trace.append(f_now)
        if f_now < f_prev:
            f_prev = f_now
            saved = (x.copy(), mom1.copy(), mom2.copy(), t)
        else:
            x, mom1, mom2, t = saved[0].copy(), saved[1].copy(), saved[2].copy(), saved[3]
            drops += 1
            if drops == 2:
                break
            lr = lr1
        if max_epochs is not None and epochs >= max_epochs:
            break
    lz, Az = unpack(x)
    return dict(lam=lz, A=Az, f_est=f_prev, epochs=epochs, trace=trace)
