"""Explicit (n^d) tensor algebra of Sec. 2, in FP64, element by element.

Test infrastructure only (see the package docstring). Every routine here forms the full
n^d array, so it is meant for tiny n (n^d up to about 1e6 entries).

Orientation follows the paper: V is n x p (one sample per column), A is n x r.
"""

import numpy as np


def outer_power(a, d):
    """a^{(x)d}: the d-way symmetric outer product of eq. outer_product (Sec. 2.4).

    Entry (i_1, ..., i_d) is prod_k a[i_k]. Built by repeated outer products."""
    a = np.asarray(a, dtype=np.float64)
    t = a.copy()
    for _ in range(d - 1):
        t = np.multiply.outer(t, a)
    return t


def kruskal_full(weights, F, d):
    """sum_j weights[j] * F[:, j]^{(x)d}: a symmetric Kruskal tensor (eq. symmDecomp, Sec. 2.5)
    formed explicitly. With (weights, F) = (lambda, A) this is M of eq. cp_element; with
    (nu, V) it is the moment tensor X of eq. tensorX."""
    F = np.asarray(F, dtype=np.float64)
    n, r = F.shape
    t = np.zeros((n,) * d)
    for j in range(r):
        t += float(weights[j]) * outer_power(F[:, j], d)
    return t


def moment_tensor(nu, V, d):
    """X = sum_l nu_l v_l^{(x)d} (eq. tensorX; eq. moment_tensor_element when nu = 1/p)."""
    return kruskal_full(nu, V, d)


def inner(X, Y):
    """<X, Y> = sum over all n^d entries of x_i * y_i (eq. tensorIP, Sec. 2.1)."""
    return float(np.sum(np.asarray(X) * np.asarray(Y)))


def ttsv_all(X, a):
    """X a^d: contract every mode of X with a (eq. ExpXbd, Sec. 2.3). Returns a scalar."""
    t = np.asarray(X, dtype=np.float64)
    for _ in range(t.ndim):
        t = np.tensordot(t, a, axes=([t.ndim - 1], [0]))
    return float(t)


def ttsv_but_one(X, a):
    """X a^{d-1}: contract all modes but the first with a (eq. ExpXbdd). Returns an n-vector."""
    t = np.asarray(X, dtype=np.float64)
    for _ in range(t.ndim - 1):
        t = np.tensordot(t, a, axes=([t.ndim - 1], [0]))
    return t


def f_bruteforce(X, lam, A):
    """f = ||X - M||^2 with M formed explicitly (eq. optFunc)."""
    d = X.ndim
    M = kruskal_full(lam, A, d)
    return float(np.sum((X - M) ** 2))


def grad_bruteforce(X, lam, A):
    """Gradient of ||X - M||^2 by direct differentiation of the n^d sum.

    d/d lambda_j ||X - M||^2 = -2 <X - M, a_j^{(x)d}>, and since X - M is symmetric,
    d/d a_j ||X - M||^2 = -2 d lambda_j (X - M) a_j^{d-1}. These are the definitions that
    eqs. gradl and gradb rewrite with Lemma 3.1; no lemma is used here."""
    d = X.ndim
    A = np.asarray(A, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    R = X - kruskal_full(lam, A, d)
    r = A.shape[1]
    g_lam = np.empty(r)
    G_A = np.empty_like(A)
    for j in range(r):
        g_lam[j] = -2.0 * inner(R, outer_power(A[:, j], d))
        G_A[:, j] = -2.0 * d * lam[j] * ttsv_but_one(R, A[:, j])
    return g_lam, G_A


def fg_explicit(X, lam, A, alpha=0.0):
    """Alg. 1 (fg_explicit, Sec. 3.4): the TTSVs y_j = X a_j^{d-1} are taken on the explicit X.

    Returns (f, g_lambda, G_A)."""
    d = X.ndim
    A = np.asarray(A, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    n, r = A.shape
    Y = np.empty((n, r))
    for j in range(r):                      # y_j = X a_j^{d-1}
        Y[:, j] = ttsv_but_one(X, A[:, j])
    w = np.array([A[:, j] @ Y[:, j] for j in range(r)])   # w_j = a_j^T y_j
    B = A.T @ A
    C = B ** (d - 1)                        # element-wise power
    u = (B * C) @ lam                       # lambda^T u = ||M||^2
    f = alpha + lam @ u - 2.0 * (w @ lam)
    g_lam = -2.0 * (w - u)                  # eq. gradl
    G_A = -2.0 * d * (Y - A @ np.diag(lam) @ C) @ np.diag(lam)   # eq. gradb
    return float(f), g_lam, G_A


def norm_x_explicit(nu, V, d, chunk=4096):
    """||X||^2 = <X, X> with X = sum_l nu_l v_l^{(x)d} formed explicitly (eq. tensorX), as the
    n^(d-1) x n matrix sum_l nu_l vec(v_l^{(x)(d-1)}) v_l^T accumulated over chunks of samples
    (V: n x p; nu: p weights or None for 1/p). Memory n^d; for d up to 4 at moderate n."""
    V = np.asarray(V, dtype=np.float64)
    n, p = V.shape
    w = np.full(p, 1.0 / p) if nu is None else np.asarray(nu, dtype=np.float64)
    X = np.zeros((n ** (d - 1), n))
    for c0 in range(0, p, chunk):
        c1 = min(p, c0 + chunk)
        Vc = V[:, c0:c1].T                      # samples x n
        K = Vc.copy()
        for _ in range(d - 2):                  # rows: v^{(x)(d-1)} flattened
            K = (K[:, :, None] * Vc[:, None, :]).reshape(c1 - c0, -1)
        X += K.T @ (w[c0:c1, None] * Vc)
    return float(np.sum(X * X))
