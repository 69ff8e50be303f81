"""Implicit evaluation of Sec. 3: Alg. 2 (fg_implicit) and ||X||^2 from Lemma 3.4.

Test infrastructure only (see the package docstring). FP64 NumPy; the sum over samples is
taken in chunks of columns only to bound host memory, which changes no arithmetic step of the
algorithm (Y is a sum over samples, eq. Y).

Orientation follows the paper: V is n x p (one sample per column), A is n x r, nu has p
positive entries (Sec. 3 allows any positive weights).
"""

import numpy as np

DEFAULT_CHUNK = 1 << 16


def _as_f64(x):
    return np.asarray(x, dtype=np.float64)


def _columns(V, c0, c1):
    """Columns c0..c1 of V as FP64 (V may be any real dtype, or a callable that returns the
    FP64 block of columns [c0, c1), used for inputs too large to hold in FP64 at once)."""
    if callable(V):
        return _as_f64(V(c0, c1))
    return _as_f64(V[:, c0:c1])


def ttsv_matrix(nu, V, A, d, p=None, chunk=DEFAULT_CHUNK):
    """Y = V D_nu [V^T A]^{d-1} (Lemma 3.3, eq. Y). Column j of Y is X a_j^{d-1}."""
    A = _as_f64(A)
    if p is None:
        p = V.shape[1]
    Y = np.zeros(A.shape)
    for c0 in range(0, p, chunk):
        c1 = min(p, c0 + chunk)
        Vc = _columns(V, c0, c1)
        nuc = np.full(c1 - c0, 1.0 / p) if nu is None else _as_f64(nu[c0:c1])
        Zc = Vc.T @ A                           # inner products v_l^T a_j
        Y += Vc @ (nuc[:, None] * Zc ** (d - 1))
    return Y


def fg_implicit(nu, V, lam, A, d, alpha=0.0, p=None, chunk=DEFAULT_CHUNK, return_parts=False):
    """Alg. 2 (fg_implicit, Sec. 3.4) in FP64.

    nu: p weights, or None for the paper's default 1/p. V: n x p (or a callable, see _columns,
    with p given). lam: r weights. A: n x r. alpha: the constant ||X||^2, or 0 for the shifted
    objective.

    Returns (f, g_lambda, G_A), and with return_parts=True also a dict of the intermediate
    quantities Y, w, B, C, u (for parity checks of the GPU path's pieces)."""
    Y = ttsv_matrix(nu, V, _as_f64(A), d, p=p, chunk=chunk)  # eq. Y
    return model_terms(Y, lam, A, d, alpha=alpha, return_parts=return_parts)


def model_terms(Y, lam, A, d, alpha=0.0, return_parts=False):
    """The steps of Alg. 2 after Y: w, B, C, u, then f, g_lambda and G_A."""
    lam = _as_f64(lam)
    A = _as_f64(A)
    w = np.einsum("ij,ij->j", A, Y)                         # w_j = a_j^T y_j
    B = A.T @ A
    C = B ** (d - 1)                                        # element-wise power
    u = (B * C) @ lam                                       # lambda^T u = ||M||^2
    f = alpha + lam @ u - 2.0 * (w @ lam)
    g_lam = -2.0 * (w - u)                                  # eq. gradl
    G_A = -2.0 * d * (Y - A @ np.diag(lam) @ C) @ np.diag(lam)   # eq. gradb
    if return_parts:
        return float(f), g_lam, G_A, dict(Y=Y, w=w, B=B, C=C, u=u)
    return float(f), g_lam, G_A


def norm_m(lam, A, d):
    """||M||^2 = lam^T [A^T A]^d lam (Lemma 3.4)."""
    lam = _as_f64(lam)
    A = _as_f64(A)
    return float(lam @ ((A.T @ A) ** d) @ lam)


def norm_x(nu, V, d, p=None, chunk=4096):
    """||X||^2 = nu^T (V^T V)^d nu: Lemma 3.4 applied to X (Sec. 3.3), O(n p^2).

    Taken block by block over pairs of column chunks so the p x p matrix is never held."""
    if p is None:
        p = V.shape[1]
    total = 0.0
    for i0 in range(0, p, chunk):
        i1 = min(p, i0 + chunk)
        Vi = _columns(V, i0, i1)
        nui = np.full(i1 - i0, 1.0 / p) if nu is None else _as_f64(nu[i0:i1])
        for k0 in range(0, p, chunk):
            k1 = min(p, k0 + chunk)
            Vk = _columns(V, k0, k1)
            nuk = np.full(k1 - k0, 1.0 / p) if nu is None else _as_f64(nu[k0:k1])
            total += float(nui @ ((Vi.T @ Vk) ** d) @ nuk)
    return total


def relative_error(f, alpha):
    """||X - M|| / ||X|| from the implicit objective: sqrt(max(f, 0) / alpha), with f computed
    with alpha = ||X||^2 (Sec. 4.2 obtains the error from the data alone through Sec. 3.3's
    terms; this is that reading)."""
    return float(np.sqrt(max(f, 0.0) / alpha))
