"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module draws random numbers and converts storage formats; it holds none of the method's
arithmetic. Everything the tests feed to both the CUDA path and the oracle comes from here.

Workloads follow the paper's synthetic data:
  * uniform(0,1) samples (Sec. 4.1);
  * spherical Gaussian mixtures v_l = mu_{j(l)} + sigma * N(0, I) (Sec. 4.2), with unit-norm
    Gaussian means or congruent means (pairwise cosine 0.5, Sec. 4.2), mixture weights equal,
    Dirichlet(1) or given, and the component of each sample drawn from the weights.

Layout: V is returned SAMPLE-MAJOR, p x n (row l is sample v_l), which is the paper's n x p
matrix V stored column-major. Rows may be padded to a row stride `ld` so that each row starts on
a 16-byte boundary; the padding holds zeros.
"""

import numpy as np

try:  # torch is only needed for the device-side generators and the format conversions
    import torch
except ImportError:  # pragma: no cover
    torch = None

ELEM_BYTES = {"f64": 8, "f32": 4, "bf16": 2, "e4m3": 1}


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def padded_ld(n, dtype):
    """Smallest row stride >= n whose byte size is a multiple of 16."""
    per = 16 // ELEM_BYTES[dtype]
    return ((n + per - 1) // per) * per


def unit_gaussian_means(n, r, g):
    M = g.standard_normal((n, r))
    return M / np.linalg.norm(M, axis=0, keepdims=True)


def congruent_means(n, r, g, cos=0.5):
    """Unit-norm means with mu_i^T mu_j = cos for i != j: mu = Q L^T with Q (n x r) orthonormal
    and L L^T = (1 - cos) I + cos 1 1^T (Cholesky), so that mu^T mu = L L^T."""
    G = (1.0 - cos) * np.eye(r) + cos * np.ones((r, r))
    L = np.linalg.cholesky(G)
    Q, _ = np.linalg.qr(g.standard_normal((n, r)))
    return Q @ L.T


def mixture_weights(r, g, kind):
    if isinstance(kind, str):
        if kind == "equal":
            return np.full(r, 1.0 / r)
        if kind == "dirichlet":
            return g.dirichlet(np.ones(r))
        raise ValueError(kind)
    w = np.asarray(kind, dtype=np.float64)
    return w / w.sum()


def gmm(n, p, r, sigma, seed, weights="dirichlet", means="gaussian", equal_counts=False):
    """Gaussian-mixture samples. Returns dict(V = p x n FP64 sample-major, means = n x r,
    weights = r, labels = p)."""
    g = rng(seed)
    mu = congruent_means(n, r, g) if means == "congruent" else unit_gaussian_means(n, r, g)
    w = mixture_weights(r, g, weights)
    if equal_counts:
        labels = np.repeat(np.arange(r), p // r + 1)[:p]
        g.shuffle(labels)
    else:
        labels = g.choice(r, size=p, p=w)
    V = mu.T[labels] + sigma * g.standard_normal((p, n))
    return dict(V=V, means=mu, weights=w, labels=labels)


def uniform(n, p, seed):
    """Entries uniform on (0, 1), sample-major p x n (Sec. 4.1's timing data)."""
    return rng(seed).random((p, n))


def random_model(n, r, seed, lam="dirichlet"):
    """A start point: A with N(0,1) entries and unit-norm columns (Sec. 4.2's random start), and
    lambda = Dirichlet(1)/r-style positive weights, or 1/r each with lam="equal"."""
    g = rng(seed)
    A = unit_gaussian_means(n, r, g)
    if lam == "equal":
        l = np.full(r, 1.0 / r)
    else:
        l = g.dirichlet(np.ones(r))
    return l, A


def positive_weights(p, seed):
    """Non-uniform positive sample weights nu summing to 1."""
    w = rng(seed).random(p) + 0.5
    return w / w.sum()


def pad_rows(V, ld):
    """p x n -> p x ld with zero padding (host, NumPy)."""
    p, n = V.shape
    out = np.zeros((p, ld), dtype=V.dtype)
    out[:, :n] = V
    return out


# ----------------------------------------------------------------------------------------------
# storage-format conversions (torch): round to nearest even, as torch's casts do
# ----------------------------------------------------------------------------------------------

def to_storage(V, dtype, device="cpu"):
    """Convert p x n samples to the storage type, padded to a 16-byte row stride.

    Returns dict(data = torch tensor p x ld of the storage type, scale = per-sample FP32 scales
    for e4m3 (else None), n, ld). e4m3 uses s_l = max_i |v_il| / 448 (448 = largest finite
    e4m3), s_l = 1 for an all-zero sample, codes q_l = e4m3(v_l / s_l)."""
    Vt = torch.as_tensor(V).to(device)
    p, n = Vt.shape
    ld = padded_ld(n, dtype)
    scale = None
    if dtype == "f64":
        data = torch.zeros((p, ld), dtype=torch.float64, device=device)
        data[:, :n] = Vt.to(torch.float64)
    elif dtype == "f32":
        data = torch.zeros((p, ld), dtype=torch.float32, device=device)
        data[:, :n] = Vt.to(torch.float32)
    elif dtype == "bf16":
        data = torch.zeros((p, ld), dtype=torch.bfloat16, device=device)
        data[:, :n] = Vt.to(torch.bfloat16)
    elif dtype == "e4m3":
        V32 = Vt.to(torch.float32)
        amax = V32.abs().amax(dim=1)
        scale = torch.where(amax > 0, amax / 448.0, torch.ones_like(amax)).to(torch.float32)
        q = (V32 / scale[:, None]).clamp(-448.0, 448.0).to(torch.float8_e4m3fn)
        data = torch.zeros((p, ld), dtype=torch.float8_e4m3fn, device=device)
        data[:, :n] = q
    else:
        raise ValueError(dtype)
    return dict(data=data, scale=scale, n=n, ld=ld, dtype=dtype)


def storage_bits(st):
    """Raw bit patterns (NumPy) of a stored sample block, for the oracle's format decoders:
    uint16 for bf16, uint8 for e4m3, else the FP64/FP32 values themselves. Shape p x n."""
    data = st["data"][:, : st["n"]].detach().cpu()
    if st["dtype"] == "bf16":
        return data.view(torch.int16).numpy().view(np.uint16)
    if st["dtype"] == "e4m3":
        return data.view(torch.uint8).numpy()
    return data.numpy()


# ----------------------------------------------------------------------------------------------
# device-side generation for full-size workloads (torch Philox on the GPU)
# ----------------------------------------------------------------------------------------------

def gmm_device(n, p, r, sigma, seed, device, out_dtype="f32", weights="dirichlet",
               chunk=1 << 20):
    """Gaussian-mixture samples generated on the device in chunks, written straight into the
    storage type with a 16-byte row stride. Means and weights come from the host generator (so
    they match `gmm`'s draws for the same seed); labels and noise come from torch's device
    generator seeded with `seed`. Returns the to_storage dict plus means, weights."""
    g = rng(seed)
    mu = unit_gaussian_means(n, r, g)
    w = mixture_weights(r, g, weights)
    tg = torch.Generator(device=device)
    tg.manual_seed(int(seed))
    ld = padded_ld(n, out_dtype)
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16,
           "e4m3": torch.float8_e4m3fn}[out_dtype]
    data = torch.zeros((p, ld), dtype=tdt, device=device)
    scale = torch.empty(p, dtype=torch.float32, device=device) if out_dtype == "e4m3" else None
    muT = torch.as_tensor(mu.T, dtype=torch.float32, device=device)
    wt = torch.as_tensor(w, dtype=torch.float32, device=device)
    for c0 in range(0, p, chunk):
        c1 = min(p, c0 + chunk)
        lab = torch.multinomial(wt, c1 - c0, replacement=True, generator=tg)
        blk = muT[lab] + sigma * torch.randn((c1 - c0, n), generator=tg, device=device,
                                            dtype=torch.float32)
        if out_dtype == "e4m3":
            amax = blk.abs().amax(dim=1)
            s = torch.where(amax > 0, amax / 448.0, torch.ones_like(amax))
            scale[c0:c1] = s
            data[c0:c1, :n] = (blk / s[:, None]).clamp(-448.0, 448.0).to(tdt)
        else:
            data[c0:c1, :n] = blk.to(tdt)
    return dict(data=data, scale=scale, n=n, ld=ld, dtype=out_dtype, means=mu, weights=w)
