"""||X||^2 from the distinct entries of the symmetric moment tensor (stmf_norm_x_method, method
"compressed"; -m gpu), against the oracle's Gram form and its explicitly formed X.

Tolerances: 1e-12 for FP64 samples; 2e-6 otherwise (FP32 products and sums over 512 samples,
FP64 beyond; a sum of squares, so no cancellation).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import explicit, formats  # noqa: E402
from paper_1911_03813_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "e4m3"])
@pytest.mark.parametrize("n,p,d,weights", [
    (10, 1000, 3, None),      # the small FP64 configuration's shape
    (1, 77, 4, None),
    (7, 33, 2, "nonuniform"),
    (33, 1001, 3, "nonuniform"),
    (100, 5003, 3, None),
    (65, 300, 4, None),
    (12, 257, 6, "nonuniform"),
    (130, 99, 2, None),
])
def test_compressed_norm_x_parity(stmf, dtype, n, p, d, weights):
    data = inputs.gmm(n, p, 4, 0.3, seed=n * p + d)
    st = inputs.to_storage(data["V"], dtype, device="cuda")
    nu = inputs.positive_weights(p, seed=p) if weights else None
    nu_t = None if nu is None else torch.tensor(nu, device="cuda")
    ref = oracle.norm_x(nu, decoded(st).T, d)
    got = stmf.norm_x(st, nu_t, d, method="compressed").item()
    gram = stmf.norm_x(st, nu_t, d, method="gram").item()
    torch.cuda.synchronize()
    assert stmf.default_context().device_status() == 0
    tol = 1e-12 if dtype == "f64" else 2e-6
    assert abs(got - ref) <= tol * abs(ref), (got, ref)
    assert abs(gram - ref) <= (1e-12 if dtype == "f64" else 2e-6) * abs(ref)


def test_auto_takes_the_cheaper_method(stmf):
    """Large p with small n d: the compressed tensor is chosen (and agrees with the Gram form);
    the BF16 benchmark slice keeps the tensor-core Gram pass."""
    data = inputs.gmm(20, 200000, 4, 0.1, seed=5)
    st = inputs.to_storage(data["V"], "f32", device="cuda")
    a = stmf.norm_x(st, None, 3).item()
    c = stmf.norm_x(st, None, 3, method="compressed").item()
    g = stmf.norm_x(st, None, 3, method="gram").item()
    torch.cuda.synchronize()
    assert a == c
    assert abs(g - c) <= 2e-6 * abs(c)


def test_compressed_full_size_fp32_d3(stmf):
    """n = 100, p = 2.5e6 FP32 Gaussian mixture, d = 3 (the FP32 workload at scale): against the
    oracle's explicitly formed X."""
    n, p, d = 100, 2500000, 3
    st = inputs.gmm_device(n, p, 10, 0.1, seed=2500, device="cuda", out_dtype="f32")
    got = stmf.norm_x(st, None, d).item()
    torch.cuda.synchronize()
    V = st["data"][:, :n].double().cpu().numpy().T
    ref = explicit.norm_x_explicit(None, V, d, chunk=8192)
    assert abs(got - ref) <= 2e-6 * abs(ref), (got, ref)


def test_compressed_limits(stmf):
    """C(n + d - 2, d - 1) past the prefix-table cap is refused before any work."""
    data = inputs.gmm(256, 100, 3, 0.1, seed=1)
    st = inputs.to_storage(data["V"], "f32", device="cuda")
    with pytest.raises(stmf.StmfError):
        stmf.norm_x(st, None, 5, method="compressed")


def test_prefix_table_survives_host_calls(stmf):
    """A context's host-buffer evaluations (stmf_fg_host) grow their small device buffers without
    touching the compressed-norm prefix table: alpha before and after host calls of growing r
    agrees bit for bit, and the context is destroyed cleanly afterwards."""
    ctx = stmf.Context()
    n, p, d = 40, 5000, 3
    data = inputs.gmm(n, p, 4, 0.1, seed=11)
    st = inputs.to_storage(data["V"], "f32", device="cuda")
    a0 = stmf.norm_x(st, None, d, method="compressed", ctx=ctx).item()
    host = inputs.to_storage(data["V"], "f32", device="cpu")
    for r in (2, 8, 16):
        lam, A = inputs.random_model(n, r, seed=r)
        f, _, _ = stmf.fg_host(host, None, d, lam, A, alpha=a0, ctx=ctx)
        assert np.isfinite(f)
    a1 = stmf.norm_x(st, None, d, method="compressed", ctx=ctx).item()
    torch.cuda.synchronize()
    assert a1 == a0
    assert ctx.device_status() == 0
    ctx.close()
