"""Sample-sharded evaluation across two CPU ranks (gloo): the orchestration of
paper_1911_03813_gb300.sharded (partial -> all-reduce -> finish) with the oracle's pieces
standing in for the device steps equals the oracle on all samples (no GPU needed)."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    from paper_1911_03813_gb300 import inputs, sharded
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        n, p, r, d = 12, 1001, 3, 4
        data = inputs.gmm(n, p, r, 0.1, seed=5)
        lam, A = inputs.random_model(n, r, seed=6)
        lo, hi = sharded.shard_bounds(p, world, rank)
        V_local = data["V"][lo:hi]

        def partial(V, nu, p_total, d_, lam_, A_):
            Y = oracle.implicit.ttsv_matrix(np.full(V.shape[0], 1.0 / p_total), V.T, A_, d_)
            return torch.from_numpy(np.concatenate([np.einsum("ij,ij->j", A_, Y),
                                                    Y.reshape(-1, order="F")]))

        def finish(yw, n_, d_, lam_, A_, alpha):
            Y = yw.numpy()[r:].reshape(n_, r, order="F")
            return oracle.implicit.model_terms(Y, lam_, A_, d_, alpha=alpha)

        f, gl, GA = sharded.fg_sharded(V_local, d, lam, A, p, n, alpha=0.0, partial=partial,
                                       finish=finish)
        f_ref, gl_ref, GA_ref = oracle.fg_implicit(None, data["V"].T, lam, A, d)
        q.put((rank, abs(f - f_ref) / abs(f_ref),
               float(np.linalg.norm(GA - GA_ref) / np.linalg.norm(GA_ref)),
               float(np.linalg.norm(gl - gl_ref) / np.linalg.norm(gl_ref))))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_evaluation_matches_oracle():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for pr in procs:
        pr.start()
    results = [q.get(timeout=120) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, ef, eG, el in results:
        assert ef < 1e-12 and eG < 1e-12 and el < 1e-12, (rank, ef, eG, el)


def test_shard_bounds_partition():
    from paper_1911_03813_gb300 import sharded
    for p, world in [(10, 3), (1001, 2), (7, 8), (2 ** 24, 8)]:
        spans = [sharded.shard_bounds(p, world, k) for k in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == p
        assert all(spans[k][1] == spans[k + 1][0] for k in range(world - 1))
        sizes = [b - a for a, b in spans]
        assert max(sizes) - min(sizes) <= 1
