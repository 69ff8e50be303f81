"""Sample-sharded evaluation of Alg. 2 across ranks.

Every sum over samples in Alg. 2 (eq. Y, Lemma 3.5) splits over disjoint shards of V. Each rank
holds its shard, computes its partial [w; vec(Y)] (stmf_fg_partial, with nu = 1 / p_total), the
partials are summed by one all-reduce of r + n r FP64 values, and every rank finishes the model terms
(stmf_fg_finish) on the summed values. The partial and finish steps are parameters so that the
same orchestration can be exercised with other implementations of the two steps.
"""

import torch

from . import stmf


def _all_reduce_sum(t, group=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def fg_sharded(V_local, d, lam, A, p_total, n, alpha=None, nu_local=None, group=None,
               partial=None, finish=None, all_reduce=None):
    """f, g_lambda, G_A of Alg. 2 over the union of all ranks' shards.

    V_local: this rank's samples; p_total: samples over all ranks; n: features.
    partial(V, nu, p_total, d, lam, A) -> yw tensor; finish(yw, n, d, lam, A, alpha) -> outputs;
    all_reduce(t, group) sums t in place across ranks (defaults: the CUDA library and
    torch.distributed)."""
    partial = partial or stmf.fg_partial
    finish = finish or stmf.fg_finish
    all_reduce = all_reduce or _all_reduce_sum
    yw = partial(V_local, nu_local, p_total, d, lam, A)
    all_reduce(yw, group)
    return finish(yw, n, d, lam, A, alpha)


def shard_bounds(p_total, world, rank):
    """Contiguous balanced shard [lo, hi) of rank `rank` among `world` ranks."""
    base, extra = divmod(p_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)
