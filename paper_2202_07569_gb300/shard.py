"""A database sharded by rows over the ranks of a process group.

Constant-weight PIR answers with r = sum over rows i of sel_i * DB_i mod Q
(Eq. baseline-pir, Sec. 2.3; the Inner Product of Sec. 3.3.3).  Rows are
independent and the sum is exact ring arithmetic, so each rank (one GPU)
holds a contiguous block of the rows with their own codewords, answers the
query over them, and the one exchange step is the modular sum of the
partial responses.  Two forms of it: an all-gather of one response per
rank, then ``cwpir_sum_responses_device`` on the gathered block; or one
all-reduce (SUM) of the u64 residues, exact while at most 1023 ranks add
values below 2^54 (the sum stays below 2^64; the int64 sum of the
collective wraps like the unsigned one), then
``cwpir_reduce_responses_device`` modulo each q_j.  Either result is bit
identical to answering over all rows on one GPU.

torch.distributed carries the partials (NCCL for device tensors, gloo for
host tensors); the arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np


def shard_rows(n: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [lo, hi) of rank `rank` out of `world`: contiguous blocks whose
    sizes differ by at most one, in rank order, covering [0, n) once."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad shard request n={n} world={world} rank={rank}")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def partial_shape(payload_len: int, N: int, L: int) -> tuple:
    """Shape of one rank's partial response: [2][L][N], or [s][2][L][N] for
    rows of s = ceil(payload_len / N) > 1 plaintexts (Sec. 3.3.1).  It
    depends on the database alone, so a rank with no rows gathers the same
    shape as the others."""
    s = max(1, -(-int(payload_len) // int(N)))
    return ((s,) if s > 1 else ()) + (2, int(L), int(N))


def _group_info(group):
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def gather_partials(partial, group=None):
    """All-gather one partial response per rank: returns a tensor
    [world, *partial.shape] on partial's device, rank order.  Without an
    initialised process group the result is partial[None]."""
    import torch
    import torch.distributed as dist

    rank, world = _group_info(group)
    if world == 1:
        return partial.unsqueeze(0)
    parts = [torch.empty_like(partial) for _ in range(world)]
    dist.all_gather(parts, partial.contiguous(), group=group)
    return torch.stack(parts)


MAX_ALLREDUCE_RANKS = 1023


def allreduce_partials(partial, group=None):
    """Sums one partial response per rank in place (SUM over int64 views of
    the u64 residues) and returns it: element-wise sums below 2^64 for at
    most MAX_ALLREDUCE_RANKS ranks, to be reduced modulo each q_j."""
    import torch.distributed as dist

    rank, world = _group_info(group)
    if world > MAX_ALLREDUCE_RANKS:
        raise ValueError(f"{world} ranks: the u64 sum of the residues could wrap")
    if world > 1:
        dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    return partial


class ShardedDatabase:
    """This rank's block of a database and the sharded answer.

    items: [n][payload_len] (every rank passes the whole database, or at
    least its block at the same row indices), codewords: [n][k]; the rank
    loads rows shard_rows(n, world, rank) into ctx.
    """

    def __init__(self, ctx, items, codewords, m: int, group=None):
        self.ctx = ctx
        self.group = group
        self.rank, self.world = _group_info(group)
        n = len(codewords)
        self.lo, self.hi = shard_rows(n, self.world, self.rank)
        self.db = None
        if self.hi > self.lo:
            self.db = ctx.load_db(np.ascontiguousarray(items[self.lo:self.hi]),
                                  np.ascontiguousarray(codewords[self.lo:self.hi]), m)
        plen = int(np.shape(items)[1]) if np.ndim(items) == 2 else 0
        self.resp_shape = partial_shape(plen, ctx.N, ctx.L)

    def answer_device(self, d_query, d_resp, c: int = 0, stream=None,
                      exchange: str = "allgather"):
        """Answer the query (device tensor [h][2][L][N], int64 view of the
        residues) over the whole database into d_resp ([s][2][L][N] or
        [2][L][N], device, int64 view).  Every rank of the group must call
        this with the same query; the result is on every rank.  exchange:
        "allgather" (gather the partials, sum them modulo q_j) or
        "allreduce" (one SUM collective, then the reduction modulo q_j)."""
        import torch

        st = stream if stream is not None else torch.cuda.current_stream()
        s = self.resp_shape[0] if len(self.resp_shape) == 4 else 1
        with torch.cuda.stream(st):
            partial = torch.zeros(self.resp_shape, dtype=torch.int64, device=d_resp.device)
            if self.db is not None:
                self.ctx.answer_device(self.db, d_query.data_ptr(), partial.data_ptr(), c,
                                       st.cuda_stream)
            if exchange == "allreduce":
                summed = allreduce_partials(partial, self.group)
                self.ctx.reduce_responses_device(s, summed.data_ptr(), d_resp.data_ptr(),
                                                 st.cuda_stream)
            elif exchange == "allgather":
                gathered = gather_partials(partial, self.group)
                self.ctx.sum_responses_device(self.world, s, gathered.data_ptr(),
                                              d_resp.data_ptr(), st.cuda_stream)
            else:
                raise ValueError(f"unknown exchange {exchange!r}")
        return d_resp

    def close(self):
        if self.db is not None:
            self.ctx.free_db(self.db)
            self.db = None
