"""A database sharded by rows over the ranks of a process group.

Constant-weight PIR answers with r = sum over rows i of sel_i * DB_i mod Q
(Eq. baseline-pir, Sec. 2.3; the Inner Product of Sec. 3.3.3).  Rows are
independent and the sum is exact ring arithmetic, so each rank (one GPU)
holds a contiguous block of the rows with their own codewords, answers the
query over them, and the one exchange step is the modular sum of the
partial responses: an all-gather of one response per rank, then
``cwpir_sum_responses_device`` on the gathered block.  The result is bit
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

    def answer_device(self, d_query, d_resp, c: int = 0, stream=None):
        """Answer the query (device tensor [h][2][L][N], int64 view of the
        residues) over the whole database into d_resp ([s][2][L][N] or
        [2][L][N], device, int64 view).  Every rank of the group must call
        this with the same query; the result is on every rank."""
        import torch

        st = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            partial = torch.zeros(self.resp_shape, dtype=torch.int64, device=d_resp.device)
            if self.db is not None:
                self.ctx.answer_device(self.db, d_query.data_ptr(), partial.data_ptr(), c,
                                       st.cuda_stream)
            gathered = gather_partials(partial, self.group)
            s = self.resp_shape[0] if len(self.resp_shape) == 4 else 1
            self.ctx.sum_responses_device(self.world, s, gathered.data_ptr(), d_resp.data_ptr(),
                                          st.cuda_stream)
        return d_resp

    def close(self):
        if self.db is not None:
            self.ctx.free_db(self.db)
            self.db = None
