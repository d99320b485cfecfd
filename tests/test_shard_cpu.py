"""Row sharding of a database over the ranks of a process group (the
multi-GPU path), on the CPU: two gloo ranks each answer over their rows
with the oracle, gather the partial responses through the package's
exchange helper, and the modular sum of the partials is the oracle's
answer over all rows (the answer is linear in the rows: Eq. baseline-pir,
Sec. 2.3, and the Inner Product of Sec. 3.3.3)."""
import os
import socket

import numpy as np
import pytest

from paper_2202_07569_gb300.shard import shard_rows

WORLD = 2
N, L, ROWS, K, M = 1024, 2, 24, 2, 8  # C(8, 2) = 28 >= 24 rows
TARGET = 17


@pytest.mark.parametrize("n", [0, 1, 5, 24, 64, 65537])
@pytest.mark.parametrize("world", [1, 2, 3, 7, 8])
def test_shard_rows_cover_every_row_once(n, world):
    spans = [shard_rows(n, world, r) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    for (lo, hi), (lo2, _) in zip(spans, spans[1:]):
        assert hi == lo2 and lo <= hi
    sizes = [hi - lo for lo, hi in spans]
    assert max(sizes) - min(sizes) <= 1


def test_partial_shape_depends_on_the_database_only():
    """Every rank, with or without rows, gathers partials of one shape:
    [2][L][N] for rows of one plaintext, [s][2][L][N] for s > 1."""
    from paper_2202_07569_gb300.shard import partial_shape

    assert partial_shape(0, 8192, 4) == (2, 4, 8192)
    assert partial_shape(8192, 8192, 4) == (2, 4, 8192)
    assert partial_shape(8193, 8192, 4) == (2, 2, 4, 8192)
    assert partial_shape(17 * 8192, 8192, 4) == (17, 2, 4, 8192)
    assert partial_shape(5000, 4096, 2) == (2, 2, 2, 4096)


def test_shard_rows_rejects_bad_ranks():
    for args in [(5, 0, 0), (5, 2, 2), (5, 2, -1), (-1, 2, 0)]:
        with pytest.raises(ValueError):
            shard_rows(*args)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, port: int, out_dir: str):
    import torch
    import torch.distributed as dist

    from paper_2202_07569_gb300.shard import gather_partials
    from tests.workloads import T, Client, database

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        cl = Client(N, L, seed=7)
        items, cw, _ = database(ROWS, N, T, K, M, seed=8)
        query = cl.query(cw[TARGET], M, 0)
        lo, hi = shard_rows(ROWS, WORLD, rank)
        partial = cl.O.answer(items[lo:hi], cw[lo:hi], M, query, cl.rlk)
        gathered = gather_partials(torch.from_numpy(partial.view(np.int64)))
        assert tuple(gathered.shape) == (WORLD,) + partial.shape
        np.save(os.path.join(out_dir, f"gathered{rank}.npy"), gathered.numpy().view(np.uint64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_of_partials_is_the_answer(tmp_path, orc):
    import torch.multiprocessing as mp

    from tests.workloads import T, Client, database

    mp.start_processes(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=WORLD,
                       join=True, start_method="spawn")
    cl = Client(N, L, seed=7)
    items, cw, _ = database(ROWS, N, T, K, M, seed=8)
    query = cl.query(cw[TARGET], M, 0)
    want = cl.O.answer(items, cw, M, query, cl.rlk)
    q = cl.q.reshape(1, L, 1)
    blocks = [np.load(tmp_path / f"gathered{r}.npy") for r in range(WORLD)]
    # every rank holds the same gathered block, in rank order
    assert np.array_equal(blocks[0], blocks[1])
    total = np.zeros_like(want)
    for part in blocks[0]:
        assert (part < q).all()
        total = (total + part) % q
    assert np.array_equal(total, want)
    # a rank's partial alone is not the answer: both shards contribute
    assert not np.array_equal(blocks[0][0], want) and not np.array_equal(blocks[0][1], want)
    mu, budget = cl.decrypt(total)
    assert np.array_equal(mu, items[TARGET]) and budget > 0


WORLD3, ROWS3 = 3, 2  # three ranks over two rows: rank 2 holds none


def _rank_main_allreduce(rank: int, port: int, out_dir: str):
    import torch
    import torch.distributed as dist

    from paper_2202_07569_gb300.shard import allreduce_partials
    from tests.workloads import T, Client, database

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD3)
    try:
        cl = Client(N, L, seed=9)
        items, cw, _ = database(ROWS3, N, T, K, M, seed=10)
        query = cl.query(cw[1], M, 0)
        lo, hi = shard_rows(ROWS3, WORLD3, rank)
        if hi > lo:
            partial = cl.O.answer(items[lo:hi], cw[lo:hi], M, query, cl.rlk)
        else:  # a rank without rows contributes zeros of the same shape
            partial = np.zeros((2, L, N), np.uint64)
        t = torch.from_numpy(partial.view(np.int64).copy())
        allreduce_partials(t)
        np.save(os.path.join(out_dir, f"summed{rank}.npy"), t.numpy().view(np.uint64))
        np.save(os.path.join(out_dir, f"span{rank}.npy"), np.array([lo, hi]))
    finally:
        dist.destroy_process_group()


def test_three_gloo_ranks_allreduce_with_an_empty_shard(tmp_path, orc):
    """The all-reduce form of the exchange over three ranks, one of them
    without rows: every rank holds the same element-wise sum, whose residues
    modulo each q_j are the oracle's answer over all rows."""
    import torch.multiprocessing as mp

    from tests.workloads import T, Client, database

    mp.start_processes(_rank_main_allreduce, args=(_free_port(), str(tmp_path)), nprocs=WORLD3,
                       join=True, start_method="spawn")
    spans = [tuple(np.load(tmp_path / f"span{r}.npy")) for r in range(WORLD3)]
    assert spans[2][0] == spans[2][1]  # the empty shard
    sums = [np.load(tmp_path / f"summed{r}.npy") for r in range(WORLD3)]
    assert all(np.array_equal(sums[0], x) for x in sums[1:])
    cl = Client(N, L, seed=9)
    items, cw, _ = database(ROWS3, N, T, K, M, seed=10)
    query = cl.query(cw[1], M, 0)
    want = cl.O.answer(items, cw, M, query, cl.rlk)
    q = cl.q.reshape(1, L, 1)
    assert np.array_equal(sums[0] % q, want)
    mu, budget = cl.decrypt(sums[0] % q)
    assert np.array_equal(mu, items[1]) and budget > 0
