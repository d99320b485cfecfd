"""A database sharded by rows: partial responses of disjoint row blocks,
summed by cwpir_sum_responses_device, equal the answer over all rows bit
for bit (the answer is linear in the rows: Eq. baseline-pir, Sec. 2.3).
The shards run one after the other on one GPU, as separate databases; no
kernel waits on another."""
import numpy as np
import pytest

from paper_2202_07569_gb300.shard import ShardedDatabase, shard_rows
from tests.workloads import T, Client, database

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2202_07569_gb300 import build

    build.build()


@pytest.mark.parametrize("N,L,n,k,m,plen,world", [
    (4096, 2, 61, 2, 12, 4096, 3),          # one plaintext per row, ragged shards
    (8192, 4, 40, 3, 8, 2 * 8192 + 77, 4),  # rows of three plaintexts
    (4096, 2, 30, 2, 9, 4096, 5),           # 6 rows per shard
])
def test_shard_partials_sum_to_full_answer(N, L, n, k, m, plen, world):
    import torch

    from paper_2202_07569_gb300 import binding as B

    cl = Client(N, L, seed=200 + world)
    ctx = cl.context()
    items, cw, _ = database(n, plen, T if N == 4096 else 1 << 16, k, m, seed=210 + world)
    target = n - 3
    query = cl.query(cw[target], m, 0)
    full = ctx.load_db(items, cw, m)
    want = ctx.answer(full, query)
    assert np.array_equal(want, cl.O.answer(items, cw, m, query, cl.rlk))
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream()
    d_query = torch.from_numpy(query.view(np.int64)).to(dev)
    shape = ctx.resp_shape(full)
    s = shape[0] if len(shape) == 4 else 1
    parts = torch.zeros((world,) + shape, dtype=torch.int64, device=dev)
    for r in range(world):
        lo, hi = shard_rows(n, world, r)
        db = ctx.load_db(items[lo:hi], cw[lo:hi], m)
        ctx.answer_device(db, d_query.data_ptr(), parts[r].data_ptr(), 0, st.cuda_stream)
        torch.cuda.synchronize()
        ctx.free_db(db)
    out = torch.empty(shape, dtype=torch.int64, device=dev)
    for _ in range(2):  # a second call gives the same sum
        ctx.sum_responses_device(world, s, parts.data_ptr(), out.data_ptr(), st.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want)
    # the all-reduce form: the element-wise u64 sum of the partials (what one
    # SUM collective over the ranks leaves), reduced modulo each q_j
    sums = parts.sum(dim=0)  # int64 wraps like the u64 sum; here no wrap occurs
    red = torch.empty(shape, dtype=torch.int64, device=dev)
    ctx.reduce_responses_device(s, sums.data_ptr(), red.data_ptr(), st.cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(red.cpu().numpy().view(np.uint64), want)
    ctx.reduce_responses_device(s, sums.data_ptr(), sums.data_ptr(), st.cuda_stream)  # in place
    torch.cuda.synchronize()
    assert np.array_equal(sums.cpu().numpy().view(np.uint64), want)
    # no partial alone is the answer
    for r in range(world):
        assert not np.array_equal(parts[r].cpu().numpy().view(np.uint64), want)
    mu, budget = cl.decrypt(got if s == 1 else got[0])
    assert budget > 0 and np.array_equal(mu[:min(N, plen)], items[target][:min(N, plen)])
    # argument checks
    for cnt, ss in [(0, s), (world, 0), (world, 257)]:  # 257 > CWPIR_MAX_PLAINTEXTS
        with pytest.raises(B.CwpirError):
            ctx.sum_responses_device(cnt, ss, parts.data_ptr(), out.data_ptr(), st.cuda_stream)
    with pytest.raises(B.CwpirError):
        ctx.sum_responses_device(world, s, 0, out.data_ptr(), st.cuda_stream)
    ctx.close()


def test_sharded_database_without_process_group_is_the_plain_answer():
    """ShardedDatabase on one rank (no process group): one shard holding
    every row, a gather of one partial, the same response as cwpir_answer."""
    import torch

    cl = Client(4096, 2, seed=230)
    ctx = cl.context()
    items, cw, _ = database(50, 4096, T, 2, 11, seed=231)
    query = cl.query(cw[9], 11, 0)
    sh = ShardedDatabase(ctx, items, cw, 11)
    assert (sh.rank, sh.world, sh.lo, sh.hi) == (0, 1, 0, 50)
    d_query = torch.from_numpy(query.view(np.int64)).cuda()
    out = torch.empty(ctx.ct_shape, dtype=torch.int64, device="cuda")
    sh.answer_device(d_query, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, ctx.answer(sh.db, query))
    assert np.array_equal(got, cl.O.answer(items, cw, 11, query, cl.rlk))
    out.zero_()
    sh.answer_device(d_query, out, exchange="allreduce")
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint64), got)
    sh.close()
    ctx.close()
