"""Rows of several plaintexts (Sec. 3.3.1 Setup, Sec. 3.3.3 inner product):
one selection vector, s inner products, s response ciphertexts.  Every
response is compared bit for bit with the oracle and decrypted."""
import numpy as np
import pytest

import oracle
from tests.workloads import T, Client, database

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2202_07569_gb300 import build

    build.build()


def _check_decrypts(cl, resp, row_payload):
    s = resp.shape[0]
    want = np.zeros(s * cl.N, np.uint32)
    want[:row_payload.size] = row_payload
    for p in range(s):
        mu, budget = cl.decrypt(resp[p])
        assert np.array_equal(mu, want[p * cl.N:(p + 1) * cl.N]) and budget > 0, p


@pytest.mark.parametrize("k,N,L,n,m,plen", [
    (2, 4096, 2, 50, 11, 2 * 4096 + 300),      # s = 3, last plaintext ragged
    (4, 8192, 4, 40, 9, 9 * 8192 - 5),         # s = 9: two plaintext chunks, shared pairs
    (1, 4096, 2, 20, 20, 3 * 4096),            # k = 1: the leaf is the selection entry
    (3, 8192, 4, 30, 8, 4 * 8192 + 1),         # s = 5, odd tree (carried leaf)
])
def test_multi_plaintext_answer_bit_exact(k, N, L, n, m, plen):
    cl = Client(N, L, seed=100 + k)
    ctx = cl.context()
    items, cw, _ = database(n, plen, T if N == 4096 else 1 << 16, k, m, seed=110 + k)
    db = ctx.load_db(items, cw, m)
    s = -(-plen // N)
    assert ctx.plaintexts(db) == s
    target = n // 3
    q = cl.query(cw[target], m, 0, stream=5)
    got = ctx.answer(db, q)
    assert got.shape == (s, 2, L, N)
    want = cl.O.answer(items, cw, m, q, cl.rlk)
    assert np.array_equal(got, want)
    _check_decrypts(cl, got, items[target])
    ctx.close()


@pytest.mark.parametrize("graph", [0, 1])
def test_multi_plaintext_batch_keyword_and_plain_mul(graph):
    """Batched compressed (keyword) queries against rows of 3 plaintexts:
    equal to the queries answered alone and to the oracle; PM by a row gives
    one product per plaintext."""
    from paper_2202_07569_gb300 import binding as B
    from paper_2202_07569_gb300 import synthetic as syn

    N, L, k, m, c = 8192, 4, 3, 12, 2
    cl = Client(N, L, seed=120, c_max=c)
    ctx = cl.context()
    st = syn.Stream(121)
    ids = np.array(sorted(set(st.below(220, 80).tolist())))[:24]
    plen = 2 * N + 77
    items = syn.payload(st, len(ids), plen, 1 << 16)
    cw = np.stack([oracle.map_perfect(int(x), m, k) for x in ids])
    db = ctx.load_db(items, cw, m)
    absent = next(v for v in range(220) if v not in set(ids.tolist()))
    words = [oracle.map_perfect(int(ids[4]), m, k), oracle.map_perfect(absent, m, k),
             oracle.map_perfect(int(ids[17]), m, k)]
    queries = np.stack([cl.query(w, m, c, stream=130 + i) for i, w in enumerate(words)])
    ctx.set_option(B.OPT_USE_GRAPH, graph)
    got = ctx.answer_batch(db, queries, c)
    got = ctx.answer_batch(db, queries, c)  # replay
    assert got.shape == (3, 3, 2, L, N)
    for i in range(3):
        assert np.array_equal(got[i], ctx.answer(db, queries[i], c))
    assert np.array_equal(got[0], cl.O.answer(items, cw, m, queries[0], cl.rlk, c=c,
                                              gkeys=cl.gkeys))
    _check_decrypts(cl, got[0], items[4])
    _check_decrypts(cl, got[1], np.zeros(0, np.uint32))
    _check_decrypts(cl, got[2], items[17])
    # PM of one ciphertext by every plaintext of row 5
    ct = queries[0][0]
    pm = ctx.plain_mul(db, 5, ct)
    assert pm.shape == (3, 2, L, N)
    chunks = np.zeros((3, N), np.uint32)
    chunks.reshape(-1)[:plen] = items[5]
    for p in range(3):
        assert np.array_equal(pm[p], cl.O.plain_mul(ct, chunks[p])), p
    ctx.close()


def test_multi_plaintext_too_many_partials_is_einval():
    """nq queries x s plaintexts beyond the multiplications per launch is
    refused with EINVAL, not truncated."""
    from paper_2202_07569_gb300 import binding as B

    cl = Client(4096, 2, seed=140)
    ctx = cl.context()
    items, cw, _ = database(40, 9 * 4096, T, 2, 10, seed=141)
    db = ctx.load_db(items, cw, 10)
    ctx.set_option(B.OPT_MAX_JOBS, 32)
    queries = np.stack([cl.query(cw[i], 10, 0, stream=150 + i) for i in range(4)])
    with pytest.raises(B.CwpirError) as ei:
        ctx.answer_batch(db, queries)  # 4 x 9 = 36 > 32
    assert ei.value.code == -1
    one = ctx.answer_batch(db, queries[:3])  # 27 <= 32
    assert np.array_equal(one[1], cl.O.answer(items, cw, 10, queries[1], cl.rlk))
    ctx.close()


def test_multi_plaintext_served():
    """A served target whose rows hold two plaintexts returns both."""
    from paper_2202_07569_gb300 import binding as B

    cl = Client(4096, 2, seed=160)
    ctx = cl.context()
    items, cw, _ = database(30, 4096 + 9, T, 2, 9, seed=161)
    db = ctx.load_db(items, cw, 9)
    qs = [cl.query(cw[i], 9, 0, stream=170 + i) for i in (2, 11, 29)]
    alone = [ctx.answer(db, q) for q in qs]
    srv = B.Server([(ctx, db, 0)], max_batch=4)
    tickets = [srv.submit(0, q) for q in qs]
    for tk, want in zip(tickets, alone):
        status, resp, _ = srv.wait(tk, 0, timeout=300)
        assert status == 1 and np.array_equal(resp, want)
    srv.close()
    assert np.array_equal(alone[0], cl.O.answer(items, cw, 9, qs[0], cl.rlk))
    ctx.close()
