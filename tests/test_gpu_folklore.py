"""Folklore PIR in the same engine (Sec. 4): the query is the ell encrypted
bits of the index, the server forms the leaves (1 - x[i], x[i]) and selects
each row by the plain folklore operator (Eq. folklore-plain-eq).  Every
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


def bits_query(cl, y, ell, stream):
    return cl.query(np.array([i for i in range(ell) if (y >> i) & 1], np.uint16), ell, 0,
                    stream=stream)


def oracle_answer(cl, items, n, ell, query):
    cw = np.stack([oracle.folklore_codeword(i, ell) for i in range(n)])
    return cl.O.answer(items, cw, 2 * ell, cl.O.folklore_leaves(query), cl.rlk)


@pytest.mark.parametrize("N,L,ell,n", [(8192, 4, 4, 13), (16384, 7, 6, 40)])
def test_folklore_answer_bit_exact(N, L, ell, n):
    cl = Client(N, L, seed=180 + ell)
    ctx = cl.context()
    items, _, _ = database(n, 500, 1 << 16, 1, n, seed=181 + ell)
    db = ctx.load_db_folklore(items, ell)
    assert ctx.query_cts(db) == ell
    for target in (0, n - 1):
        q = bits_query(cl, target, ell, 190 + target)
        got = ctx.answer(db, q)
        assert np.array_equal(got, oracle_answer(cl, items, n, ell, q))
        mu, budget = cl.decrypt(got)
        want = np.zeros(N, np.uint32)
        want[:500] = items[target]
        assert np.array_equal(mu, want) and budget > 0
    ctx.close()


@pytest.mark.parametrize("graph", [0, 1])
def test_folklore_batch_selection_and_serving(graph):
    from paper_2202_07569_gb300 import binding as B

    N, L, ell, n = 8192, 4, 4, 16
    cl = Client(N, L, seed=200)
    ctx = cl.context()
    items, _, _ = database(n, 300, 1 << 16, 1, n, seed=201)
    db = ctx.load_db_folklore(items, ell)
    targets = [3, 15, 0]
    queries = np.stack([bits_query(cl, y, ell, 210 + i) for i, y in enumerate(targets)])
    ctx.set_option(B.OPT_USE_GRAPH, graph)
    got = ctx.answer_batch(db, queries)
    got = ctx.answer_batch(db, queries)
    for i, y in enumerate(targets):
        assert np.array_equal(got[i], ctx.answer(db, queries[i]))
    assert np.array_equal(got[1], oracle_answer(cl, items, n, ell, queries[1]))
    # selection entries: the folklore operator per row, decrypting to [x == y]
    rows = np.array([3, 4, 15], np.uint64)
    sel = ctx.selection(db, queries[0], rows)
    leaves = cl.O.folklore_leaves(queries[0])
    for r, s in zip(rows, sel):
        assert np.array_equal(s, cl.O.selection(leaves, oracle.folklore_codeword(int(r), ell),
                                                cl.rlk))
        mu, _ = cl.decrypt(s)
        assert mu[0] == (1 if int(r) == targets[0] else 0) and not mu[1:].any()
    if graph:
        srv = B.Server([(ctx, db, 0)], max_batch=2)
        tk = [srv.submit(0, q) for q in queries]
        for i, t in enumerate(tk):
            status, resp, _ = srv.wait(t, 0, timeout=300)
            assert status == 1 and np.array_equal(resp, got[i])
        srv.close()
    with pytest.raises(B.CwpirError) as ei:
        ctx.answer(db, queries[0], 2)  # folklore queries are not compressed
    assert ei.value.code == -1
    with pytest.raises(B.CwpirError):
        ctx.load_db_folklore(items, 3)  # 16 rows need 4 bits
    ctx.close()
