"""Batched answering (configuration 4's pattern): several queries share every
launch, optionally replayed from a captured CUDA graph.  Each response must
be bit-identical to the query answered alone, and to the oracle."""
import numpy as np
import pytest

import oracle
from paper_2202_07569_gb300 import synthetic as syn
from tests.workloads import CONFIGS, T, Client, database

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2202_07569_gb300 import build

    build.build()


@pytest.mark.parametrize("graph", [0, 1])
def test_batch_equals_single_and_oracle_index(graph):
    from paper_2202_07569_gb300 import binding as B

    cl = Client(8192, 4, seed=51)  # depth 2 needs more than two primes
    ctx = cl.context()
    n, k, m = 90, 3, 12  # k = 3: shared first level plus a carried leaf
    items, cw, _ = database(n, 700, T, k, m, seed=52)
    db = ctx.load_db(items, cw, m)
    targets = [0, 17, 89, 44, 17]
    queries = np.stack([cl.query(cw[t], m, 0, stream=60 + i) for i, t in enumerate(targets)])
    ctx.set_option(B.OPT_USE_GRAPH, graph)
    for rep in range(2):  # the second call replays the graph
        got = ctx.answer_batch(db, queries)
        for i, t in enumerate(targets):
            assert np.array_equal(got[i], ctx.answer(db, queries[i])), (rep, i)
    for i in (0, 2):
        assert np.array_equal(got[i], cl.O.answer(items, cw, m, queries[i], cl.rlk))
        mu, budget = cl.decrypt(got[i])
        want = np.zeros(8192, np.uint32)
        want[:700] = items[targets[i]]
        assert np.array_equal(mu, want) and budget > 0
    ctx.close()


@pytest.mark.parametrize("graph", [0, 1])
def test_batch_keyword_compressed_queries(graph):
    from paper_2202_07569_gb300 import binding as B

    cl = Client(8192, 4, seed=53, c_max=3)
    ctx = cl.context()
    n, k, m, c = 40, 4, 12, 3  # h = 2 ciphertexts per query
    st = syn.Stream(54)
    ids = np.array(sorted(set(st.below(495, 120).tolist())))[:n]
    items = syn.payload(st, len(ids), 64, 1 << 16)
    cw = np.stack([oracle.map_perfect(int(x), m, k) for x in ids])
    db = ctx.load_db(items, cw, m)
    absent = next(v for v in range(495) if v not in set(ids.tolist()))
    words = [oracle.map_perfect(int(ids[3]), m, k), oracle.map_perfect(absent, m, k),
             oracle.map_perfect(int(ids[30]), m, k)]
    queries = np.stack([cl.query(w, m, c, stream=70 + i) for i, w in enumerate(words)])
    ctx.set_option(B.OPT_USE_GRAPH, graph)
    got = ctx.answer_batch(db, queries, c)
    got = ctx.answer_batch(db, queries, c)
    for i in range(3):
        assert np.array_equal(got[i], ctx.answer(db, queries[i], c))
    assert np.array_equal(got[1], cl.O.answer(items, cw, m, queries[1], cl.rlk, c=c,
                                              gkeys=cl.gkeys))
    mu, _ = cl.decrypt(got[1])
    assert not mu.any()
    mu, _ = cl.decrypt(got[2])
    assert np.array_equal(mu[:64], items[30])
    ctx.close()


def test_batch_full_size_c2_graph_and_autotune():
    """Four queries against the full configuration-2 database in one graph:
    each response equals the query answered alone."""
    import torch

    from paper_2202_07569_gb300 import binding as B

    cfg = CONFIGS["c2"]
    cl = Client(cfg["N"], cfg["L"], seed=cfg["seed"])
    ctx = cl.context()
    items, cw, _ = database(cfg["n"], cfg["plen"], cfg["bound"], cfg["k"], cfg["m"],
                            cfg["seed"] + 1)
    db = ctx.load_db(items, cw, cfg["m"])
    targets = syn.Stream(cfg["seed"] + 5).below(cfg["n"], 4).tolist()
    queries = np.stack([cl.query(cw[t], cfg["m"], 0, stream=80 + i)
                        for i, t in enumerate(targets)])
    ctx.set_option(B.OPT_USE_GRAPH, 1)
    got = ctx.answer_batch(db, queries)
    for i, t in enumerate(targets):
        assert np.array_equal(got[i], ctx.answer(db, queries[i]))
        mu, budget = cl.decrypt(got[i])
        assert np.array_equal(mu, items[t]) and budget > 0
    dq = torch.from_numpy(queries.view(np.int64)).cuda()
    dr = torch.empty((4,) + ctx.ct_shape, dtype=torch.int64, device="cuda")
    best, ms = ctx.autotune(db, 4, dq.data_ptr(), dr.data_ptr(), [256, 0])
    assert best in (256, 0) and ms > 0
    ctx.answer_batch_device(db, 4, dq.data_ptr(), dr.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(dr.cpu().numpy().view(np.uint64), got)
    ctx.close()


@pytest.mark.parametrize("graph", [0, 1])
def test_multi_database_batch_equals_alone(graph):
    """Queries of three databases over two contexts (N = 4096 and N = 8192,
    k = 2, 3 and a compressed keyword query) in one forked launch sequence,
    one item answered two queries at a time: every response equals the
    query answered alone, on two calls in a row (the second replays the
    graph), and one equals the oracle's."""
    import torch

    from paper_2202_07569_gb300 import binding as B

    ca, cb = Client(4096, 2, seed=121), Client(8192, 4, seed=122, c_max=2)
    xa, xb = ca.context(), cb.context()
    ia, cwa, _ = database(70, 300, T, 2, 13, seed=123)
    ib, cwb, _ = database(90, 500, T, 3, 12, seed=124)
    ik, cwk, _ = database(40, 200, T, 4, 12, seed=125)
    dba, dbb, dbk = xa.load_db(ia, cwa, 13), xb.load_db(ib, cwb, 12), xb.load_db(ik, cwk, 12)
    specs = [(xa, dba, 0, 4, 2, ca, cwa, 13), (xb, dbb, 0, 3, 0, cb, cwb, 12),
             (xb, dbk, 2, 2, 0, cb, cwk, 12)]
    qs, alone = [], []
    for j, (ctx, db, c, nq, _, cl, cw, m) in enumerate(specs):
        q = np.stack([cl.query(cw[(11 * i + 3 * j) % len(cw)], m, c, stream=130 + 10 * j + i)
                      for i in range(nq)])
        qs.append(q)
        alone.append(np.stack([ctx.answer(db, q[i], c) for i in range(nq)]))
    assert np.array_equal(alone[0][1], ca.O.answer(ia, cwa, 13, qs[0][1], ca.rlk))
    mb = B.Multi([(ctx, db, c, nq, nqc) for ctx, db, c, nq, nqc, *_ in specs])
    dq = [torch.from_numpy(q.view(np.int64)).cuda() for q in qs]
    dr = [torch.zeros(a.shape, dtype=torch.int64, device="cuda") for a in alone]
    st = torch.cuda.current_stream()
    for rep in range(2):
        for r in dr:
            r.zero_()
        mb.answer_device([t.data_ptr() for t in dq], [t.data_ptr() for t in dr], graph,
                         st.cuda_stream)
        assert mb.status(st.cuda_stream) == 0
        for j in range(3):
            assert np.array_equal(dr[j].cpu().numpy().view(np.uint64), alone[j]), (rep, j)
    assert mb.stats()["mults"] > 0
    mb.close()
    xa.close()
    xb.close()
