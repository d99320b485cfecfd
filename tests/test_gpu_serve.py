"""Online serving (configuration 5's pattern): continuous batching over
resident databases of two parameter sets, several lanes per target.  Every
response must be the same as the query answered alone (and, for sampled
queries, the oracle's)."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2202_07569_gb300 import synthetic as syn
from tests.workloads import T, Client, database

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2202_07569_gb300 import build

    build.build()


def test_serving_mix_equals_alone_and_oracle():
    from paper_2202_07569_gb300 import binding as B

    ca = Client(4096, 2, seed=91)
    cb = Client(8192, 4, seed=92, c_max=2)
    xa, xb = ca.context(), cb.context()
    ia, cwa, _ = database(50, 300, T, 2, 12, seed=93)
    ib, cwb, _ = database(80, 500, T, 4, 12, seed=94)
    st = syn.Stream(95)
    kid = np.array(sorted(set(st.below(220, 90).tolist())))[:30]
    ik = syn.payload(st, len(kid), 200, 1 << 16)
    cwk = np.stack([oracle.map_perfect(int(x), 12, 3) for x in kid])
    dba, dbb = xa.load_db(ia, cwa, 12), xb.load_db(ib, cwb, 12)
    dbk = xb.load_db(ik, cwk, 12)
    targets = [(xa, dba, 0), (xb, dbb, 0), (xb, dbk, 2)]
    pools = []  # (target, query) pairs with their responses answered alone
    for i in range(30):
        t = i % 3
        if t == 0:
            q = ca.query(cwa[(7 * i) % 50], 12, 0, stream=200 + i)
        elif t == 1:
            q = cb.query(cwb[(5 * i) % 80], 12, 0, stream=300 + i)
        else:
            w = int(kid[i % 30]) if i % 2 else 219  # 219 is absent
            q = cb.query(oracle.map_perfect(w, 12, 3), 12, 2, stream=400 + i)
        ctx, db, c = targets[t]
        pools.append((t, q, ctx.answer(db, q, c)))
    # a few oracle checks of the alone-answers
    assert np.array_equal(pools[0][2], ca.O.answer(ia, cwa, 12, pools[0][1], ca.rlk))
    assert np.array_equal(pools[2][2], cb.O.answer(ik, cwk, 12, pools[2][1], cb.rlk, c=2,
                                                   gkeys=cb.gkeys))
    srv = B.Server(targets, max_batch=8, lanes_per_target=2)
    tickets = []
    lock = threading.Lock()

    def submit(lo, hi):
        for i in range(lo, hi):
            t, q, _ = pools[i]
            tk = srv.submit(t, q)
            with lock:
                tickets.append((i, tk))

    submit(0, 20)  # a burst ...
    th = threading.Thread(target=submit, args=(20, 30))  # ... and arrivals during it
    th.start()
    th.join()
    for i, tk in sorted(tickets):
        t = pools[i][0]
        status, resp, lat = srv.wait(tk, t, timeout=600)
        assert status == 1 and lat >= 0
        assert np.array_equal(resp, pools[i][2]), i
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == 30 and stats["max_batch_seen"] > 1
    xa.close()
    xb.close()


def test_serving_backpressure():
    from paper_2202_07569_gb300 import binding as B

    cb = Client(8192, 4, seed=96)
    xb = cb.context()
    ib, cwb, _ = database(200, 100, T, 4, 14, seed=97)
    db = xb.load_db(ib, cwb, 14)
    q = cb.query(cwb[3], 14, 0, stream=1)
    srv = B.Server([(xb, db, 0)], max_batch=2, max_pending=2)
    accepted, busy = [], 0
    for _ in range(6):
        try:
            accepted.append(srv.submit(0, q))
        except B.CwpirError as e:
            assert e.code == -6
            busy += 1
    assert busy >= 1 and len(accepted) >= 1
    for tk in accepted:
        status, resp, _ = srv.wait(tk, 0)
        assert status == 1
    assert srv.stats()["rejected_busy"] == busy
    srv.close()
    xb.close()


def test_request_arriving_mid_batch_completes_before_that_batch():
    """A request for another database that arrives while a long batch runs
    starts at once on its own lane: it completes before the batch it arrived
    during, and both give the responses of the queries answered alone."""
    from paper_2202_07569_gb300 import binding as B

    cl = Client(8192, 4, seed=98)
    ctx = cl.context()
    ibig, cwbig, _ = database(12000, 200, T, 4, 25, seed=99)
    ismall, cwsmall, _ = database(8, 200, T, 2, 5, seed=100)
    dbig, dsmall = ctx.load_db(ibig, cwbig, 25), ctx.load_db(ismall, cwsmall, 5)
    qbig = [cl.query(cwbig[7 * i + 1], 25, 0, stream=500 + i) for i in range(4)]
    qsmall = cl.query(cwsmall[3], 5, 0, stream=510)
    alone_big = [ctx.answer(dbig, q) for q in qbig]
    alone_small = ctx.answer(dsmall, qsmall)
    srv = B.Server([(ctx, dbig, 0), (ctx, dsmall, 0)], max_batch=4)
    for q in qbig:  # warm both lanes' plans and graphs
        srv.wait(srv.submit(0, q), 0)
    srv.wait(srv.submit(1, qsmall), 1)
    t_big = time.perf_counter()
    big = [srv.submit(0, q) for q in qbig]
    time.sleep(0.005)  # the big batch is on the GPU by now
    t_small = time.perf_counter()
    small = srv.submit(1, qsmall)
    st, resp, lat_small = srv.wait(small, 1)
    assert st == 1 and np.array_equal(resp, alone_small)
    done_small = t_small + lat_small
    done_big = []
    for tk, want in zip(big, alone_big):
        st, resp, lat = srv.wait(tk, 0)
        assert st == 1 and np.array_equal(resp, want)
        done_big.append(t_big + lat)
    assert done_small < min(done_big), (done_small - t_big, [d - t_big for d in done_big])
    stats = srv.stats()
    srv.close()
    assert stats["max_concurrent"] >= 2 and stats["failed"] == 0
    ctx.close()


def test_failed_device_check_fails_its_batch_only():
    """A device check that fails (raised here by the test hook on the
    lane's slot flag, no kernel involved) fails the requests of the batch
    that reads it with EINTERNAL; the next batch is answered normally."""
    from paper_2202_07569_gb300 import binding as B

    cl = Client(4096, 2, seed=101)
    ctx = cl.context()
    items, cw, _ = database(30, 100, T, 2, 9, seed=102)
    db = ctx.load_db(items, cw, 9)
    q = cl.query(cw[4], 9, 0, stream=520)
    want = ctx.answer(db, q)
    srv = B.Server([(ctx, db, 0)], max_batch=1)
    st, resp, _ = srv.wait(srv.submit(0, q), 0)
    assert st == 1 and np.array_equal(resp, want)
    ctx.inject_status(1)  # the server's one lane holds slot 1
    st, resp, _ = srv.wait(srv.submit(0, q), 0)
    assert st == B.EINTERNAL and resp is None
    st, resp, _ = srv.wait(srv.submit(0, q), 0)
    assert st == 1 and np.array_equal(resp, want)
    assert srv.stats()["failed"] == 1
    srv.close()
    ctx.close()
