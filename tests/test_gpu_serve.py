"""Online serving (configuration 5's pattern): continuous batching over
resident databases of two parameter sets.  Every response must be the same
as the query answered alone (and, for sampled queries, the oracle's)."""
import threading

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
    srv = B.Server(targets, max_batch=8)
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
