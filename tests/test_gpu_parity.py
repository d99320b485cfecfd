"""Parity of the CUDA path (called through the C ABI) with the oracle.

Every comparison is bit for bit: the path is exact integer arithmetic and
the oracle computes the same exact function step by step.
"""
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


_clients = {}


def client(N, L, seed=3, c_max=0):
    key = (N, L, seed, c_max)
    if key not in _clients:
        cl = Client(N, L, seed, c_max)
        cl.ctx = cl.context()
        _clients[key] = cl
    return _clients[key]


# ------------------------------------------------------------ multiplication
@pytest.mark.parametrize("N,L", [(1024, 1), (4096, 2), (2048, 3), (8192, 4), (4096, 5),
                                 (4096, 6), (16384, 7), (4096, 8)])
def test_mul_matches_oracle(N, L):
    """M for every count of ciphertext primes (extension bases of 5 to 30
    primes, each scale-down instantiation) against the oracle."""
    cl = client(N, L)
    st = syn.Stream(100, N + L)
    for trial in range(2):
        a = syn.uniform_residues(st, cl.q, (2,), N)
        b = syn.uniform_residues(st, cl.q, (2,), N)
        got = cl.ctx.mul(a, b)
        assert np.array_equal(got, cl.O.bfv_mul(a, b, cl.rlk)), trial


@pytest.mark.parametrize("N,L", [(1024, 1), (8192, 4), (16384, 7), (4096, 8)])
def test_scale_down_exact_path_matches_oracle(N, L):
    """The scale-down's exact path, forced for every coefficient
    (CWPIR_OPT_SCALE_EXACT = 1): products and a selection entry equal the
    oracle's, and the default again afterwards."""
    from paper_2202_07569_gb300 import binding as B

    cl = client(N, L)
    st = syn.Stream(102, N + L)
    a = syn.uniform_residues(st, cl.q, (2,), N)
    b = syn.uniform_residues(st, cl.q, (2,), N)
    want = cl.O.bfv_mul(a, b, cl.rlk)
    cl.ctx.set_option(B.OPT_SCALE_EXACT, 1)
    try:
        assert cl.ctx.get_option(B.OPT_SCALE_EXACT) == 1
        assert np.array_equal(cl.ctx.mul(a, b), want)
        items, cw, _ = database(20, 16, T, 3, 8, seed=9)
        db = cl.ctx.load_db(items, cw, 8)
        query = cl.query(cw[5], 8, 0, stream=7)
        got = cl.ctx.selection(db, query, np.array([5, 11], np.uint64))
        for i, r in enumerate((5, 11)):
            assert np.array_equal(got[i], cl.O.selection(query, cw[r], cl.rlk)), r
        cl.ctx.free_db(db)
    finally:
        cl.ctx.set_option(B.OPT_SCALE_EXACT, 0)
    assert np.array_equal(cl.ctx.mul(a, b), want)


def test_mul_edge_coefficients():
    """Coefficients at 0, 1, Q-1 and next to Q/2 (mixed-radix branch)."""
    import math

    N, L = 4096, 2
    cl = client(N, L)
    q = [int(v) for v in cl.q]
    Q = math.prod(q)
    st = syn.Stream(101)
    a = syn.uniform_residues(st, q, (2,), N)
    b = syn.uniform_residues(st, q, (2,), N)
    specials = [0, 1, Q - 1, (Q - 1) // 2, (Q + 1) // 2, (Q - 3) // 2, (Q + 3) // 2]
    for i, v in enumerate(specials):
        for poly in range(2):
            for j, qq in enumerate(q):
                a[poly, j, 7 * i] = v % qq
                b[poly, j, 11 * i + 1] = (Q - 1 - v) % qq
    assert np.array_equal(cl.ctx.mul(a, b), cl.O.bfv_mul(a, b, cl.rlk))


def test_mul_decrypts_to_product():
    N, L = 8192, 4
    cl = client(N, L)
    mu = [np.zeros(N, np.uint32) for _ in range(2)]
    mu[0][0], mu[0][5] = 1, 7
    mu[1][0], mu[1][1] = 3, 1
    a, e = cl.cd.encryption(2, 5)
    ca = cl.O.encrypt(mu[0], cl.cd.s, a[0], e[0])
    cb = cl.O.encrypt(mu[1], cl.cd.s, a[1], e[1])
    got, budget = cl.decrypt(cl.ctx.mul(ca, cb))
    want = np.zeros(N, np.uint32)
    want[0], want[1], want[5], want[6] = 3, 1, 21, 7
    assert np.array_equal(got, want) and budget > 0


# ------------------------------------------------------------ substitution, expansion
@pytest.mark.parametrize("N,L", [(4096, 2), (16384, 7)])
def test_substitute_matches_oracle(N, L):
    cl = client(N, L, c_max=3)
    for g in cl.galois:
        ct = syn.uniform_residues(syn.Stream(102, g), cl.q, (2,), N)
        assert np.array_equal(cl.ctx.substitute(g, ct), cl.O.substitute(g, ct, cl.galois[g]))


@pytest.mark.parametrize("N,L,m,c", [(4096, 2, 24, 3), (8192, 4, 37, 2), (16384, 7, 64, 6)])
def test_expand_matches_oracle(N, L, m, c):
    cl = client(N, L, c_max=c)
    pos = oracle.map_perfect(12345 % oracle.binom(m, 4), m, 4)
    query = cl.query(pos, m, c, stream=3)
    got = cl.ctx.expand(query, c, m)
    want = cl.O.expand(query, c, m, cl.gkeys)
    assert np.array_equal(got, want)
    bits = np.zeros(m, np.uint32)
    bits[pos] = 1
    for j in (int(pos[0]), (int(pos[0]) + 1) % m):
        mu, budget = cl.decrypt(got[j])
        assert mu[0] == bits[j] and not mu[1:].any() and budget > 0


# ------------------------------------------------------------ plain multiplication
def test_plain_mul_matches_oracle():
    N, L = 8192, 4
    cl = client(N, L)
    items, cw, _ = database(5, 3000, T, 2, 5, seed=7)
    db = cl.ctx.load_db(items, cw, 5)
    ct = syn.uniform_residues(syn.Stream(103), cl.q, (2,), N)
    for row in (0, 4):
        assert np.array_equal(cl.ctx.plain_mul(db, row, ct), cl.O.plain_mul(ct, items[row]))
    cl.ctx.free_db(db)


# ------------------------------------------------------------ selection vector
@pytest.mark.parametrize("k,m", [(2, 24), (3, 14), (4, 37), (5, 12)])
def test_selection_matches_oracle(k, m):
    N, L = 4096, 2
    cl = client(N, L)
    n = 60
    items, cw, _ = database(n, 16, T, k, m, seed=8)
    db = cl.ctx.load_db(items, cw, m)
    query = cl.query(cw[17], m, 0, stream=4)
    rows = np.array([0, 17, 59, 33], np.uint64)
    for share in (1, 0):
        cl.ctx.set_option(1, share)
        got = cl.ctx.selection(db, query, rows)
        for i, r in enumerate(rows.tolist()):
            assert np.array_equal(got[i], cl.O.selection(query, cw[r], cl.rlk)), (share, r)
    cl.ctx.set_option(1, 1)
    cl.ctx.free_db(db)


# ------------------------------------------------------------ full answers
def test_c1_answer_bit_exact_and_decrypts():
    """Configuration 1 at full size: n=256, k=2, m=24, N=4096, L=2."""
    cfg = CONFIGS["c1"]
    cl = Client(cfg["N"], cfg["L"], cfg["seed"])
    ctx = cl.context()
    items, cw, _ = database(cfg["n"], cfg["plen"], cfg["bound"], cfg["k"], cfg["m"], cfg["seed"] + 1)
    db = ctx.load_db(items, cw, cfg["m"])
    target = int(syn.Stream(cfg["seed"] + 2).below(cfg["n"], 1)[0])
    query = cl.query(cw[target], cfg["m"], 0)
    got = ctx.answer(db, query)
    want = cl.O.answer(items, cw, cfg["m"], query, cl.rlk)
    assert np.array_equal(got, want)
    mu, budget = cl.decrypt(got)
    assert np.array_equal(mu, items[target]) and budget > 0
    stats = ctx.last_stats()
    assert stats["rows"] == cfg["n"] and stats["mults"] == cfg["n"]


@pytest.mark.parametrize("share,batch", [(1, 0), (0, 0), (1, 7), (0, 13)])
def test_c2_params_answer_bit_exact(share, batch):
    """N=8192, L=4, k=4, m=37 on 150 rows: shared first level on and off and
    batch splits with ragged tails all give the oracle's response."""
    cl = client(8192, 4, seed=11)
    n, k, m = 150, 4, 37
    items, cw, _ = database(n, 8192, 1 << 16, k, m, seed=12)
    ctx = cl.ctx
    ctx.set_option(1, share)
    ctx.set_option(2, batch)
    db = ctx.load_db(items, cw, m)
    query = cl.query(cw[77], m, 0, stream=6)
    got = ctx.answer(db, query)
    if "c2small" not in _clients:
        _clients["c2small"] = cl.O.answer(items, cw, m, query, cl.rlk)
    assert np.array_equal(got, _clients["c2small"])
    mu, budget = cl.decrypt(got)
    assert np.array_equal(mu, items[77]) and budget > 0
    ctx.set_option(1, 1)
    ctx.set_option(2, 0)
    ctx.free_db(db)


@pytest.mark.parametrize("N,L,n,k,m,nq", [(4096, 2, 61, 2, 12, 1), (8192, 4, 100, 4, 9, 3),
                                           (16384, 3, 40, 3, 8, 2)])
def test_row_basis_equals_ciphertext_basis(N, L, n, k, m, nq):
    """Databases of one plaintext per row answered through the four-prime
    row basis (default) and modulo the ciphertext primes
    (CWPIR_OPT_ROW_BASIS = 0) give the same bits: single and batched
    answers, plain multiplications, and the oracle's answer."""
    from paper_2202_07569_gb300 import binding as B

    cl = Client(N, L, seed=300 + L)
    ctx = cl.context()
    items, cw, _ = database(n, N, T if N == 4096 else 1 << 16, k, m, seed=310 + L)
    dbs = []
    for rb in (1, 0):
        ctx.set_option(B.OPT_ROW_BASIS, rb)
        dbs.append(ctx.load_db(items, cw, m))
    ctx.set_option(B.OPT_ROW_BASIS, 1)
    targets = [n - 1 - 7 * i for i in range(nq)]
    queries = np.stack([cl.query(cw[r], m, 0, stream=40 + i) for i, r in enumerate(targets)])
    want = [cl.O.answer(items, cw, m, queries[i], cl.rlk) for i in range(nq)]
    for db in dbs:
        for i in range(nq):
            assert np.array_equal(ctx.answer(db, queries[i]), want[i])
        got = ctx.answer_batch(db, queries)
        for i in range(nq):
            assert np.array_equal(got[i], want[i])
    ct = syn.uniform_residues(syn.Stream(320), cl.q, (2,), N)
    for row in (0, n - 1):
        pm = cl.O.plain_mul(ct, items[row])
        for db in dbs:
            assert np.array_equal(ctx.plain_mul(db, row, ct), pm)
    mu, budget = cl.decrypt(want[0])
    assert np.array_equal(mu, items[targets[0]]) and budget > 0
    ctx.close()


def _sparse_rows(n, count, seed):
    rows = syn.Stream(seed, 9).below(n, 4 * count)
    return np.array(sorted(set(rows.tolist())))[:count]


def test_c2_full_size_sparse_parity_and_random_decrypt():
    """Configuration 2 at full size (n=65536, k=4, m=37, N=8192, L=4) in the
    launch configuration of the benchmark.  The response is linear in the
    rows: with all but a sample of rows zero the oracle computes the exact
    response from the sampled rows alone while the GPU still runs the full
    selection vector.  A second answer over uniform rows must decrypt to the
    target row."""
    cfg = CONFIGS["c2"]
    cl = client(cfg["N"], cfg["L"], seed=cfg["seed"])
    ctx = cl.ctx
    n, k, m = cfg["n"], cfg["k"], cfg["m"]
    items, cw, _ = database(n, cfg["plen"], cfg["bound"], k, m, cfg["seed"] + 1)
    target = int(syn.Stream(cfg["seed"] + 2).below(n, 1)[0])
    query = cl.query(cw[target], m, 0)
    db = ctx.load_db(items, cw, m)
    got = ctx.answer(db, query)
    mu, budget = cl.decrypt(got)
    assert np.array_equal(mu, items[target]) and budget > 0
    ctx.free_db(db)
    sample = np.union1d(_sparse_rows(n, 6, 13), [target])
    sparse = np.zeros_like(items)
    sparse[sample] = items[sample]
    db = ctx.load_db(sparse, cw, m)
    got = ctx.answer(db, query)
    want = cl.O.answer(items[sample], cw[sample], m, query, cl.rlk)
    assert np.array_equal(got, want)
    ctx.free_db(db)


def test_c3_keyword_full_size_sparse_parity_present_and_absent():
    """Configuration 3 at full size: 16384 rows keyed by uniform 32-bit
    keywords, k=8, m=64, N=16384, L=7, compressed query (c=6, one ct).
    Present keyword decrypts to its row; absent keyword to zeros; sampled
    rows give the oracle's exact response."""
    cfg = CONFIGS["c3"]
    cl = client(cfg["N"], cfg["L"], seed=cfg["seed"], c_max=cfg["c"])
    ctx = cl.ctx
    n, k, m, c = cfg["n"], cfg["k"], cfg["m"], cfg["c"]
    items, cw, ids = database(n, cfg["plen"], cfg["bound"], k, m, cfg["seed"] + 1, keyword=True)
    db = ctx.load_db(items, cw, m)
    present = int(syn.Stream(cfg["seed"] + 2).below(n, 1)[0])
    q1 = cl.query(cw[present], m, c, stream=1)
    got = ctx.answer(db, q1, c)
    mu, budget = cl.decrypt(got)
    want = np.zeros(cfg["N"], np.uint32)
    want[: cfg["plen"]] = items[present]
    assert np.array_equal(mu, want) and budget > 0
    absent = int(syn.distinct_u32(syn.Stream(cfg["seed"] + 3), 1, exclude=ids)[0])
    q2 = cl.query(oracle.map_perfect(absent, m, k), m, c, stream=2)
    got2 = ctx.answer(db, q2, c)
    mu2, budget2 = cl.decrypt(got2)
    assert not mu2.any() and budget2 > 0
    ctx.free_db(db)
    sample = np.union1d(_sparse_rows(n, 3, 23), [present])
    sparse = np.zeros_like(items)
    sparse[sample] = items[sample]
    db = ctx.load_db(sparse, cw, m)
    got = ctx.answer(db, q1, c)
    want = cl.O.answer(items[sample], cw[sample], m, q1, cl.rlk, c=c, gkeys=cl.gkeys)
    assert np.array_equal(got, want)
    ctx.free_db(db)


def _overlap_rows(cw, qpos, rng_rows, want_each):
    """Rows of rng_rows grouped by how many codeword positions they share
    with the query's, at most want_each of every overlap."""
    qs = set(int(x) for x in qpos)
    by = {}
    for r in rng_rows:
        ov = len(qs & set(int(x) for x in cw[r]))
        if len(by.setdefault(ov, [])) < want_each:
            by[ov].append(int(r))
    return by


def test_c2_full_size_selection_entries_bit_exact():
    """Selection-vector entries (Alg. Selection Vector Calculation: the
    balanced product tree of Eq. plain-cw-eq) of 80 rows of the full
    configuration-2 database (n=65536, k=4, m=37, N=8192, L=4), each equal
    to the oracle's bit for bit: the target row, rows sharing 0 ... 3
    positions with the query (the number of factors that encrypt 1), rows
    that reuse one shared first-level pair product with another sampled row
    (same first pair, or same second pair), and uniform rows.  The entries
    come from the shared pair products of the sampled rows, the context's
    multiplications per launch and the same kernels as the answer."""
    cfg = CONFIGS["c2"]
    cl = client(cfg["N"], cfg["L"], seed=cfg["seed"])
    ctx = cl.ctx
    n, k, m = cfg["n"], cfg["k"], cfg["m"]
    cw = np.stack([oracle.map_perfect(i, m, k) for i in range(n)])
    db = ctx.load_db(np.zeros((n, 1), np.uint32), cw, m)
    st = syn.Stream(cfg["seed"] + 40)
    target = int(st.below(n, 1)[0])
    query = cl.query(cw[target], m, 0, stream=41)
    rows = [target]
    by = _overlap_rows(cw, cw[target], st.below(n, 20000).tolist(), 6)
    assert set(by) >= {0, 1, 2}
    for ov in sorted(by):
        rows += by[ov]
    for r in st.below(n, 12).tolist():  # partners sharing a first-level pair
        p = [int(x) for x in cw[r]]
        for alt in ([p[0], p[1], p[2], p[3] + 1], [p[0] - 1, p[1], p[2], p[3]]):
            if 0 <= alt[0] and alt[3] < m and len(set(alt)) == 4 and alt == sorted(alt):
                x = int(oracle.map_inverse(np.array(alt, np.uint16)))
                if x < n:
                    rows += [int(r), x]
    rows += [int(r) for r in st.below(n, 80).tolist()]
    rows = np.array(list(dict.fromkeys(rows))[:80], np.uint64)
    assert rows.size == 80 and target in rows.tolist()
    got = ctx.selection(db, query, rows)
    for i, r in enumerate(rows.tolist()):
        assert np.array_equal(got[i], cl.O.selection(query, cw[r], cl.rlk)), r
    ctx.free_db(db)


def test_c3_full_size_selection_entries_bit_exact():
    """Selection entries of 16 rows of the full configuration-3 keyword
    database (16384 uniform 32-bit keywords, k=8, m=64, N=16384, L=7) for a
    compressed query (c=6, expanded on the GPU by Alg. Query Expansion):
    the present keyword's row, rows sharing several positions with it, and
    uniform rows, each equal to the oracle's entry over the oracle's
    expansion of the same query."""
    cfg = CONFIGS["c3"]
    cl = client(cfg["N"], cfg["L"], seed=cfg["seed"], c_max=cfg["c"])
    ctx = cl.ctx
    n, k, m, c = cfg["n"], cfg["k"], cfg["m"], cfg["c"]
    ids = syn.distinct_u32(syn.Stream(cfg["seed"] + 1, 2), n)
    cw = np.stack([oracle.map_perfect(int(x), m, k) for x in ids])
    db = ctx.load_db(np.zeros((n, 1), np.uint32), cw, m)
    st = syn.Stream(cfg["seed"] + 50)
    target = int(st.below(n, 1)[0])
    query = cl.query(cw[target], m, c, stream=51)
    rows = [target]
    by = _overlap_rows(cw, cw[target], range(n), 2)
    for ov in sorted(by, reverse=True):
        if ov < k:
            rows += by[ov]
    rows += [int(r) for r in st.below(n, 32).tolist()]
    rows = np.array(list(dict.fromkeys(rows))[:16], np.uint64)
    assert rows.size == 16
    got = ctx.selection(db, query, rows, c)
    cts = cl.O.expand(query, c, m, cl.gkeys)
    for i, r in enumerate(rows.tolist()):
        assert np.array_equal(got[i], cl.O.selection(cts, cw[r], cl.rlk)), r
    ctx.free_db(db)


# ------------------------------------------------------------ edge cases and errors
def test_single_row_and_unary_code():
    cl = client(4096, 2)
    items, cw, _ = database(1, 100, T, 2, 5, seed=31)
    db = cl.ctx.load_db(items, cw, 5)
    q = cl.query(cw[0], 5, 0, stream=8)
    assert np.array_equal(cl.ctx.answer(db, q), cl.O.answer(items, cw, 5, q, cl.rlk))
    cl.ctx.free_db(db)
    items, cw, _ = database(9, 50, T, 1, 9, seed=32)  # k = 1: unary selection
    db = cl.ctx.load_db(items, cw, 9)
    q = cl.query(cw[4], 9, 0, stream=9)
    got = cl.ctx.answer(db, q)
    assert np.array_equal(got, cl.O.answer(items, cw, 9, q, cl.rlk))
    cl.ctx.free_db(db)


def test_errors_are_reported():
    from paper_2202_07569_gb300 import binding as B

    cl = client(4096, 2)
    bad = syn.uniform_residues(syn.Stream(1), cl.q, (2,), 4096)
    bad[0, 0, 0] = cl.q[0]
    with pytest.raises(B.CwpirError) as ei:
        cl.ctx.mul(bad, bad)
    assert ei.value.code == -1
    with pytest.raises(B.CwpirError) as ei:
        cl.ctx.answer(12345, bad[None])
    assert ei.value.code == -3
    with pytest.raises(B.CwpirError) as ei:
        cl.ctx.substitute(7, bad)
    assert ei.value.code == -7
    items, cw, _ = database(4, 10, T, 2, 4, seed=33)
    cw[1] = cw[1][::-1]
    with pytest.raises(B.CwpirError):
        cl.ctx.load_db(items, cw, 4)


def test_keyword_pir_lossy_mapping_64bit_keywords():
    """Alg. Lossy Mapping for a domain beyond a perfect mapping's reach:
    64-bit keywords mapped into CW(12, 3) (220 codewords) with compressed
    queries.  Keywords whose codewords collide are left out of the database
    (they would be selected together); present keywords return their row,
    an absent keyword's codeword not in the database returns zeros, and the
    responses equal the oracle's bit for bit."""
    from paper_2202_07569_gb300 import binding as B

    N, L, k, m, c = 8192, 4, 3, 12, 2
    cl = Client(N, L, seed=75, c_max=c)
    ctx = cl.context()
    st = syn.Stream(76)
    words = [int(w) for w in st.words(40)]
    cws, keep = {}, []
    for w in words:
        key = tuple(B.map_lossy(w, m, k).tolist())
        if key not in cws:
            cws[key] = w
            keep.append(w)
    items = syn.payload(st, len(keep), 300, 1 << 16)
    cw = np.stack([B.map_lossy(w, m, k) for w in keep])
    db = ctx.load_db(items, cw, m)
    absent = next(int(w) for w in st.words(1000)
                  if tuple(B.map_lossy(int(w), m, k).tolist()) not in cws)
    for i, w in ((0, keep[0]), (len(keep) - 1, keep[-1]), (None, absent)):
        q = cl.query(oracle.map_lossy(w, m, k), m, c, stream=77 + (i or 0))
        got = ctx.answer(db, q, c)
        assert np.array_equal(got, cl.O.answer(items, cw, m, q, cl.rlk, c=c, gkeys=cl.gkeys))
        mu, budget = cl.decrypt(got)
        want = np.zeros(N, np.uint32)
        if i is not None:
            want[:300] = items[i]
        assert np.array_equal(mu, want) and budget > 0
    ctx.close()
