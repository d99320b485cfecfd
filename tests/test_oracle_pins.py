"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, never against the oracle itself.

Each test names what it pins.  Python integers (exact) serve as the
independent brute force at tiny sizes; closed forms and decryption
invariants cover the rest.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from paper_2202_07569_gb300 import synthetic as syn

T = 65537


# ---------------------------------------------------------------- helpers
def schoolbook_nega(a, b, mod=None):
    """Negacyclic product in Z[x]/(x^N+1) (optionally mod `mod`), exact ints."""
    N = len(a)
    out = [0] * N
    for i, x in enumerate(a):
        if x == 0:
            continue
        for j, y in enumerate(b):
            d = i + j
            if d >= N:
                out[d - N] -= x * y
            else:
                out[d] += x * y
    if mod is not None:
        out = [v % mod for v in out]
    return out


def crt_int(res, primes):
    Q = math.prod(primes)
    x = 0
    for r, p in zip(res, primes):
        h = Q // p
        x += int(r) * h * pow(h, -1, p)
    return x % Q


def centered(x, M):
    return x - M if x > M // 2 else x


def lift_poly(poly, primes):
    Q = math.prod(primes)
    N = poly.shape[1]
    return [centered(crt_int([poly[j, i] for j in range(len(primes))], primes), Q)
            for i in range(N)]


def to_rns(vals, primes):
    return np.array([[int(v) % p for v in vals] for p in primes], dtype=np.uint64)


def small_setup(orc, N, L, seed=5):
    q = [int(p) for p in orc.primes(N, L)]
    O = orc.Oracle(N, q)
    cd = syn.ClientDraws(seed, q, N)
    a, e = cd.relin()
    rlk = O.keygen_relin(cd.s, a, e)
    return O, q, cd, rlk


def encrypt_many(O, cd, mus, stream=0):
    ea, ee = cd.encryption(len(mus), stream)
    return [O.encrypt(mu, cd.s, ea[i], ee[i]) for i, mu in enumerate(mus)]


def rt_mul(a, b):
    return [v % T for v in schoolbook_nega([int(x) for x in a], [int(x) for x in b])]


# ------------------------------------------------------------ primes
def test_primes_are_the_largest_ntt_friendly_primes(orc):
    sympy = pytest.importorskip("sympy")
    for N, L in ((16, 3), (4096, 2), (8192, 4), (16384, 7)):
        got = [int(p) for p in orc.primes(N, L)]
        # brute force: walk down from 2^54 over values = 1 mod 2N
        want, p = [], (1 << 54) - 2 * N + 1
        while len(want) < L:
            if sympy.isprime(p):
                want.append(p)
            p -= 2 * N
        assert got == want
        assert all(x % (2 * N) == 1 and x < (1 << 54) for x in got)


def test_miller_rabin_against_sympy(orc):
    sympy = pytest.importorskip("sympy")
    st = syn.Stream(99)
    for v in st.words(300).tolist():
        v = int(v) >> 1
        assert orc.is_prime(v) == bool(sympy.isprime(v))
    for v in (2, 3, 4, 561, 3215031751, 18014398509309953, (1 << 61) - 1):
        assert orc.is_prime(v) == bool(sympy.isprime(v))


# ------------------------------------------------------------ ring arithmetic
@pytest.mark.parametrize("N", [8, 16, 64, 256])
def test_negacyclic_ntt_product_matches_schoolbook(orc, N):
    for p in (int(orc.primes(N, 1)[0]), int(orc.primes(N, 1, bits=62)[0])):
        st = syn.Stream(N, p & 0xFFFF)
        a = st.below(p, N)
        b = st.below(p, N)
        got = orc.negacyclic_mul_mod(a, b, p)
        want = schoolbook_nega(a.tolist(), b.tolist(), p)
        assert got.tolist() == want


@pytest.mark.parametrize("N", [8, 64])
def test_x_to_the_N_is_minus_one(orc, N):
    """Closed form of R = Z[x]/(x^N+1): x^(N-1) * x = -1."""
    p = int(orc.primes(N, 1)[0])
    a = np.zeros(N, np.uint64)
    b = np.zeros(N, np.uint64)
    a[N - 1] = 1
    b[1] = 1
    got = orc.negacyclic_mul_mod(a, b, p)
    assert got[0] == p - 1 and not got[1:].any()


@pytest.mark.parametrize("N,L", [(8, 2), (16, 3), (32, 2)])
def test_exact_integer_product_matches_bigint_schoolbook(orc, N, L):
    """The tensor's integer products: centered lifts multiplied exactly."""
    q = [int(p) for p in orc.primes(N, L)]
    O = orc.Oracle(N, q)
    Q = math.prod(q)
    st = syn.Stream(11, N)
    for trial in range(3):
        a = syn.uniform_residues(st, q, (), N)
        b = syn.uniform_residues(st, q, (), N)
        if trial == 2:  # extremes of the centered range: (Q-1)/2 and (Q+1)/2
            for j, p in enumerate(q):
                a[j, :] = ((Q - 1) // 2) % p
                b[j, :] = ((Q + 1) // 2) % p
        want = schoolbook_nega(lift_poly(a, q), lift_poly(b, q))
        assert O.exact_product(a, b) == want


def test_scale_round_is_nearest_integer(orc):
    """round(t*d/Q) by exact rationals, including values closest to a tie."""
    N, L = 16, 3
    q = [int(p) for p in orc.primes(N, L)]
    O = orc.Oracle(N, q)
    Q = math.prod(q)
    st = syn.Stream(12)
    ds = [0, 1, -1, Q, -Q, 2 * N * (Q // 2) ** 2, -2 * N * (Q // 2) ** 2]
    for w in st.words(40).tolist():
        ds.append((int(w) * Q * Q) >> 63 - (int(w) & 7))
        ds.append(-((int(w) * Q) >> 20))
    # d with t*d/Q as close to x + 1/2 as possible (Q odd: never equal)
    inv_t = pow(T, -1, Q)
    for r in ((Q - 1) // 2, (Q + 1) // 2):
        d = (r * inv_t) % Q
        ds += [d, d - Q, d + 5 * Q]
    for d in ds:
        want = round(Fraction(T * d, Q))  # nearest; no ties can occur
        got = O.scale_round(d)
        assert got.tolist() == [want % p for p in q], d


@pytest.mark.parametrize("N,L", [(8, 2), (16, 3)])
def test_tensor_matches_fv_definition(orc, N, L):
    """FV multiplication before relinearisation, by brute force:
    e_l = round(t/Q * d_l) with d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1."""
    q = [int(p) for p in orc.primes(N, L)]
    O = orc.Oracle(N, q)
    Q = math.prod(q)
    st = syn.Stream(13, N)
    a = syn.uniform_residues(st, q, (2,), N)
    b = syn.uniform_residues(st, q, (2,), N)
    A = [lift_poly(a[i], q) for i in range(2)]
    B = [lift_poly(b[i], q) for i in range(2)]
    d0 = schoolbook_nega(A[0], B[0])
    d1 = [x + y for x, y in zip(schoolbook_nega(A[0], B[1]), schoolbook_nega(A[1], B[0]))]
    d2 = schoolbook_nega(A[1], B[1])
    got = O.tensor(a, b)
    for l, d in enumerate((d0, d1, d2)):
        e = [round(Fraction(T * v, Q)) for v in d]
        assert got[l].tolist() == [[v % p for v in e] for p in q]


def test_keyswitch_identity_exact(orc):
    """u0 + u1*s = z*w + sum_i [z]_{q_i} e_i (mod Q), digits in [0, q_i)."""
    N, L = 16, 3
    q = [int(p) for p in orc.primes(N, L)]
    O = orc.Oracle(N, q)
    Q = math.prod(q)
    cd = syn.ClientDraws(21, q, N)
    a, e = cd.relin()
    rlk = O.keygen_relin(cd.s, a, e)
    z = syn.uniform_residues(syn.Stream(22), q, (), N)
    u = O.keyswitch(z, rlk)
    s = [int(v) for v in cd.s]
    w = schoolbook_nega(s, s)
    zi = [crt_int(z[:, i], q) for i in range(N)]
    lhs = [(crt_int(u[0][:, i], q) + x) % Q
           for i, x in enumerate(schoolbook_nega([crt_int(u[1][:, i], q) for i in range(N)], s))]
    noise = [0] * N
    for i in range(L):
        Di = [int(v) for v in z[i]]
        noise = [x + y for x, y in zip(noise, schoolbook_nega(Di, [int(v) for v in e[i]]))]
    rhs = [(x + y) % Q for x, y in zip(schoolbook_nega(zi, w), noise)]
    assert lhs == rhs


# ------------------------------------------------------------ BFV invariants
def test_encrypt_decrypt_roundtrip(orc):
    O, q, cd, rlk = small_setup(orc, 64, 2)
    st = syn.Stream(31)
    mus = [st.below(T, 64).astype(np.uint32) for _ in range(3)]
    for mu, ct in zip(mus, encrypt_many(O, cd, mus)):
        got, budget = O.decrypt(ct, cd.s)
        assert np.array_equal(got, mu) and budget > 50


def invariant_budget(ct, s, q):
    """log2 Q - 1 - log2 max_i |t x_i - Q round(t x_i / Q)| with
    x = c0 + c1 s (mod Q), computed with Python integers from the secret."""
    Q = math.prod(q)
    c0, c1 = lift_poly(ct[0], q), lift_poly(ct[1], q)
    x = [(a + b) % Q for a, b in zip(c0, schoolbook_nega(c1, [int(v) for v in s]))]
    worst = 0
    for v in x:
        r = (T * v + Q // 2) // Q  # round half up; t x / Q is never a half integer
        worst = max(worst, abs(T * v - Q * r))
    return math.log2(Q) - 1 - math.log2(worst)


def test_noise_budget_matches_its_definition(orc):
    """The budget that decryption reports is log2 Q - 1 - log2 of the largest
    |t (c0 + c1 s) - Q mu'| (mu' the rounded quotient), recomputed here from
    the secret with exact integers at N = 16, L = 3: for a fresh ciphertext,
    a product M(a, b) and a plain product.  Each step adds noise, so the
    budgets also decrease in that order."""
    N, L = 16, 3
    O, q, cd, rlk = small_setup(orc, N, L)
    st = syn.Stream(34)
    mus = [st.below(T, N).astype(np.uint32) for _ in range(2)]
    ca, cb = encrypt_many(O, cd, mus, stream=3)
    prod = O.bfv_mul(ca, cb, rlk)
    pm = O.plain_mul(prod, st.below(T, N).astype(np.uint32))
    budgets = []
    for ct in (ca, prod, pm):
        _, got = O.decrypt(ct, cd.s)
        assert abs(got - invariant_budget(ct, cd.s, q)) < 1e-9
        budgets.append(got)
    assert budgets[0] > budgets[1] > budgets[2] > 0


@pytest.mark.parametrize("N,L", [(64, 2), (4096, 2)])
def test_multiplication_decrypts_to_ring_product(orc, N, L):
    """Dec(M(a,b)) = Dec(a) Dec(b) in R_t; the size-3 tensor decrypts the
    same before relinearisation."""
    O, q, cd, rlk = small_setup(orc, N, L)
    st = syn.Stream(32, N)
    mu = [np.zeros(N, np.uint32) for _ in range(2)]
    for v in mu:  # sparse messages keep the Python product cheap at N=4096
        idx = st.below(N, 6).astype(np.int64)
        v[idx] = st.below(T, 6).astype(np.uint32)
    ca, cb = encrypt_many(O, cd, mu)
    want = rt_mul(mu[0], mu[1])
    got, budget = O.decrypt(O.bfv_mul(ca, cb, rlk), cd.s)
    assert got.tolist() == want and budget > 0
    got3, _ = O.decrypt(O.tensor(ca, cb), cd.s)
    assert got3.tolist() == want


def test_plain_mul_and_monomial_and_automorphism(orc):
    N = 64
    O, q, cd, rlk = small_setup(orc, N, 2)
    st = syn.Stream(33)
    mu = st.below(T, N).astype(np.uint32)
    item = st.below(T, 40).astype(np.uint32)
    (ct,) = encrypt_many(O, cd, [mu])
    pad = np.zeros(N, np.uint32)
    pad[:40] = item
    got, _ = O.decrypt(O.plain_mul(ct, item), cd.s)
    assert got.tolist() == rt_mul(mu, pad)
    for e in (-5, -1, 0, 3, N - 1, N + 7, -(2 * N - 1)):
        xe = [0] * N
        r = e % (2 * N)
        xe[r % N] = 1 if r < N else T - 1
        ctm = np.stack([O.monomial(e, ct[0]), O.monomial(e, ct[1])])
        got, _ = O.decrypt(ctm, cd.s)
        assert got.tolist() == rt_mul(mu, xe), e
    # Sub_g: decrypts to mu(x^g)
    for gi, g in enumerate((N + 1, N // 2 + 1, 5, 2 * N - 1)):
        a, e = cd.galois(gi)
        gk = O.keygen_galois(g, cd.s, a, e)
        got, budget = O.decrypt(O.substitute(g, ct, gk), cd.s)
        want = [0] * N
        for i, v in enumerate(mu.tolist()):
            d = (i * g) % (2 * N)
            if d >= N:
                want[d - N] = (-v) % T
            else:
                want[d] = v
        assert got.tolist() == want and budget > 0


# ------------------------------------------------------------ expansion
def galois_keys(O, cd, N, c):
    ks = []
    for a_ in range(c):
        a, e = cd.galois(a_)
        ks.append(O.keygen_galois(N // (1 << a_) + 1, cd.s, a, e))
    return np.stack(ks)


@pytest.mark.parametrize("m,c", [(20, 3), (9, 2), (5, 0), (64, 6)])
def test_expansion_recovers_query_bits(orc, m, c):
    """Alg. Query + Alg. Query Expansion: expanded ct j decrypts to the
    constant E_q[j]."""
    N = 64
    O, q, cd, rlk = small_setup(orc, N, 2)
    gk = galois_keys(O, cd, N, c) if c else np.zeros((1,) + O.key_shape, np.uint64)
    k = min(3, m)
    pos = orc.map_perfect(7 % orc.binom(m, k), m, k)
    h = -(-m // (1 << c))
    a, e = cd.encryption(h, 9)
    query = O.make_query(pos, m, c, cd.s, a, e)
    cts = O.expand(query, c, m, gk) if c else query
    bits = np.zeros(m, np.int64)
    bits[pos] = 1
    for j in range(m):
        got, budget = O.decrypt(cts[j], cd.s)
        assert got[0] == bits[j] and not got[1:].any() and budget > 0


def test_modified_expansion_equals_sealpir_expansion(orc):
    """App. B theorem: both expansion loops produce ciphertexts with the same
    decryptions, 2^c * sum_l mu_{i + l 2^c} x^{l 2^c} for output i."""
    N, c = 32, 3
    O, q, cd, rlk = small_setup(orc, N, 2)
    gk = galois_keys(O, cd, N, c)
    mu = syn.Stream(41).below(T, N).astype(np.uint32)
    (ct,) = encrypt_many(O, cd, [mu])
    mod = O.expand(ct[None], c, 1 << c, gk)
    seal = O.expand_sealpir(ct, c, gk)
    B = 1 << c
    for i in range(B):
        want = [0] * N
        for l in range(N // B):
            want[l * B] = (B * int(mu[i + l * B])) % T
        g1, _ = O.decrypt(mod[i], cd.s)
        g2, _ = O.decrypt(seal[i], cd.s)
        assert g1.tolist() == want and g2.tolist() == want
    # SealPIR with its final 2^-c scaling recovers the plain coefficients
    inv = pow(B, -1, T)
    g, _ = O.decrypt(O.scalar_mul(seal[3], inv), cd.s)
    assert g[0] == mu[3]


# ------------------------------------------------------------ equality operator
@pytest.mark.parametrize("m,k", [(6, 2), (8, 3), (8, 4)])
def test_cw_equality_operator_brute_force(orc, m, k):
    """Eq. plain-cw-eq: prod_{y[j]=1} Enc(x[j]) decrypts to 1 iff x == y,
    over every pair of codewords of CW(m, k)."""
    N = 16
    O, q, cd, rlk = small_setup(orc, N, 3)
    n = orc.binom(m, k)
    words = [orc.map_perfect(x, m, k) for x in range(n)]
    for xi, xw in enumerate(words):
        bits = np.zeros(m, np.uint32)
        bits[xw] = 1
        mus = []
        for j in range(m):
            v = np.zeros(N, np.uint32)
            v[0] = bits[j]
            mus.append(v)
        ctxts = np.stack(encrypt_many(O, cd, mus, stream=xi))
        for yi, yw in enumerate(words):
            got, budget = O.decrypt(O.selection(ctxts, yw, rlk), cd.s)
            assert got[0] == (1 if xi == yi else 0) and not got[1:].any()
            assert budget > 0


def test_one_minus_decrypts_to_complement(orc):
    """The factor (1 - x[i]) of Eq. folklore-plain-eq: the constant plaintext
    1 minus a ciphertext of mu decrypts to 1 - mu (mod t), coefficient-wise."""
    N = 64
    O, q, cd, rlk = small_setup(orc, N, 2)
    mu = syn.payload(syn.Stream(81), 1, N, T)[0]
    ct = encrypt_many(O, cd, [mu], stream=5)[0]
    got, budget = O.decrypt(O.one_minus(ct), cd.s)
    want = [(-int(v)) % T for v in mu]
    want[0] = (1 - int(mu[0])) % T
    assert got.tolist() == want and budget > 0


@pytest.mark.parametrize("ell", [1, 3])
def test_folklore_equality_operator_brute_force(orc, ell):
    """Eq. folklore-plain-eq: prod_{y[i]=0} (1 - Enc(x[i])) prod_{y[i]=1}
    Enc(x[i]) decrypts to 1 iff x == y, for every pair of ell-bit values."""
    N = 16
    O, q, cd, rlk = small_setup(orc, N, 3)
    for x in range(1 << ell):
        mus = []
        for i in range(ell):
            v = np.zeros(N, np.uint32)
            v[0] = (x >> i) & 1
            mus.append(v)
        leaves = O.folklore_leaves(np.stack(encrypt_many(O, cd, mus, stream=90 + x)))
        for y in range(1 << ell):
            pos = orc.folklore_codeword(y, ell)
            assert pos.tolist() == [2 * i + ((y >> i) & 1) for i in range(ell)]
            got, budget = O.decrypt(O.selection(leaves, pos, rlk), cd.s)
            assert got[0] == (1 if x == y else 0) and not got[1:].any() and budget > 0


def test_batch_encoding_is_a_ring_isomorphism(orc):
    """SIMD batch encoding (Sec. 4: all circuits run slot-wise): decoding
    inverts encoding, the negacyclic product mod t of two encodings decodes
    to the slot-wise product (schoolbook in Python integers), and the
    constant polynomial j fills every slot with j."""
    N = 64
    O, q, cd, rlk = small_setup(orc, N, 2)
    st = syn.Stream(83)
    v = st.below(T, N).astype(np.uint32)
    w = st.below(T, N).astype(np.uint32)
    ev, ew = O.batch_encode(v), O.batch_encode(w)
    assert np.array_equal(O.batch_decode(ev), v)
    prod = np.array(schoolbook_nega([int(a) for a in ev], [int(b) for b in ew], T), np.uint32)
    assert np.array_equal(O.batch_decode(prod), (v.astype(np.uint64) * w % T).astype(np.uint32))
    const = np.zeros(N, np.uint32)
    const[0] = 7
    assert np.array_equal(O.batch_decode(const), np.full(N, 7, np.uint32))


@pytest.mark.parametrize("m,k", [(6, 2), (5, 3)])
def test_arith_cw_equality_operator_brute_force(orc, m, k):
    """Alg. Arithmetic Constant-weight Equality Operator, Theorem: with both
    operands encrypted and batch-encoded (slot s holds the pair (x_s, y_s)),
    the output decrypts to 1 in exactly the slots where x_s == y_s, over
    every pair of codewords of CW(m, k)."""
    N = 256
    O, q, cd, rlk = small_setup(orc, N, 3)
    words = [orc.map_perfect(i, m, k) for i in range(orc.binom(m, k))]
    pairs = [(a, b) for a in range(len(words)) for b in range(len(words))]
    assert len(pairs) <= N
    xb = np.zeros((m, N), np.uint32)
    yb = np.zeros((m, N), np.uint32)
    for s, (a, b) in enumerate(pairs):
        xb[words[a], s] = 1
        yb[words[b], s] = 1
    x = np.stack(encrypt_many(O, cd, [O.batch_encode(r) for r in xb], stream=1))
    y = np.stack(encrypt_many(O, cd, [O.batch_encode(r) for r in yb], stream=2))
    mu, budget = O.decrypt(O.arith_cw_eq(m, k, x, y, rlk), cd.s)
    e = O.batch_decode(mu)
    want = np.zeros(N, np.uint32)
    for s, (a, b) in enumerate(pairs):
        want[s] = 1 if a == b else 0
    assert np.array_equal(e, want) and budget > 0


# ------------------------------------------------------------ PIR answers
def run_pir(orc, O, cd, rlk, items, ids, target_id, m, k, c, gk=None, nthreads=0):
    cw = np.stack([orc.map_perfect(int(i), m, k) for i in ids])
    qpos = orc.map_perfect(int(target_id), m, k)
    h = -(-m // (1 << c))
    a, e = cd.encryption(h, 77)
    query = O.make_query(qpos, m, c, cd.s, a, e)
    resp = O.answer(items, cw, m, query, rlk, c=c, gkeys=gk, nthreads=nthreads)
    return O.decrypt(resp, cd.s)


def test_index_pir_returns_selected_row(orc):
    N, L = 64, 2
    O, q, cd, rlk = small_setup(orc, N, L)
    n, k = 40, 2
    m = orc.code_length(6, k)  # 2^6 >= 40
    items = syn.payload(syn.Stream(51), n, N, T)
    for target in (0, 17, n - 1):
        got, budget = run_pir(orc, O, cd, rlk, items, range(n), target, m, k, 0)
        assert np.array_equal(got, items[target]) and budget > 0


def test_keyword_pir_present_and_absent(orc):
    """Sec. 3.3.6: codewords of the keywords present; an absent keyword's
    response decrypts to all zeros."""
    N, L = 64, 3
    O, q, cd, rlk = small_setup(orc, N, L)
    k, m, c = 3, 12, 2  # C(12,3) = 220 >= 2^7 keywords of 7 bits
    st = syn.Stream(52)
    ids = np.array(sorted(set(st.below(128, 40).tolist())))[:20]
    items = syn.payload(st, len(ids), 48, 1 << 16)
    gk = galois_keys(O, cd, N, c)
    got, budget = run_pir(orc, O, cd, rlk, items, ids, ids[5], m, k, c, gk)
    want = np.zeros(N, np.uint32)
    want[:48] = items[5]
    assert np.array_equal(got, want) and budget > 0
    absent = next(v for v in range(128) if v not in set(ids.tolist()))
    got, budget = run_pir(orc, O, cd, rlk, items, ids, absent, m, k, c, gk)
    assert not got.any() and budget > 0


def test_multi_plaintext_rows_return_every_plaintext(orc):
    """Sec. 3.3.1 / 3.3.3: a row of s plaintexts is answered by s inner
    products with one selection vector; response p decrypts to plaintext p
    of the selected row (the last one zero-padded), for a present index and
    for rows the query does not select."""
    N, L = 64, 2
    O, q, cd, rlk = small_setup(orc, N, L)
    n, k = 30, 2
    m = orc.code_length(5, k)
    plen = 2 * N + 21  # three plaintexts, the third ragged
    items = syn.payload(syn.Stream(53), n, plen, T)
    cw = np.stack([orc.map_perfect(i, m, k) for i in range(n)])
    for target in (0, 13, n - 1):
        a, e = cd.encryption(m, 80 + target)
        query = O.make_query(orc.map_perfect(target, m, k), m, 0, cd.s, a, e)
        resp = O.answer(items, cw, m, query, rlk)
        assert resp.shape == (3, 2, L, N)
        want = np.zeros(3 * N, np.uint32)
        want[:plen] = items[target]
        for p in range(3):
            got, budget = O.decrypt(resp[p], cd.s)
            assert np.array_equal(got, want[p * N:(p + 1) * N]) and budget > 0, (target, p)


def test_folklore_pir_returns_selected_row(orc):
    """Folklore PIR (Sec. 4): the query is the ell encrypted bits of the
    index; the server forms the 2 ell leaves and the plain folklore operator
    per row.  n = 13 rows (a ragged last power of two), ell = 4."""
    N, L = 64, 3
    O, q, cd, rlk = small_setup(orc, N, L)
    n, ell = 13, 4
    items = syn.payload(syn.Stream(82), n, N, T)
    cw = np.stack([orc.folklore_codeword(i, ell) for i in range(n)])
    for target in (0, 6, n - 1):
        mus = []
        for i in range(ell):
            v = np.zeros(N, np.uint32)
            v[0] = (target >> i) & 1
            mus.append(v)
        query = O.folklore_leaves(np.stack(encrypt_many(O, cd, mus, stream=100 + target)))
        got, budget = O.decrypt(O.answer(items, cw, 2 * ell, query, rlk), cd.s)
        assert np.array_equal(got, items[target]) and budget > 0


def test_c1_full_answer_decrypts_with_positive_budget(orc):
    """Workload of the first configuration: n=256, k=2, m=24, N=4096, two
    54-bit primes, t=65537."""
    N = 4096
    q = [int(p) for p in orc.primes(N, 2)]
    O = orc.Oracle(N, q)
    cd = syn.ClientDraws(1, q, N)
    a, e = cd.relin()
    rlk = O.keygen_relin(cd.s, a, e)
    items = syn.payload(syn.Stream(2), 256, N, T)
    target = int(syn.Stream(3).below(256, 1)[0])
    got, budget = run_pir(orc, O, cd, rlk, items, range(256), target, 24, 2, 0)
    assert np.array_equal(got, items[target])
    assert budget > 0


@pytest.mark.parametrize("N,L,n,k,m,c,seeds,domain", [
    (8192, 4, 65536, 4, 37, 0, (11, 12, 13), 65536),   # index PIR, configuration 2
    (16384, 7, 16384, 8, 64, 6, (21, 22, 23), 1 << 32),  # keyword PIR, configuration 3
])
def test_full_size_answers_keep_a_positive_budget(orc, N, L, n, k, m, c, seeds, domain):
    """Decryption of the full answers of the second and third
    configurations, bounded without computing them.  The answer is the sum
    over the n rows of sel_i * DB_i (Sec. 3.3.3); the invariant noise of a
    sum of ciphertexts is the sum of their invariant noises while that sum
    stays below Q/2, so its budget is at least the smallest row term's
    budget minus log2 n.  The row terms are computed for the target row and
    rows whose codewords share 0 ... k-1 positions with the target's (the
    number of factors that encrypt 1); each must decrypt to the row or to
    zero and leave more than 16 bits after the log2 n of the sum."""
    q = [int(p) for p in orc.primes(N, L)]
    O = orc.Oracle(N, q)
    cd = syn.ClientDraws(seeds[0], q, N)
    a, e = cd.relin()
    rlk = O.keygen_relin(cd.s, a, e)
    st = syn.Stream(seeds[2])
    target = int(st.below(domain, 1)[0])
    qpos = orc.map_perfect(target, m, k)
    a, e = cd.encryption(-(-m // (1 << c)), 77)
    query = O.make_query(qpos, m, c, cd.s, a, e)
    cts = O.expand(query, c, m, galois_keys(O, cd, N, c)) if c else query
    rows, overlaps = [target], {k}
    for x in st.below(domain, 4096).tolist():
        ov = len(set(orc.map_perfect(int(x), m, k).tolist()) & set(qpos.tolist()))
        if ov not in overlaps and len(rows) < 4:
            overlaps.add(ov)
            rows.append(int(x))
    assert len(rows) == 4
    payload = syn.payload(syn.Stream(seeds[1]), len(rows), 8192, 1 << 16)
    worst = math.inf
    for i, x in enumerate(rows):
        term = O.plain_mul(O.selection(cts, orc.map_perfect(x, m, k), rlk), payload[i])
        mu, budget = O.decrypt(term, cd.s)
        want = np.zeros(N, np.uint32)
        if x == target:
            want[:8192] = payload[i]
        assert np.array_equal(mu, want), x
        worst = min(worst, budget)
    assert worst - math.log2(n) > 16


# ------------------------------------------------------------ mappings
@pytest.mark.parametrize("m,k", [(10, 3), (12, 5), (9, 1), (7, 7)])
def test_perfect_mapping_roundtrip_and_order(orc, m, k):
    """Alg. Perfect Mapping and its inverse (App. A): a bijection [C(m,k)] ->
    CW(m,k) that is increasing in the bitmask value sum_j y[j] 2^j."""
    n = orc.binom(m, k)
    assert n == math.comb(m, k)
    prev = -1
    seen = set()
    for x in range(n):
        pos = orc.map_perfect(x, m, k)
        assert len(set(pos.tolist())) == k and list(pos) == sorted(pos)
        assert orc.map_inverse(pos) == x
        mask = sum(1 << int(p) for p in pos)
        assert mask > prev
        prev = mask
        seen.add(mask)
    # every weight-k mask below 2^m is hit
    assert len(seen) == n
    with pytest.raises(ValueError):
        orc.map_perfect(n, m, k)


def read_golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                rows.append(line)
    return rows


def splitmix64_outputs(seed: int, count: int):
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) from its definition:
    the 64-bit state advances by 0x9E3779B97F4A7C15 and each output is the
    state through the xor-shift-multiply finaliser."""
    mask = (1 << 64) - 1
    st, out = seed, []
    for _ in range(count):
        st = (st + 0x9E3779B97F4A7C15) & mask
        z = ((st ^ (st >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


@pytest.mark.parametrize("m,k", [(8, 2), (12, 5), (64, 8), (5, 5)])
def test_lossy_mapping_keeps_first_k_distinct_hash_positions(orc, m, k):
    """Alg. Lossy Mapping (App. A): the codeword's positions are the first k
    distinct values of H_1(x), H_2(x), ... (here the SplitMix64 outputs of
    seed x, mod m), ascending; exactly k positions below m."""
    st = syn.Stream(71)
    xs = [int(v) for v in st.words(200)] + [0, 1, (1 << 64) - 1]
    for x in xs:
        want = []
        for h in splitmix64_outputs(x, 64 * m + 1024):
            if h % m not in want:
                want.append(h % m)
            if len(want) == k:
                break
        assert orc.map_lossy(x, m, k).tolist() == sorted(want)


@pytest.mark.parametrize("m,k", [(8, 2), (7, 3), (10, 4)])
def test_lossy_mapping_codewords_are_uniform(orc, m, k):
    """Theorem lossy-coll-prob: every codeword of CW(m,k) is hit with
    probability 1/C(m,k), so two different elements collide with that
    probability.  Chi-square of 100000 mapped elements against the uniform
    distribution (bound about 8 standard deviations above its mean), and the
    pairwise collision rate within 10% of 1/C(m,k)."""
    from collections import Counter

    n = 100000
    xs = syn.Stream(72).words(n)
    cnt = Counter(tuple(orc.map_lossy(int(x), m, k).tolist()) for x in xs)
    cells = math.comb(m, k)
    assert len(cnt) == cells
    exp = n / cells
    chi2 = sum((cnt.get(c, 0) - exp) ** 2 / exp for c in cnt)
    df = cells - 1
    assert chi2 < df + 8 * math.sqrt(2 * df), chi2
    coll = sum(v * (v - 1) for v in cnt.values()) / (n * (n - 1))
    assert abs(coll * cells - 1) < 0.1, coll * cells


def test_code_lengths_reproduce_paper_encoding_size_table(orc):
    for row in read_golden("encoding_size.txt"):
        bits = int(row[0])
        for k, v in zip((1, 2, 3, 4), row[1:]):
            if v == "-":
                continue
            assert orc.code_length(bits, k) == int(v), (bits, k)


def test_code_lengths_reproduce_paper_pir_table(orc):
    for n, m in read_golden("packed_pir_code_length.txt"):
        n, m = int(n), int(m)
        bits = n.bit_length() - 1
        assert 1 << bits == n
        assert orc.code_length(bits, 2) == m


def test_keyword_code_weight_8_length_64():
    """32-bit keywords with k = 8 need m = 64: C(64,8) >= 2^32 > C(63,8)."""
    assert math.comb(64, 8) >= 1 << 32 > math.comb(63, 8)
    assert math.comb(37, 4) >= 1 << 16 > math.comb(36, 4)
