"""The CUDA kernels' arithmetic, run on the CPU through the test-only
emulator (tests/emu), against the oracle and exact integers.

These need no GPU: they check the modular arithmetic, the exact base
conversion (including the values next to Q/2 that take the mixed-radix
path), the exact scale-down and the order of the multiplication steps.
"""
import math

import numpy as np
import pytest

from paper_2202_07569_gb300 import synthetic as syn
from tests import emu

T = 65537


def centered(x, M):
    return x - M if x > M // 2 else x


def _ext_primes(N, L, q):
    """The library's extension primes: 30-bit, = 1 mod 2N, with product
    at least 2 N Q^2 (the tensor alone) and above 2^17 t N Q (the exact
    scale-down's bound)."""
    k = emu.lib().emu_ext_count(L)
    p = np.zeros(k, np.uint64)
    emu.lib().emu_ext_primes(N, L, np.array(q, np.uint64), p)
    p = [int(v) for v in p]
    assert all((1 << 29) < v < (1 << 30) and v % (2 * N) == 1 for v in p)
    assert math.prod(p) > (1 << 17) * T * N * math.prod(q)
    assert math.prod(p) >= 2 * N * math.prod(q) ** 2
    return p


@pytest.mark.parametrize("L", range(1, 9))
def test_extension_basis_covers_every_accepted_parameter_set(L):
    """The tensor of two centered lifts is at most N Q^2 / 2 in magnitude,
    so the extension basis alone holds it exactly, with v read by rounding,
    while P >= 2 N Q^2; the exact scale-down needs P > 2^17 t N Q.  The
    library accepts t < 2^20, N <= 16384 and ciphertext primes below 2^54,
    so the K(L) extension primes must exceed 2 N 2^(108 L) and
    2^17 2^20 N 2^(54 L) at every N, and be distinct 30-bit primes = 1 mod
    2N; one prime fewer must not reach the first bound at N = 16384 (K is
    the smallest such count)."""
    k = emu.lib().emu_ext_count(L)
    for logn in range(10, 15):
        N = 1 << logn
        p = np.zeros(k, np.uint64)
        emu.lib().emu_ext_primes(N, L, np.zeros(L, np.uint64), p)
        p = [int(v) for v in p]
        assert len(set(p)) == k
        for v in p:
            assert (1 << 29) < v < (1 << 30) and v % (2 * N) == 1
            assert all(v % d for d in range(3, 1 << 15, 2)), v
        assert math.prod(p) > 1 << (17 + 20 + logn + 54 * L), (N, L)
        assert math.prod(p) >= 1 << (1 + logn + 108 * L), (N, L)
        if logn == 14:
            assert math.prod(p[:-1]) < 1 << (1 + logn + 108 * L), (N, L)


@pytest.mark.parametrize("L", range(1, 9))
def test_row_basis_group_sizes_over_the_accepted_parameters(orc, L):
    """Rows per group that the row basis holds exactly: with four row
    primes at least 2048 (a whole launch's group cap) for every N and the
    largest t the library accepts; with three primes at t = 65537 at least
    63, so the three-prime basis serves the default t everywhere."""
    t_max = max(v for v in range((1 << 20) - 64, 1 << 20) if orc.is_prime(v))
    for logn in range(10, 15):
        N = 1 << logn
        q = np.array(orc.primes(N, L), np.uint64)
        assert emu.lib().emu_row_limit(N, L, q, t_max, 4) >= 2048, (N, L)
        assert emu.lib().emu_row_limit(N, L, q, T, 3) >= 63, (N, L)


def _setup(orc, N, L, seed=3):
    q = orc.primes(N, L)
    O = orc.Oracle(N, q)
    cd = syn.ClientDraws(seed, q, N)
    a, e = cd.relin()
    rlk = O.keygen_relin(cd.s, a, e)
    return q, O, cd, rlk


@pytest.mark.parametrize("N,L", [(1024, 1), (1024, 3), (4096, 2), (8192, 4)])
@pytest.mark.parametrize("force_exact", [0, 1])
def test_emulated_multiplication_matches_oracle(orc, N, L, force_exact):
    """The kernels' multiplication (tensor on the extension limbs alone,
    scale-down from them, key switch) equals the oracle's; with force_exact
    every scale-down coefficient takes the exact path instead."""
    q, O, cd, rlk = _setup(orc, N, L)
    st = syn.Stream(5, N + L)
    a = syn.uniform_residues(st, q, (2,), N)
    b = syn.uniform_residues(st, q, (2,), N)
    out = np.zeros((2, L, N), np.uint64)
    bad = emu.lib().emu_bfv_mul(N, L, q, T, np.ascontiguousarray(rlk), a, b, out, force_exact)
    assert bad == 0
    assert np.array_equal(out, O.bfv_mul(a, b, rlk))


def test_emulated_multiplication_matches_oracle_n16384(orc):
    q, O, cd, rlk = _setup(orc, 16384, 7)
    st = syn.Stream(6)
    a = syn.uniform_residues(st, q, (2,), 16384)
    b = syn.uniform_residues(st, q, (2,), 16384)
    out = np.zeros((2, 7, 16384), np.uint64)
    assert emu.lib().emu_bfv_mul(16384, 7, q, T, np.ascontiguousarray(rlk), a, b, out, 0) == 0
    assert np.array_equal(out, O.bfv_mul(a, b, rlk))


@pytest.mark.parametrize("N,L", [(1024, 2), (2048, 3), (8192, 4), (16384, 7), (16384, 8)])
def test_centered_lift_near_half(orc, N, L):
    """Values next to Q/2 and 0 take the exact mixed-radix branch."""
    q = [int(v) for v in orc.primes(N, L)]
    Q = math.prod(q)
    p = _ext_primes(N, L, q)
    vals = [0, 1, Q - 1, (Q - 1) // 2, (Q + 1) // 2, (Q - 3) // 2, (Q + 3) // 2]
    vals += [(Q >> 1) + d for d in (-(1 << 12), 1 << 12)]
    st = syn.Stream(7)
    vals += [int(w) * (Q >> 64) for w in st.words(5)]
    for x in vals:
        res = np.array([x % qq for qq in q], np.uint64)
        y = np.zeros(len(p), np.uint64)
        emu.lib().emu_lift(N, L, np.array(q, np.uint64), T, res, y)
        xc = centered(x, Q)
        assert [int(v) for v in y] == [xc % pp for pp in p], x


@pytest.mark.parametrize("N,L", [(1024, 2), (2048, 3), (8192, 4), (16384, 7), (16384, 8)])
def test_exact_scale_down(orc, N, L):
    """round(t d / Q) for extreme and near-tie d, including t d = (Q +- 1)/2
    (mod Q), which takes the mixed-radix branch."""
    q = [int(v) for v in orc.primes(N, L)]
    Q = math.prod(q)
    p = _ext_primes(N, L, q)
    dmax = 2 * N * (Q // 2) ** 2
    inv_t = pow(T, -1, Q)
    ds = [0, 1, -1, dmax, -dmax, dmax - 12345, -(dmax // 3)]
    for r in ((Q - 1) // 2, (Q + 1) // 2, (Q - 5) // 2):
        base = (r * inv_t) % Q
        ds += [base, base - Q, base + 7 * Q, base - 11 * Q]
    st = syn.Stream(8)
    for w in st.words(10).tolist():
        ds.append((int(w) * dmax) >> 64)
        ds.append(-((int(w) * dmax) >> 65))
    qa = np.array(q, np.uint64)
    for i, d in enumerate(ds):
        assert abs(d) <= dmax
        # the kernels hand over N d in lazy form: residues in [0, 2q),
        # here each residue plus 0 or 1 times its prime
        dq = np.array([(N * d) % v + (i + j) % 2 * v for j, v in enumerate(q)], np.uint64)
        dp = np.array([(N * d) % v + (i + j + 1) % 2 * v for j, v in enumerate(p)],
                      np.uint64)
        out = np.zeros(L, np.uint64)
        assert emu.lib().emu_scale(N, L, qa, T, dq, dp, out) == 1
        num = T * d
        want = (num + Q // 2) // Q  # nearest integer: Q odd, no ties
        assert [int(v) for v in out] == [want % v for v in q], d


@pytest.mark.parametrize("N,L", [(1024, 1), (2048, 3), (8192, 4), (16384, 7), (16384, 8)])
def test_scale_down_from_the_extension_basis(orc, N, L):
    """round(t d / Q) mod q_j from the residues of N d modulo the extension
    primes alone.  Extreme d, random d, and d whose t d / Q lies within
    t / Q of a half integer (the fast path must hand those to the exact
    path); each through the fast path with its hand-over and, separately,
    through the exact path alone, against exact integers."""
    q = [int(v) for v in orc.primes(N, L)]
    Q = math.prod(q)
    p = _ext_primes(N, L, q)
    K = len(p)
    dmax = N * Q * Q // 2
    ds = [0, 1, -1, dmax, -dmax, dmax - 1, 1 - dmax]
    st = syn.Stream(9)
    ties = []
    for w in st.words(12).tolist():
        n = (int(w) * (T * dmax // Q)) >> 64  # t d / Q next to n + 1/2
        base = ((2 * n + 1) * Q) // (2 * T)
        for d in (base - 1, base, base + 1, -base, -base - 1):
            if abs(d) <= dmax:
                ties.append(len(ds))
                ds.append(d)
    for w in st.words(60).tolist():
        ds.append(((int(w) * 2 * dmax) >> 64) - dmax)
    # lazy residues as the tensor kernel leaves them: [0, 2p)
    dp = np.array([[(N * d) % v + (i + k) % 2 * v for k, v in enumerate(p)]
                   for i, d in enumerate(ds)], np.uint32)
    want = [[((T * d + Q // 2) // Q) % v for v in q] for d in ds]
    qa = np.array(q, np.uint64)
    for force in (0, 1):
        out = np.zeros((len(ds), L), np.uint64)
        path = np.zeros(len(ds), np.int32)
        emu.lib().emu_scale_p(N, L, qa, T, len(ds), dp, out, force, path)
        assert [[int(v) for v in row] for row in out] == want
        assert set(path.tolist()) <= ({0, 1} if not force else {1})
        if not force:
            assert all(path[i] == 1 for i in ties)
            assert (path[len(ds) - 60:] == 0).all()

def test_reduction_below_2_62(orc):
    """The 32-bit reduction of sums below 2^62 modulo a 30-bit extension
    prime: values at 0, 2^62 - 1, next to multiples of p and of 2^32, and
    random ones, against Python integers."""
    for N, L in ((1024, 1), (16384, 8)):
        for p in _ext_primes(N, L, [int(v) for v in orc.primes(N, L)]):
            vals = [0, 1, p - 1, p, p + 1, (1 << 32) - 1, 1 << 32, (1 << 62) - 1,
                    ((1 << 62) // p) * p, ((1 << 62) // p) * p - 1, (1 << 61) + 12345]
            vals += [int(w) >> 2 for w in syn.Stream(12, p % 1000).words(64).tolist()]
            v = np.array(vals, np.uint64)
            out = np.zeros(len(vals), np.uint32)
            emu.lib().emu_reduce62(p, v, len(vals), out)
            assert [int(x) for x in out] == [x % p for x in vals]


@pytest.mark.parametrize("nr", [3, 4])
@pytest.mark.parametrize("N,L", [(1024, 1), (8192, 4), (16384, 7), (16384, 8)])
def test_row_basis_crt(orc, N, L, nr):
    """Sums of row products recovered modulo the ciphertext primes from N x
    modulo the nr row primes (the first nr extension primes), for |x| up to
    the bound that the rows-per-group limit guarantees (rows N q_max (t-1)/2
    for that many rows), including the extremes and lazy residues below 2r."""
    q = [int(v) for v in orc.primes(N, L)]
    r = _ext_primes(N, L, q)[:nr]
    R = math.prod(r)
    rows = int(emu.lib().emu_row_limit(N, L, np.array(q, np.uint64), T, nr))
    assert rows >= (32 if nr == 3 else 2048)
    xmax = min(rows, 1 << 30) * N * max(q) * ((T - 1) // 2)
    assert 2 * xmax < R  # the limit keeps the sums inside the basis
    xs = [0, 1, -1, xmax, -xmax, xmax - 77, -(xmax // 3)]
    st = syn.Stream(11, N + L + nr)
    for w in st.words(12).tolist():
        xs.append((int(w) * xmax) >> 64)
        xs.append(-((int(w) * xmax) >> 64))
    for i, x in enumerate(xs):
        xr = np.array([(N * x) % rk + (rk if (i + k) % 3 == 0 else 0)
                       for k, rk in enumerate(r)] + [0] * (4 - nr), np.uint32)
        out = np.zeros(L, np.uint64)
        assert emu.lib().emu_row_crt(N, L, np.array(q, np.uint64), T, nr, xr, out) == 0
        assert [int(v) for v in out] == [x % qq for qq in q], x


@pytest.mark.parametrize("logn,L", [(13, 4), (14, 7)])
def test_tensor_inverse_schedules(orc, logn, L):
    """The tensor kernel's inverse transforms at N = 8192 and 16384: the
    32-bit schedule that runs the three outputs in lock-step, with the
    kernel's shared-memory slots in each exchange, equals three single
    transforms for every extension prime."""
    q = orc.primes(1 << logn, L)
    data = syn.Stream(13).words(8192)
    assert emu.lib().emu_tensor_intt_compare(logn, L, np.array(q, np.uint64), T, data) == 0


@pytest.mark.parametrize("N,L", [(1024, 2), (8192, 4), (16384, 7), (16384, 8)])
def test_key_switch_basis_crt(orc, N, L):
    """The key switch of the internal tree nodes sums the products of the
    L digits D_i < q_i with the key limbs < q_j as integer polynomials in
    the basis of the first five extension primes: |x| < L N q_max^2.  x is
    recovered modulo every q_j from N x modulo the five primes at that
    bound, its negative and values in between, with lazy residues."""
    q = [int(v) for v in orc.primes(N, L)]
    r = _ext_primes(N, L, q)[:5]
    R = math.prod(r)
    xmax = L * N * max(q) ** 2
    assert 2 * xmax < R * (1 - 2.0 ** -23)  # the basis holds every sum
    xs = [0, 1, -1, xmax, -xmax, xmax - 12345, -(xmax // 7)]
    st = syn.Stream(12, N + L)
    for w in st.words(12).tolist():
        xs.append((int(w) * xmax) >> 64)
        xs.append(-((int(w) * xmax) >> 64))
    for i, x in enumerate(xs):
        xr = np.array([(N * x) % rk + (rk if (i + k) % 2 == 0 else 0)
                       for k, rk in enumerate(r)], np.uint32)
        out = np.zeros(L, np.uint64)
        assert emu.lib().emu_row_crt(N, L, np.array(q, np.uint64), T, 5, xr, out) == 0
        assert [int(v) for v in out] == [x % qq for qq in q], x


@pytest.mark.parametrize("N,L,nr", [(8192, 4, 3), (16384, 7, 3), (1024, 2, 4)])
def test_row_basis_sums_at_the_group_limit(orc, N, L, nr):
    """The row path of the last tree level (transforms modulo the row
    primes, row products summed over a group, inverse transform, exact CRT)
    returns sum_r z_r * lift(db_r) mod q_j for a full group of rows at the
    extremes the limit allows: every limb word at q_max - 1 and every row
    coefficient at +-(t-1)/2, whose negacyclic sum has the closed form
    x_i = rows z d (2i + 2 - N), reaching rows N q_max (t-1)/2 at i = N-1.
    Twice the rows overflow the basis there, so the limit is within a factor
    two of the largest group the basis holds.  A random group is checked
    against the oracle's products."""
    q = [int(v) for v in orc.primes(N, L)]
    qa = np.array(q, np.uint64)
    rows = min(int(emu.lib().emu_row_limit(N, L, qa, T, nr)), 2048)
    zmax = max(q) - 1
    i = np.arange(N, dtype=object)

    def run(nrows, zval, v):
        z = np.full((nrows, N), zval, np.uint64)
        db = np.full((nrows, N), v, np.uint32)
        out = np.zeros((L, N), np.uint64)
        tripped = emu.lib().emu_row_sum(N, L, qa, T, nr, nrows, z, db, out)
        d = v - T if v > T // 2 else v
        x = nrows * zval * d * (2 * i + 2 - N)
        return out, tripped, x

    for v in ((T - 1) // 2, (T + 1) // 2):  # d = +(t-1)/2 and -(t-1)/2
        out, tripped, x = run(rows, zmax, v)
        assert tripped == 0
        for j, qj in enumerate(q):
            assert [int(w) for w in out[j]] == [int(w) % qj for w in x], (v, j)
    if nr == 3:
        out, tripped, x = run(2 * rows, zmax, (T - 1) // 2)
        assert tripped > 0 or int(out[0][N - 1]) != int(x[N - 1]) % q[0]

    st = syn.Stream(12, N + nr)
    nrand = 6
    z = st.below(max(q), nrand * N).reshape(nrand, N)
    db = syn.payload(st, nrand, N, T)
    out = np.zeros((L, N), np.uint64)
    assert emu.lib().emu_row_sum(N, L, qa, T, nr, nrand, z, db, out) == 0
    lift = [[int(v) - T if v > T // 2 else int(v) for v in row] for row in db]
    for j, qj in enumerate(q):
        want = np.zeros(N, np.uint64)
        for r in range(nrand):
            zr = np.array([int(w) % qj for w in z[r]], np.uint64)
            dr = np.array([w % qj for w in lift[r]], np.uint64)
            want = (want + orc.negacyclic_mul_mod(zr, dr, qj)) % np.uint64(qj)
        assert np.array_equal(out[j], want), j


def test_emulated_substitution_matches_oracle(orc):
    N, L = 1024, 3
    q, O, cd, rlk = _setup(orc, N, L)
    for gi, g in enumerate((N + 1, N // 4 + 1, 3)):
        a, e = cd.galois(gi)
        gk = O.keygen_galois(g, cd.s, a, e)
        ct = syn.uniform_residues(syn.Stream(9, g), q, (2,), N)
        out = np.zeros((2, L, N), np.uint64)
        emu.lib().emu_substitute(N, L, q, T, g, np.ascontiguousarray(gk), ct, out)
        assert np.array_equal(out, O.substitute(g, ct, gk))


@pytest.mark.parametrize("rb", [4, 5])
@pytest.mark.parametrize("N,L", [(1024, 2), (2048, 1), (4096, 2), (8192, 4), (16384, 3)])
def test_register_blocked_ntt_schedule_equals_stagewise(orc, N, L, rb):
    """The kernels' pass schedule (2^rb registers per thread, lazy
    reduction) gives the same forward and inverse transforms as the
    level-by-level butterflies, for every prime the library uses at this N,
    from lazy inputs below 4q (forward) and 2q (inverse)."""
    q = orc.primes(N, L)
    data = syn.Stream(10, N).words(N)
    assert emu.lib().emu_ntt_compare(N, L, q, T, data, rb) == 0
