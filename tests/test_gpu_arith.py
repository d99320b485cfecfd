"""Arithmetic constant-weight equality operator (Alg. Arithmetic
Constant-weight Equality Operator) on two encrypted, batch-encoded operands:
bit for bit against the oracle, and decrypting to 1 exactly in the slots
whose codewords agree."""
import numpy as np
import pytest

import oracle
from paper_2202_07569_gb300 import synthetic as syn
from tests.workloads import Client

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2202_07569_gb300 import build

    build.build()


def encrypt_rows(cl, rows, stream):
    a, e = cl.cd.encryption(len(rows), stream)
    return np.stack([cl.O.encrypt(cl.O.batch_encode(r), cl.cd.s, a[i], e[i])
                     for i, r in enumerate(rows)])


def test_arith_operator_all_pairs_cw62():
    N, L, m, k = 8192, 4, 6, 2
    cl = Client(N, L, seed=230)
    ctx = cl.context()
    words = [oracle.map_perfect(i, m, k) for i in range(15)]
    pairs = [(a, b) for a in range(15) for b in range(15)]
    xb = np.zeros((m, N), np.uint32)
    yb = np.zeros((m, N), np.uint32)
    for s, (a, b) in enumerate(pairs):
        xb[words[a], s] = 1
        yb[words[b], s] = 1
    x, y = encrypt_rows(cl, xb, 1), encrypt_rows(cl, yb, 2)
    got = ctx.arith_cw_eq(m, k, x, y)
    assert np.array_equal(got, cl.O.arith_cw_eq(m, k, x, y, cl.rlk))
    mu, budget = cl.decrypt(got)
    e = cl.O.batch_decode(mu)
    want = np.zeros(N, np.uint32)
    for s, (a, b) in enumerate(pairs):
        want[s] = 1 if a == b else 0
    assert np.array_equal(e, want) and budget > 0
    ctx.close()


@pytest.mark.parametrize("N,L,m,k", [(16384, 7, 11, 4), (4096, 2, 3, 1), (8192, 4, 9, 3)])
def test_arith_operator_bit_exact(N, L, m, k):
    """Uniform residues as operands: the same exact arithmetic on both sides
    (the products, the sum, the k factors, the tree and 1/k!)."""
    from paper_2202_07569_gb300 import binding as B

    cl = Client(N, L, seed=240 + k)
    ctx = cl.context()
    x = syn.uniform_ciphertexts(241 + k, cl.q, m, N)
    y = syn.uniform_ciphertexts(251 + k, cl.q, m, N)
    assert np.array_equal(ctx.arith_cw_eq(m, k, x, y), cl.O.arith_cw_eq(m, k, x, y, cl.rlk))
    with pytest.raises(B.CwpirError) as ei:
        ctx.arith_cw_eq(m, m + 1, x, y)
    assert ei.value.code == -1
    # a second call with the same (m, k) reuses the kept buffers and plans;
    # other operands, and the swapped operands
    x2 = syn.uniform_ciphertexts(261 + k, cl.q, m, N)
    assert np.array_equal(ctx.arith_cw_eq(m, k, x2, y), cl.O.arith_cw_eq(m, k, x2, y, cl.rlk))
    assert np.array_equal(ctx.arith_cw_eq(m, k, y, x2), cl.O.arith_cw_eq(m, k, y, x2, cl.rlk))
    # a residue at q_j (checked on the device) is rejected, and the next
    # call is unaffected
    bad = y.copy()
    bad[m - 1, 1, L - 1, N - 1] = cl.q[L - 1]
    with pytest.raises(B.CwpirError) as ei:
        ctx.arith_cw_eq(m, k, x, bad)
    assert ei.value.code == -1
    assert np.array_equal(ctx.arith_cw_eq(m, k, x, y), cl.O.arith_cw_eq(m, k, x, y, cl.rlk))
    ctx.close()
