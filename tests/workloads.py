"""Seeded workloads of the five configurations, built from the synthetic
generators and the oracle's client (key generation and query encryption).

Used by the tests and the smoke check only.  Seeds follow one scheme per
configuration: keys, database, query.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2202_07569_gb300 import synthetic as syn

T = 65537

# name: N, L, n, k, m, c, payload_len, payload bound, keyword?, seeds
CONFIGS = {
    "c1": dict(N=4096, L=2, n=256, k=2, m=24, c=0, plen=4096, bound=T, keyword=False, seed=1),
    "c2": dict(N=8192, L=4, n=65536, k=4, m=37, c=0, plen=8192, bound=1 << 16, keyword=False,
               seed=11),
    "c3": dict(N=16384, L=7, n=16384, k=8, m=64, c=6, plen=8192, bound=1 << 16, keyword=True,
               seed=21),
}


class Client:
    """Keys (secret, relinearisation, Galois) for one parameter set."""

    def __init__(self, N: int, L: int, seed: int, c_max: int = 0):
        self.N, self.L = N, L
        self.q = oracle.primes(N, L)
        self.O = oracle.Oracle(N, self.q, T)
        self.cd = syn.ClientDraws(seed, self.q, N)
        a, e = self.cd.relin()
        self.rlk = self.O.keygen_relin(self.cd.s, a, e)
        self.galois = {}
        for i in range(c_max):
            g = N // (1 << i) + 1
            a, e = self.cd.galois(i)
            self.galois[g] = self.O.keygen_galois(g, self.cd.s, a, e)

    @property
    def gkeys(self):
        """Galois keys stacked by expansion round a (element N/2^a + 1)."""
        if not self.galois:
            return None
        return np.stack([self.galois[self.N // (1 << a) + 1] for a in range(len(self.galois))])

    def query(self, positions, m: int, c: int, stream: int = 0):
        h = -(-m // (1 << c))
        a, e = self.cd.encryption(h, stream)
        return self.O.make_query(positions, m, c, self.cd.s, a, e)

    def decrypt(self, ct):
        return self.O.decrypt(ct, self.cd.s)

    def context(self):
        from paper_2202_07569_gb300 import binding as B

        return B.Context(self.N, self.q, T, self.rlk, self.galois)


def database(n: int, plen: int, bound: int, k: int, m: int, seed: int, keyword: bool = False):
    """Rows, their codewords and (keyword DBs) their keywords."""
    st = syn.Stream(seed, 1)
    items = syn.payload(st, n, plen, bound)
    if keyword:
        ids = syn.distinct_u32(syn.Stream(seed, 2), n)
    else:
        ids = np.arange(n, dtype=np.uint64)
    cw = np.stack([oracle.map_perfect(int(x), m, k) for x in ids])
    return items, cw, ids
