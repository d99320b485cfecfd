"""Seeded synthetic inputs for the constant-weight PIR answer path.

This module holds no arithmetic of the method.  It only draws random
numbers, with the shapes and value distributions of the paper's workloads
(arXiv 2202.07569, Sec. 5 and 6: uniform payloads of 16-bit coefficients,
uniform keywords, a uniformly chosen target row), and the random inputs of
BFV key generation and encryption (uniform residues, a ternary secret,
centered-binomial errors).  Both the CUDA path's tests and the oracle draw
from here; the benchmark draws its inputs from here too.

Every draw comes from numpy's Philox-4x64 counter-based generator (Salmon
et al., SC'11) keyed directly with (seed, stream); only its raw 64-bit words
are used and every transform is written out below, so a draw is the same on
any platform and numpy version.
"""
from __future__ import annotations

import numpy as np


class Stream:
    """A keyed stream of raw 64-bit words."""

    def __init__(self, seed: int, stream: int = 0):
        self.seed, self.stream = int(seed), int(stream)
        self._bg = np.random.Philox(key=np.array([seed, stream], dtype=np.uint64))

    def words(self, n: int) -> np.ndarray:
        if n == 0:
            return np.zeros(0, np.uint64)
        return np.asarray(self._bg.random_raw(n), dtype=np.uint64)

    def below(self, bound: int, n: int) -> np.ndarray:
        """n values uniform in [0, bound) by rejection on masked words."""
        bound = int(bound)
        if bound <= 0:
            raise ValueError("bound must be positive")
        bits = max(1, (bound - 1).bit_length())
        mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        out = np.empty(n, np.uint64)
        have = 0
        while have < n:
            need = n - have
            w = self.words(need + need // 2 + 16) & mask
            w = w[w < np.uint64(bound)][:need]
            out[have:have + w.size] = w
            have += w.size
        return out


def uniform_residues(st: Stream, primes, lead_shape, N: int) -> np.ndarray:
    """Uniform element(s) of R_Q in RNS form: shape lead_shape + (L, N).

    A uniform value mod Q is the same as independent uniform residues mod
    each prime (CRT)."""
    primes = [int(p) for p in np.asarray(primes).ravel()]
    lead_shape = tuple(lead_shape)
    count = int(np.prod(lead_shape)) if lead_shape else 1
    out = np.empty((count, len(primes), N), np.uint64)
    for c in range(count):
        for j, p in enumerate(primes):
            out[c, j] = st.below(p, N)
    return out.reshape(lead_shape + (len(primes), N))


def ternary(st: Stream, N: int) -> np.ndarray:
    """Secret key: coefficients uniform in {-1, 0, 1}."""
    v = st.below(3, N).astype(np.int64) - 1
    return v.astype(np.int8)


def cbd(st: Stream, shape, eta: int = 21) -> np.ndarray:
    """Centered binomial error: popcount of eta bits minus popcount of eta bits."""
    shape = tuple(np.atleast_1d(shape)) if not isinstance(shape, tuple) else shape
    n = int(np.prod(shape))
    w = st.words(n)
    m = np.uint64((1 << eta) - 1)
    lo = w & m
    hi = (w >> np.uint64(eta)) & m
    pc = lambda x: np.array([bin(int(v)).count("1") for v in x], dtype=np.int32)
    return (pc(lo) - pc(hi)).reshape(shape)


def payload(st: Stream, n: int, length: int, bound: int) -> np.ndarray:
    """n items of `length` coefficients uniform in [0, bound) as u32.

    A bound of 2^16 (16-bit coefficients) takes four coefficients from each
    64-bit word, low half-word first; other bounds use rejection sampling."""
    count = n * length
    if bound == 1 << 16:
        w = st.words((count + 3) // 4).astype("<u8")
        return w.view("<u2")[:count].astype(np.uint32).reshape(n, length)
    return st.below(bound, count).astype(np.uint32).reshape(n, length)


def distinct_u32(st: Stream, n: int, exclude=None) -> np.ndarray:
    """n distinct uniform 32-bit keywords (optionally avoiding `exclude`)."""
    taken = set(int(x) for x in exclude) if exclude is not None else set()
    out = []
    seen = set()
    while len(out) < n:
        for v in st.words(max(16, 2 * (n - len(out)))):
            v = int(v) & 0xFFFFFFFF
            if v in seen or v in taken:
                continue
            seen.add(v)
            out.append(v)
            if len(out) == n:
                break
    return np.array(out, dtype=np.uint64)


class ClientDraws:
    """Random inputs of BFV key generation and query encryption.

    keys: secret s, relinearisation key randomness (a: [L][L][N], e: [L][N])
    and Galois key randomness per substitution element."""

    def __init__(self, seed: int, primes, N: int):
        self.seed, self.N = int(seed), int(N)
        self.primes = [int(p) for p in np.asarray(primes).ravel()]
        self.L = len(self.primes)
        st = Stream(seed, 0)
        self.s = ternary(st, N)

    def relin(self):
        st = Stream(self.seed, 1)
        a = uniform_residues(st, self.primes, (self.L,), self.N)
        e = cbd(st, (self.L, self.N))
        return a, e

    def galois(self, index: int):
        st = Stream(self.seed, 100 + int(index))
        a = uniform_residues(st, self.primes, (self.L,), self.N)
        e = cbd(st, (self.L, self.N))
        return a, e

    def encryption(self, h: int, stream: int = 0):
        st = Stream(self.seed, 1000 + int(stream))
        a = uniform_residues(st, self.primes, (h,), self.N)
        e = cbd(st, (h, self.N))
        return a, e


def uniform_ciphertexts(seed: int, primes, count: int, N: int) -> np.ndarray:
    """`count` uniform ciphertexts [count][2][L][N]: the distribution of fresh
    RLWE ciphertexts and keys, used where only shapes and timing matter."""
    return uniform_residues(Stream(seed, 7), primes, (count, 2), N)
