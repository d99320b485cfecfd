"""Python handle on the plain C oracle (``cwpir_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
(``__graft_entry__.build`` compiles it) and by the CPU legs of ``bench.py``
(the CPU baseline and ``--impl reference``).  The product package never
imports this module, and this module never imports the product package.

The oracle follows the paper (arXiv 2202.07569) step by step; see the C
source for the section each function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cwpir_oracle.c")
_HDR = os.path.join(_HERE, "cwpir_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libcwpir_oracle.so")
_lock = threading.Lock()
_lib = None

u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libcwpir_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-Wall", "-Wextra", "-Wno-unused-parameter", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        l = C.CDLL(build())
        I, U32, U64 = C.c_int, C.c_uint32, C.c_uint64
        vp = C.c_void_p
        sig = {
            "orc_is_prime": (I, [U64]),
            "orc_primes": (I, [U32, U32, U32, u64p]),
            "orc_create": (vp, [U32, U32, u64p, U64]),
            "orc_destroy": (None, [vp]),
            "orc_aux_count": (U32, [vp]),
            "orc_negacyclic_mul_mod": (I, [U32, U64, u64p, u64p, u64p]),
            "orc_exact_product": (I, [vp, u64p, u64p, U32, i32p, u64p]),
            "orc_scale_round": (I, [vp, C.c_int32, u64p, U32, u64p]),
            "orc_tensor": (I, [vp, u64p, u64p, u64p]),
            "orc_keyswitch": (I, [vp, u64p, u64p, u64p]),
            "orc_bfv_mul": (I, [vp, u64p, u64p, u64p, u64p]),
            "orc_automorphism": (I, [vp, U32, u64p, u64p]),
            "orc_monomial": (I, [vp, C.c_int64, u64p, u64p]),
            "orc_substitute": (I, [vp, U32, u64p, u64p, u64p]),
            "orc_expand": (I, [vp, U32, u64p, U32, U32, u64p, u64p]),
            "orc_expand_sealpir": (I, [vp, u64p, U32, u64p, u64p]),
            "orc_scalar_mul": (I, [vp, u64p, U64, u64p]),
            "orc_one_minus": (I, [vp, u64p, u64p]),
            "orc_arith_cw_eq": (I, [vp, U32, U32, u64p, u64p, u64p, u64p]),
            "orc_batch_encode": (I, [vp, u32p, u32p]),
            "orc_batch_decode": (I, [vp, u32p, u32p]),
            "orc_folklore_codeword": (I, [U64, U32, u16p]),
            "orc_plain_mul": (I, [vp, u64p, u32p, U32, u64p]),
            "orc_selection": (I, [vp, u64p, u16p, U32, u64p, u64p]),
            "orc_answer": (I, [vp, U64, U32, u32p, u16p, U32, U32, U32, u64p,
                               u64p, vp, C.c_int, u64p]),
            "orc_keygen_relin": (I, [vp, i8p, u64p, i32p, u64p]),
            "orc_keygen_galois": (I, [vp, U32, i8p, u64p, i32p, u64p]),
            "orc_encrypt": (I, [vp, u32p, i8p, u64p, i32p, u64p]),
            "orc_make_query": (I, [vp, u16p, U32, U32, U32, i8p, u64p, i32p,
                                   u64p]),
            "orc_decrypt": (I, [vp, u64p, U32, i8p, u32p,
                                C.POINTER(C.c_double)]),
            "orc_binom": (None, [U64, U64, C.POINTER(U64), C.POINTER(U64)]),
            "orc_map_perfect": (I, [U64, U32, U32, u16p]),
            "orc_map_lossy": (I, [U64, U32, U32, u16p]),
            "orc_map_inverse": (I, [u16p, U32, C.POINTER(U64)]),
            "orc_code_length": (U64, [U32, U32, U64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
        return l


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def is_prime(p: int) -> bool:
    return bool(lib().orc_is_prime(p))


def primes(N: int, count: int, bits: int = 54) -> np.ndarray:
    out = np.zeros(count, np.uint64)
    _check(lib().orc_primes(N, count, bits, out), "primes")
    return out


def negacyclic_mul_mod(a, b, p: int) -> np.ndarray:
    a = _c(a, np.uint64)
    b = _c(b, np.uint64)
    out = np.zeros_like(a)
    _check(lib().orc_negacyclic_mul_mod(a.size, p, a, b, out), "negacyclic mul")
    return out


def binom(n: int, r: int) -> int:
    lo, hi = C.c_uint64(), C.c_uint64()
    lib().orc_binom(n, r, C.byref(lo), C.byref(hi))
    return lo.value | (hi.value << 64)


def map_perfect(x: int, m: int, k: int) -> np.ndarray:
    pos = np.zeros(k, np.uint16)
    _check(lib().orc_map_perfect(x, m, k, pos), "perfect map")
    return pos


def map_lossy(x: int, m: int, k: int) -> np.ndarray:
    pos = np.zeros(k, np.uint16)
    _check(lib().orc_map_lossy(x, m, k, pos), "lossy map")
    return pos


def folklore_codeword(y: int, ell: int) -> np.ndarray:
    pos = np.zeros(ell, np.uint16)
    _check(lib().orc_folklore_codeword(y, ell, pos), "folklore codeword")
    return pos


def map_inverse(pos) -> int:
    pos = _c(pos, np.uint16)
    x = C.c_uint64()
    _check(lib().orc_map_inverse(pos, pos.size, C.byref(x)), "inverse map")
    return x.value


def code_length(bits: int, k: int, limit: int = 1 << 22) -> int:
    return int(lib().orc_code_length(bits, k, limit))


class Oracle:
    """One parameter set (N, q, t) of the oracle."""

    def __init__(self, N: int, q, t: int = 65537):
        q = _c(q, np.uint64)
        self.N, self.L, self.t = int(N), int(q.size), int(t)
        self.q = q
        self._ctx = lib().orc_create(self.N, self.L, q, self.t)
        if not self._ctx:
            raise ValueError("oracle rejected the parameters")
        self.Q = 1
        for p in q.tolist():
            self.Q *= int(p)

    def __del__(self):
        ctx = getattr(self, "_ctx", None)
        if ctx and _lib is not None:
            _lib.orc_destroy(ctx)
            self._ctx = None

    # shapes
    @property
    def ct_shape(self):
        return (2, self.L, self.N)

    @property
    def key_shape(self):
        return (self.L, 2, self.L, self.N)

    @property
    def aux_count(self) -> int:
        return int(lib().orc_aux_count(self._ctx))

    def _ct(self, a):
        a = _c(a, np.uint64)
        return a

    def exact_product(self, a, b, words: int = 20):
        sign = np.zeros(self.N, np.int32)
        mag = np.zeros((self.N, words), np.uint64)
        _check(lib().orc_exact_product(self._ctx, _c(a, np.uint64),
                                       _c(b, np.uint64), words, sign, mag),
               "exact product")
        out = []
        for i in range(self.N):
            v = 0
            for w in reversed(mag[i].tolist()):
                v = (v << 64) | int(w)
            out.append(-v if sign[i] else v)
        return out

    def scale_round(self, d: int, words: int = 20) -> np.ndarray:
        mag = abs(int(d))
        arr = np.array([(mag >> (64 * i)) & ((1 << 64) - 1) for i in range(words)],
                       dtype=np.uint64)
        out = np.zeros(self.L, np.uint64)
        _check(lib().orc_scale_round(self._ctx, 1 if d < 0 else 0, arr, words, out),
               "scale round")
        return out

    def tensor(self, a, b) -> np.ndarray:
        out = np.zeros((3, self.L, self.N), np.uint64)
        _check(lib().orc_tensor(self._ctx, self._ct(a), self._ct(b), out), "tensor")
        return out

    def keyswitch(self, z, key) -> np.ndarray:
        out = np.zeros(self.ct_shape, np.uint64)
        _check(lib().orc_keyswitch(self._ctx, _c(z, np.uint64), _c(key, np.uint64),
                                   out), "keyswitch")
        return out

    def bfv_mul(self, a, b, rlk) -> np.ndarray:
        out = np.zeros(self.ct_shape, np.uint64)
        _check(lib().orc_bfv_mul(self._ctx, self._ct(a), self._ct(b),
                                 _c(rlk, np.uint64), out), "bfv mul")
        return out

    def automorphism(self, g: int, poly) -> np.ndarray:
        out = np.zeros((self.L, self.N), np.uint64)
        _check(lib().orc_automorphism(self._ctx, g, _c(poly, np.uint64), out),
               "automorphism")
        return out

    def monomial(self, e: int, poly) -> np.ndarray:
        out = np.zeros((self.L, self.N), np.uint64)
        _check(lib().orc_monomial(self._ctx, e, _c(poly, np.uint64), out), "monomial")
        return out

    def substitute(self, g: int, ct, gkey) -> np.ndarray:
        out = np.zeros(self.ct_shape, np.uint64)
        _check(lib().orc_substitute(self._ctx, g, self._ct(ct), _c(gkey, np.uint64),
                                    out), "substitute")
        return out

    def expand(self, query, c: int, m: int, gkeys) -> np.ndarray:
        query = _c(query, np.uint64).reshape(-1, 2, self.L, self.N)
        out = np.zeros((m, 2, self.L, self.N), np.uint64)
        _check(lib().orc_expand(self._ctx, query.shape[0], query, c, m,
                                _c(gkeys, np.uint64), out), "expand")
        return out

    def expand_sealpir(self, ct, c: int, gkeys) -> np.ndarray:
        out = np.zeros((1 << c, 2, self.L, self.N), np.uint64)
        _check(lib().orc_expand_sealpir(self._ctx, self._ct(ct), c,
                                        _c(gkeys, np.uint64), out), "expand sealpir")
        return out

    def scalar_mul(self, ct, scalar: int) -> np.ndarray:
        out = np.zeros(self.ct_shape, np.uint64)
        _check(lib().orc_scalar_mul(self._ctx, self._ct(ct), scalar, out), "scalar")
        return out

    def arith_cw_eq(self, m: int, k: int, x, y, rlk) -> np.ndarray:
        out = np.zeros(self.ct_shape, np.uint64)
        _check(lib().orc_arith_cw_eq(self._ctx, m, k, _c(x, np.uint64), _c(y, np.uint64),
                                     _c(rlk, np.uint64), out), "arithmetic CW operator")
        return out

    def batch_encode(self, slots) -> np.ndarray:
        slots = np.zeros(self.N, np.uint32) + _c(slots, np.uint32)
        mu = np.zeros(self.N, np.uint32)
        _check(lib().orc_batch_encode(self._ctx, slots, mu), "batch encode")
        return mu

    def batch_decode(self, mu) -> np.ndarray:
        slots = np.zeros(self.N, np.uint32)
        _check(lib().orc_batch_decode(self._ctx, _c(mu, np.uint32), slots), "batch decode")
        return slots

    def one_minus(self, ct) -> np.ndarray:
        out = np.zeros(self.ct_shape, np.uint64)
        _check(lib().orc_one_minus(self._ctx, self._ct(ct), out), "one minus")
        return out

    def folklore_leaves(self, query) -> np.ndarray:
        """(1 - x[0], x[0], 1 - x[1], x[1], ...) from the ell bit ciphertexts."""
        query = _c(query, np.uint64)
        return np.stack([v for ct in query for v in (self.one_minus(ct), ct)])

    def plain_mul(self, ct, mu) -> np.ndarray:
        mu = _c(mu, np.uint32)
        out = np.zeros(self.ct_shape, np.uint64)
        _check(lib().orc_plain_mul(self._ctx, self._ct(ct), mu, mu.size, out),
               "plain mul")
        return out

    def selection(self, ctxts, positions, rlk) -> np.ndarray:
        pos = _c(positions, np.uint16)
        out = np.zeros(self.ct_shape, np.uint64)
        _check(lib().orc_selection(self._ctx, _c(ctxts, np.uint64), pos, pos.size,
                                   _c(rlk, np.uint64), out), "selection")
        return out

    def answer(self, items, codewords, m: int, query, rlk, c: int = 0,
               gkeys=None, nthreads: int = 0) -> np.ndarray:
        items = _c(items, np.uint32)
        cw = _c(codewords, np.uint16)
        n, plen = items.shape
        k = cw.shape[1]
        s = max(1, -(-plen // self.N))  # plaintexts per row (Sec. 3.3.1)
        out = np.zeros(((s,) if s > 1 else ()) + self.ct_shape, np.uint64)
        gk = None
        if gkeys is not None:
            gkeys = _c(gkeys, np.uint64)
            gk = gkeys.ctypes.data
        _check(lib().orc_answer(self._ctx, n, plen, items, cw, k, m, c,
                                _c(query, np.uint64), _c(rlk, np.uint64), gk,
                                nthreads, out), "answer")
        return out

    # client side
    def keygen_relin(self, s, a, e) -> np.ndarray:
        out = np.zeros(self.key_shape, np.uint64)
        _check(lib().orc_keygen_relin(self._ctx, _c(s, np.int8), _c(a, np.uint64),
                                      _c(e, np.int32), out), "relin keygen")
        return out

    def keygen_galois(self, g: int, s, a, e) -> np.ndarray:
        out = np.zeros(self.key_shape, np.uint64)
        _check(lib().orc_keygen_galois(self._ctx, g, _c(s, np.int8), _c(a, np.uint64),
                                       _c(e, np.int32), out), "galois keygen")
        return out

    def encrypt(self, mu, s, a, e) -> np.ndarray:
        mu = np.zeros(self.N, np.uint32) + _c(mu, np.uint32)
        out = np.zeros(self.ct_shape, np.uint64)
        _check(lib().orc_encrypt(self._ctx, _c(mu, np.uint32), _c(s, np.int8),
                                 _c(a, np.uint64), _c(e, np.int32), out), "encrypt")
        return out

    def make_query(self, positions, m: int, c: int, s, a, e) -> np.ndarray:
        pos = _c(positions, np.uint16)
        h = -(-m // (1 << c))
        out = np.zeros((h, 2, self.L, self.N), np.uint64)
        _check(lib().orc_make_query(self._ctx, pos, pos.size, m, c, _c(s, np.int8),
                                    _c(a, np.uint64), _c(e, np.int32), out), "query")
        return out

    def decrypt(self, ct, s):
        ct = _c(ct, np.uint64)
        size = ct.shape[0]
        mu = np.zeros(self.N, np.uint32)
        budget = C.c_double()
        _check(lib().orc_decrypt(self._ctx, ct, size, _c(s, np.int8), mu,
                                 C.byref(budget)), "decrypt")
        return mu, budget.value
