"""ctypes binding of the C ABI in ``include/cwpir.h`` (argument marshalling
only: every step of the answer path runs in the CUDA library).

The library is ``_build/libcwpir.so`` built by ``build.py``.  Loading fails
loudly when it is missing; there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")

OPT_SHARE_LEVEL1 = 1
OPT_BATCH_ROWS = 2
OPT_USE_GRAPH = 3
OPT_KERNEL_TIMING = 4
OPT_MAX_JOBS = 5
OPT_ROW_BASIS = 6
OPT_MEM_LIMIT = 7
OPT_ROW_GROUP_WAVES = 8
OPT_SCALE_EXACT = 9
K_CLASSES = 8
EINTERNAL = -8


class CwpirError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"cwpir error {code}: {msg}")
        self.code = code


class _Params(C.Structure):
    _fields_ = [("N", C.c_uint32), ("L", C.c_uint32), ("q", C.POINTER(C.c_uint64)),
                ("t", C.c_uint64)]


class _Keys(C.Structure):
    _fields_ = [("relin", C.POINTER(C.c_uint64)), ("n_galois", C.c_uint32),
                ("galois_elts", C.POINTER(C.c_uint32)), ("galois", C.POINTER(C.c_uint64))]


class _Target(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("db_id", C.c_int32), ("c", C.c_uint32)]


class _ServerConfig(C.Structure):
    _fields_ = [("max_batch", C.c_uint32), ("lanes_per_target", C.c_uint32),
                ("max_pending", C.c_uint32), ("hbm_reserve_bytes", C.c_uint64)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("batches", C.c_uint64),
                ("max_batch_seen", C.c_uint64), ("rejected_busy", C.c_uint64),
                ("failed", C.c_uint64), ("max_concurrent", C.c_uint64),
                ("busy_s", C.c_double)]

    def as_dict(self):
        return {f: (float(getattr(self, f)) if f == "busy_s" else int(getattr(self, f)))
                for f, _ in self._fields_}


class _MultiItem(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("db_id", C.c_int32), ("c", C.c_uint32),
                ("nq", C.c_uint32), ("nq_call", C.c_uint32)]


class IntPeaks(C.Structure):
    _fields_ = [("imad32_per_s", C.c_double), ("mulhi32_per_s", C.c_double),
                ("mullo64_per_s", C.c_double), ("mulhi64_per_s", C.c_double),
                ("iadd32_per_s", C.c_double), ("sms", C.c_int), ("max_sm_mhz", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("rows", C.c_uint64), ("mults", C.c_uint64), ("substitutions", C.c_uint64),
                ("ntt_polys", C.c_uint64), ("kernel_launches", C.c_uint64),
                ("db_bytes_read", C.c_uint64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(
                f"CUDA library {path} is missing: run paper_2202_07569_gb300.build.build() "
                "(or __graft_entry__.build()) first")
        l = C.CDLL(path)
        I, U32, U64, vp = C.c_int, C.c_uint32, C.c_uint64, C.c_void_p
        sig = {
            "cwpir_abi_version": (I, []),
            "cwpir_strerror": (C.c_char_p, [I]),
            "cwpir_last_error": (C.c_char_p, [vp]),
            "cwpir_default_primes": (I, [U32, U32, u64p]),
            "cwpir_map_perfect": (I, [U64, U32, U32, u16p]),
            "cwpir_map_lossy": (I, [U64, U32, U32, u16p]),
            "cwpir_map_folklore": (I, [U64, U32, u16p]),
            "cwpir_load_db_folklore": (I, [vp, U64, U32, U32, u32p, C.POINTER(C.c_int32)]),
            "cwpir_query_cts": (I, [vp, C.c_int32, U32, C.POINTER(U32)]),
            "cwpir_arith_cw_eq": (I, [vp, U32, U32, u64p, u64p, u64p]),
            "cwpir_code_length": (I, [U64, U32, C.POINTER(U32)]),
            "cwpir_setup": (I, [C.POINTER(_Params), C.POINTER(_Keys), C.POINTER(vp)]),
            "cwpir_destroy": (None, [vp]),
            "cwpir_load_db": (I, [vp, U64, U32, U32, U32, u32p, u16p, C.POINTER(C.c_int32)]),
            "cwpir_free_db": (I, [vp, C.c_int32]),
            "cwpir_answer": (I, [vp, C.c_int32, U32, u64p, u64p]),
            "cwpir_answer_device": (I, [vp, C.c_int32, U32, vp, vp, vp]),
            "cwpir_sum_responses_device": (I, [vp, U32, U32, vp, vp, vp]),
            "cwpir_reduce_responses_device": (I, [vp, U32, vp, vp, vp]),
            "cwpir_mul": (I, [vp, u64p, u64p, u64p]),
            "cwpir_substitute": (I, [vp, U32, u64p, u64p]),
            "cwpir_expand": (I, [vp, U32, U32, u64p, u64p]),
            "cwpir_selection": (I, [vp, C.c_int32, U32, u64p, U64, u64p, u64p]),
            "cwpir_plain_mul": (I, [vp, C.c_int32, U64, u64p, u64p]),
            "cwpir_set_option": (I, [vp, I, C.c_int64]),
            "cwpir_get_option": (I, [vp, I, C.POINTER(C.c_int64)]),
            "cwpir_mem_used": (I, [vp, C.POINTER(U64)]),
            "cwpir_slot_create": (I, [vp, C.POINTER(U32)]),
            "cwpir_answer_batch_slot": (I, [vp, U32, C.c_int32, U32, U32, vp, vp, vp]),
            "cwpir_plan_bytes_slot": (I, [vp, U32, C.c_int32, U32, U32, C.POINTER(U64)]),
            "cwpir_device_status": (I, [vp, U32, vp]),
            "cwpir_inject_status": (I, [vp, U32]),
            "cwpir_last_stats": (I, [vp, C.POINTER(Stats)]),
            "cwpir_kernel_times": (I, [vp, C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
            "cwpir_kernel_class_name": (C.c_char_p, [I]),
            "cwpir_mul_noalloc": (I, [vp, vp, vp, vp, vp]),
            "cwpir_measure_int_peaks": (I, [C.c_int, C.POINTER(IntPeaks)]),
            "cwpir_multi_create": (I, [C.POINTER(_MultiItem), U32, C.POINTER(vp)]),
            "cwpir_multi_answer_device": (I, [vp, C.POINTER(vp), C.POINTER(vp), I, vp]),
            "cwpir_multi_status": (I, [vp, vp]),
            "cwpir_multi_stats": (I, [vp, C.POINTER(Stats)]),
            "cwpir_multi_last_error": (C.c_char_p, [vp]),
            "cwpir_multi_destroy": (None, [vp]),
            "cwpir_plan_bytes": (I, [vp, C.c_int32, U32, U32, C.POINTER(U64)]),
            "cwpir_release_plans": (I, [vp, C.c_int32]),
            "cwpir_db_shape": (I, [vp, C.c_int32, C.POINTER(U32), C.POINTER(U32),
                                   C.POINTER(U32)]),
            "cwpir_db_plaintexts": (I, [vp, C.c_int32, C.POINTER(U32)]),
            "cwpir_ctx_device": (I, [vp, C.POINTER(C.c_int)]),
            "cwpir_server_create": (I, [C.POINTER(_Target), U32, C.POINTER(_ServerConfig),
                                        C.POINTER(vp)]),
            "cwpir_slot_release": (I, [vp, U32]),
            "cwpir_submit": (I, [vp, U32, u64p, C.POINTER(U64)]),
            "cwpir_poll": (I, [vp, U64, u64p, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
            "cwpir_wait": (I, [vp, U64, u64p, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                               C.c_double]),
            "cwpir_server_get_stats": (I, [vp, C.POINTER(ServerStats)]),
            "cwpir_server_destroy": (None, [vp]),
            "cwpir_answer_batch": (I, [vp, C.c_int32, U32, U32, u64p, u64p]),
            "cwpir_answer_batch_device": (I, [vp, C.c_int32, U32, U32, vp, vp, vp]),
            "cwpir_autotune": (I, [vp, C.c_int32, U32, U32, vp, vp, C.POINTER(C.c_int64), U32,
                                   C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
            "cwpir_autotune_grid": (I, [vp, C.c_int32, U32, U32, vp, vp, C.POINTER(C.c_int64),
                                        U32, C.POINTER(C.c_int64), U32, C.POINTER(C.c_int64),
                                        C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
        return l


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def abi_version() -> int:
    return int(lib().cwpir_abi_version())


def default_primes(N: int, L: int) -> np.ndarray:
    out = np.zeros(L, np.uint64)
    rc = lib().cwpir_default_primes(N, L, out)
    if rc:
        raise CwpirError(rc, "default primes")
    return out


def map_perfect(x: int, m: int, k: int) -> np.ndarray:
    pos = np.zeros(k, np.uint16)
    rc = lib().cwpir_map_perfect(int(x), m, k, pos)
    if rc:
        raise CwpirError(rc, f"perfect mapping of {x} into CW({m},{k})")
    return pos


def map_lossy(x: int, m: int, k: int) -> np.ndarray:
    """Alg. Lossy Mapping of a 64-bit element into CW(m, k)."""
    pos = np.zeros(k, np.uint16)
    rc = lib().cwpir_map_lossy(int(x), m, k, pos)
    if rc:
        raise CwpirError(rc, f"lossy mapping of {x} into CW({m},{k})")
    return pos


def map_folklore(y: int, ell: int) -> np.ndarray:
    """Positions 2i + y[i] of the plain folklore operator's factors."""
    pos = np.zeros(ell, np.uint16)
    rc = lib().cwpir_map_folklore(int(y), ell, pos)
    if rc:
        raise CwpirError(rc, f"folklore codeword of {y} with {ell} bits")
    return pos


def measure_int_peaks(device: int = 0) -> dict:
    """Measured integer-pipe rates of a device (operations per second)."""
    p = IntPeaks()
    rc = lib().cwpir_measure_int_peaks(device, C.byref(p))
    if rc:
        raise CwpirError(rc, "integer peak probe")
    return p.as_dict()


def code_length(n: int, k: int) -> int:
    m = C.c_uint32()
    rc = lib().cwpir_code_length(int(n), k, C.byref(m))
    if rc:
        raise CwpirError(rc, "code length")
    return int(m.value)


class Context:
    """A cwpir_ctx: parameters, evaluation keys and resident databases."""

    def __init__(self, N: int, q, t: int, relin, galois: dict | None = None):
        l = lib()
        self._q = _u64(q)
        self.N, self.L, self.t = int(N), int(self._q.size), int(t)
        self._relin = _u64(relin)
        galois = galois or {}
        elts = np.array(sorted(galois), dtype=np.uint32)
        gk = (np.stack([_u64(galois[g]) for g in elts]) if len(elts)
              else np.zeros(1, np.uint64))
        self._gk = np.ascontiguousarray(gk)
        self._elts = elts if len(elts) else np.zeros(1, np.uint32)
        p = _Params(self.N, self.L, self._q.ctypes.data_as(C.POINTER(C.c_uint64)), self.t)
        k = _Keys(self._relin.ctypes.data_as(C.POINTER(C.c_uint64)), len(elts),
                  self._elts.ctypes.data_as(C.POINTER(C.c_uint32)),
                  self._gk.ctypes.data_as(C.POINTER(C.c_uint64)))
        h = C.c_void_p()
        rc = l.cwpir_setup(C.byref(p), C.byref(k), C.byref(h))
        if rc:
            raise CwpirError(rc, l.cwpir_last_error(None).decode())
        self._h = h
        # the library copied what it needs
        del self._relin, self._gk

    def close(self):
        if getattr(self, "_h", None):
            lib().cwpir_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise CwpirError(rc, lib().cwpir_last_error(self._h).decode())

    @property
    def ct_shape(self):
        return (2, self.L, self.N)

    def load_db(self, items, codewords, m: int) -> int:
        items = np.ascontiguousarray(items, dtype=np.uint32)
        cw = np.ascontiguousarray(codewords, dtype=np.uint16)
        n = cw.shape[0]
        plen = items.shape[1] if items.ndim == 2 else 0
        if items.ndim == 2 and items.shape[0] != n:
            raise ValueError("items and codewords disagree on n")
        db = C.c_int32()
        self._check(lib().cwpir_load_db(self._h, n, plen, cw.shape[1], m,
                                        items.reshape(-1) if plen else np.zeros(1, np.uint32),
                                        cw.reshape(-1), C.byref(db)))
        return int(db.value)

    def load_db_folklore(self, items, ell: int) -> int:
        """Folklore PIR database: rows 0..n-1 indexed by ell bits."""
        items = np.ascontiguousarray(items, dtype=np.uint32)
        n, plen = items.shape
        db = C.c_int32()
        self._check(lib().cwpir_load_db_folklore(self._h, n, plen, ell, items.reshape(-1),
                                                 C.byref(db)))
        return int(db.value)

    def query_cts(self, db: int, c: int = 0) -> int:
        """Ciphertexts of one query against the database."""
        h = C.c_uint32()
        self._check(lib().cwpir_query_cts(self._h, db, c, C.byref(h)))
        return int(h.value)

    def plaintexts(self, db: int) -> int:
        """Plaintexts per row s of a database (Sec. 3.3.1)."""
        s = C.c_uint32()
        self._check(lib().cwpir_db_plaintexts(self._h, db, C.byref(s)))
        return int(s.value)

    def resp_shape(self, db: int):
        """Shape of one query's response: [2][L][N], or [s][2][L][N] for rows
        of s > 1 plaintexts."""
        s = self.plaintexts(db)
        return ((s,) if s > 1 else ()) + self.ct_shape

    def free_db(self, db: int):
        self._check(lib().cwpir_free_db(self._h, db))

    def answer(self, db: int, query, c: int = 0) -> np.ndarray:
        out = np.zeros(self.resp_shape(db), np.uint64)
        self._check(lib().cwpir_answer(self._h, db, c, _u64(query), out))
        return out

    def answer_device(self, db: int, query_ptr: int, resp_ptr: int, c: int = 0,
                      stream: int = 0):
        self._check(lib().cwpir_answer_device(self._h, db, c, query_ptr, resp_ptr, stream))

    def sum_responses_device(self, count: int, s: int, parts_ptr: int, out_ptr: int,
                             stream: int = 0):
        """Sum of `count` partial responses [count][s][2][L][N] (device) into
        [s][2][L][N] modulo each q_j: the exchange step of a sharded database."""
        self._check(lib().cwpir_sum_responses_device(self._h, count, s, parts_ptr, out_ptr,
                                                     stream))

    def reduce_responses_device(self, s: int, sums_ptr: int, out_ptr: int, stream: int = 0):
        """Element-wise u64 sums of partial responses [s][2][L][N] (device)
        modulo each q_j: the all-reduce form of the sharded exchange."""
        self._check(lib().cwpir_reduce_responses_device(self._h, s, sums_ptr, out_ptr, stream))

    def answer_batch(self, db: int, queries, c: int = 0) -> np.ndarray:
        q = _u64(queries)
        nq = q.shape[0]
        out = np.zeros((nq,) + self.resp_shape(db), np.uint64)
        self._check(lib().cwpir_answer_batch(self._h, db, c, nq, q.reshape(-1), out))
        return out

    def answer_batch_device(self, db: int, nq: int, queries_ptr: int, resp_ptr: int,
                            c: int = 0, stream: int = 0):
        self._check(lib().cwpir_answer_batch_device(self._h, db, c, nq, queries_ptr, resp_ptr,
                                                    stream))

    def autotune(self, db: int, nq: int, queries_ptr: int, resp_ptr: int, candidates,
                 c: int = 0):
        cand = (C.c_int64 * len(candidates))(*candidates)
        best, ms = C.c_int64(), C.c_double()
        self._check(lib().cwpir_autotune(self._h, db, c, nq, queries_ptr, resp_ptr, cand,
                                         len(candidates), C.byref(best), C.byref(ms)))
        return int(best.value), float(ms.value)

    def autotune_grid(self, db: int, nq: int, queries_ptr: int, resp_ptr: int, jobs, waves,
                      c: int = 0):
        """(best jobs per launch, best row-group waves, ms per call)."""
        ja = (C.c_int64 * len(jobs))(*jobs)
        wa = (C.c_int64 * max(1, len(waves)))(*(waves or [0]))
        bj, bw, ms = C.c_int64(), C.c_int64(), C.c_double()
        self._check(lib().cwpir_autotune_grid(self._h, db, c, nq, queries_ptr, resp_ptr, ja,
                                              len(jobs), wa, len(waves), C.byref(bj),
                                              C.byref(bw), C.byref(ms)))
        return int(bj.value), int(bw.value), float(ms.value)

    def mul(self, a, b) -> np.ndarray:
        out = np.zeros(self.ct_shape, np.uint64)
        self._check(lib().cwpir_mul(self._h, _u64(a), _u64(b), out))
        return out

    def mul_noalloc(self, d_a: int, d_b: int, d_out: int, stream: int = 0):
        """cwpir_mul_noalloc on device pointers (no device allocation)."""
        self._check(lib().cwpir_mul_noalloc(self._h, d_a, d_b, d_out, stream))

    def substitute(self, g: int, ct) -> np.ndarray:
        out = np.zeros(self.ct_shape, np.uint64)
        self._check(lib().cwpir_substitute(self._h, g, _u64(ct), out))
        return out

    def expand(self, query, c: int, m: int) -> np.ndarray:
        out = np.zeros((m,) + self.ct_shape, np.uint64)
        self._check(lib().cwpir_expand(self._h, c, m, _u64(query), out))
        return out

    def selection(self, db: int, query, rows, c: int = 0) -> np.ndarray:
        rows = np.ascontiguousarray(rows, dtype=np.uint64)
        out = np.zeros((rows.size,) + self.ct_shape, np.uint64)
        self._check(lib().cwpir_selection(self._h, db, c, _u64(query), rows.size, rows, out))
        return out

    def arith_cw_eq(self, m: int, k: int, x, y) -> np.ndarray:
        """Arithmetic constant-weight equality operator on encrypted operands."""
        out = np.zeros(self.ct_shape, np.uint64)
        self._check(lib().cwpir_arith_cw_eq(self._h, m, k, _u64(x), _u64(y), out))
        return out

    def plain_mul(self, db: int, row: int, ct) -> np.ndarray:
        out = np.zeros(self.resp_shape(db), np.uint64)
        self._check(lib().cwpir_plain_mul(self._h, db, row, _u64(ct), out))
        return out

    def set_option(self, option: int, value: int):
        self._check(lib().cwpir_set_option(self._h, option, value))

    def get_option(self, option: int) -> int:
        v = C.c_int64()
        self._check(lib().cwpir_get_option(self._h, option, C.byref(v)))
        return int(v.value)

    def mem_used(self) -> int:
        """Device bytes held by the context's buffers."""
        v = C.c_uint64()
        self._check(lib().cwpir_mem_used(self._h, C.byref(v)))
        return int(v.value)

    def slot_create(self) -> int:
        """A new scratch slot for answers concurrent with other slots."""
        v = C.c_uint32()
        self._check(lib().cwpir_slot_create(self._h, C.byref(v)))
        return int(v.value)

    def answer_batch_slot(self, slot: int, db: int, nq: int, queries_ptr: int, resp_ptr: int,
                          c: int = 0, stream: int = 0):
        self._check(lib().cwpir_answer_batch_slot(self._h, slot, db, c, nq, queries_ptr,
                                                  resp_ptr, stream))

    def plan_bytes(self, db: int, nq: int, c: int = 0, slot: int = 0) -> int:
        v = C.c_uint64()
        self._check(lib().cwpir_plan_bytes_slot(self._h, slot, db, nq, c, C.byref(v)))
        return int(v.value)

    def device_status(self, slot: int = 0, stream: int = 0) -> int:
        """Waits for `stream`, reads and clears the slot's device check flag:
        0, or EINTERNAL (returned, not raised)."""
        rc = lib().cwpir_device_status(self._h, slot, stream)
        if rc not in (0, EINTERNAL):
            self._check(rc)
        return int(rc)

    def release_plans(self, db: int = -1):
        """Frees the cached answer plans (and graphs) of a database, or of all
        databases when db < 0."""
        self._check(lib().cwpir_release_plans(self._h, db))

    def slot_release(self, slot: int):
        self._check(lib().cwpir_slot_release(self._h, slot))

    def inject_status(self, slot: int = 0):
        """Test hook: marks the slot's device check flag as failed."""
        self._check(lib().cwpir_inject_status(self._h, slot))

    def last_stats(self) -> dict:
        s = Stats()
        self._check(lib().cwpir_last_stats(self._h, C.byref(s)))
        return s.as_dict()

    def kernel_times(self) -> dict:
        """{class name: (milliseconds, launches)} since the previous call."""
        ms = (C.c_double * K_CLASSES)()
        n = (C.c_uint64 * K_CLASSES)()
        self._check(lib().cwpir_kernel_times(self._h, ms, n))
        return {lib().cwpir_kernel_class_name(i).decode(): (ms[i], int(n[i]))
                for i in range(K_CLASSES)}


class Server:
    """cwpir_server: continuous batching over registered (context, database,
    c) targets, lanes_per_target concurrent lanes each."""

    def __init__(self, targets, max_batch: int = 16, hbm_reserve: int = 1 << 30,
                 max_pending: int = 4096, lanes_per_target: int = 1):
        arr = (_Target * len(targets))()
        self._shapes = []
        for i, (ctx, db, c) in enumerate(targets):
            arr[i] = _Target(ctx._h, db, c)
            self._shapes.append(ctx.resp_shape(db))
        cfg = _ServerConfig(max_batch, lanes_per_target, max_pending, hbm_reserve)
        h = C.c_void_p()
        rc = lib().cwpir_server_create(arr, len(targets), C.byref(cfg), C.byref(h))
        if rc:
            raise CwpirError(rc, "server create")
        self._h = h
        self._ctxs = [t[0] for t in targets]  # keep contexts alive

    def submit(self, target: int, query) -> int:
        t = C.c_uint64()
        rc = lib().cwpir_submit(self._h, target, _u64(query).reshape(-1), C.byref(t))
        if rc:
            raise CwpirError(rc, "submit")
        return int(t.value)

    def poll(self, ticket: int, target: int):
        """(status, response or None, latency seconds)."""
        out = np.zeros(self._shapes[target], np.uint64)
        st, lat = C.c_int32(), C.c_double()
        rc = lib().cwpir_poll(self._h, ticket, out.reshape(-1), C.byref(st), C.byref(lat))
        if rc:
            raise CwpirError(rc, "poll")
        return int(st.value), (out if st.value == 1 else None), float(lat.value)

    def wait(self, ticket: int, target: int, timeout: float = 600.0):
        out = np.zeros(self._shapes[target], np.uint64)
        st, lat = C.c_int32(), C.c_double()
        rc = lib().cwpir_wait(self._h, ticket, out.reshape(-1), C.byref(st), C.byref(lat),
                              timeout)
        if rc:
            raise CwpirError(rc, "wait")
        return int(st.value), (out if st.value == 1 else None), float(lat.value)

    def stats(self) -> dict:
        s = ServerStats()
        lib().cwpir_server_get_stats(self._h, C.byref(s))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib().cwpir_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """cwpir_multi: the queries of several resident databases (of one or
    more contexts) answered in one forked launch sequence, one branch per
    item, optionally captured into one CUDA graph.  items: (ctx, db, c, nq,
    nq_call) tuples."""

    def __init__(self, items):
        arr = (_MultiItem * len(items))()
        self.items = []
        for i, (ctx, db, c, nq, nq_call) in enumerate(items):
            arr[i] = _MultiItem(ctx._h, db, c, nq, nq_call)
            self.items.append((ctx, db, c, nq))
        h = C.c_void_p()
        rc = lib().cwpir_multi_create(arr, len(items), C.byref(h))
        if rc:
            msg = items[0][0] and lib().cwpir_last_error(items[0][0]._h).decode()
            raise CwpirError(rc, f"multi create: {msg}")
        self._h = h
        self._ctxs = [it[0] for it in items]  # contexts must outlive the object

    def _check(self, rc):
        if rc:
            raise CwpirError(rc, lib().cwpir_multi_last_error(self._h).decode())

    def answer_device(self, query_ptrs, resp_ptrs, use_graph: bool = True, stream: int = 0):
        qa = (C.c_void_p * len(query_ptrs))(*query_ptrs)
        ra = (C.c_void_p * len(resp_ptrs))(*resp_ptrs)
        self._check(lib().cwpir_multi_answer_device(self._h, qa, ra, int(bool(use_graph)),
                                                    stream))

    def status(self, stream: int = 0) -> int:
        rc = lib().cwpir_multi_status(self._h, stream)
        if rc not in (0, EINTERNAL):
            self._check(rc)
        return int(rc)

    def stats(self) -> dict:
        s = Stats()
        self._check(lib().cwpir_multi_stats(self._h, C.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib().cwpir_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
