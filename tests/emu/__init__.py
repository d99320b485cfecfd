"""Test-only CPU emulation of the CUDA kernels' arithmetic (see emu.cpp)."""
import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "emu.cpp")
CSRC = os.path.join(os.path.dirname(os.path.dirname(HERE)), "paper_2202_07569_gb300", "csrc")
SO = os.path.join(HERE, "_build", "libemu.so")
_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    deps = [SRC] + [os.path.join(CSRC, f) for f in ("arith.cuh", "host_tables.hpp", "ntt_pass.cuh")]
    if not os.path.exists(SO) or os.path.getmtime(SO) < max(map(os.path.getmtime, deps)):
        os.makedirs(os.path.dirname(SO), exist_ok=True)
        tmp = SO + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-x", "c++", SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, SO)
    l = C.CDLL(SO)
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    U32, U64 = C.c_uint32, C.c_uint64
    l.emu_tensor_intt_compare.argtypes = [U32, U32, u64p, U64, u64p]
    l.emu_tensor_intt_compare.restype = U64
    l.emu_bfv_mul.argtypes = [U32, U32, u64p, U64, u64p, u64p, u64p, u64p, C.c_int]
    l.emu_scale_p.argtypes = [U32, U32, u64p, U64, U64,
                              np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS"), u64p, C.c_int,
                              np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")]
    l.emu_scale_p.restype = None
    l.emu_bfv_mul.restype = C.c_int
    l.emu_lift.argtypes = [U32, U32, u64p, U64, u64p, u64p]
    l.emu_lift.restype = None
    l.emu_ext_primes.argtypes = [U32, U32, u64p, u64p]
    l.emu_ext_primes.restype = None
    l.emu_ext_count.argtypes = [U32]
    l.emu_ext_count.restype = U32
    l.emu_row_crt.argtypes = [U32, U32, u64p, U64, U32,
                              np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS"), u64p]
    l.emu_row_limit.argtypes = [U32, U32, u64p, U64, U32]
    l.emu_row_limit.restype = U64
    l.emu_row_crt.restype = C.c_int
    l.emu_reduce62.argtypes = [U64, u64p, U64,
                               np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")]
    l.emu_reduce62.restype = None
    l.emu_row_sum.argtypes = [U32, U32, u64p, U64, U32, U64, u64p,
                              np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS"), u64p]
    l.emu_row_sum.restype = U64
    l.emu_substitute.argtypes = [U32, U32, u64p, U64, U32, u64p, u64p, u64p]
    l.emu_substitute.restype = None
    l.emu_scale.argtypes = [U32, U32, u64p, U64, u64p, u64p, u64p]
    l.emu_scale.restype = C.c_int
    l.emu_ntt_compare.argtypes = [U32, U32, u64p, U64, u64p, U32]
    l.emu_ntt_compare.restype = C.c_uint64
    _lib = l
    return l
