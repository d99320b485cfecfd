"""The C-ABI library loads and exports every symbol include/cwpir.h declares;
host-only helpers agree with the paper's definitions.  No GPU needed."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cudalib():
    from paper_2202_07569_gb300 import build

    build.build()
    return build.LIB


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cwpir.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cwpir_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cwpir_setup", "cwpir_load_db", "cwpir_answer", "cwpir_answer_device",
                 "cwpir_destroy", "cwpir_last_error", "cwpir_mul", "cwpir_expand"):
        assert must in names


def test_library_exports_every_declared_symbol(cudalib):
    lib = ctypes.CDLL(cudalib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing


def test_host_helpers_match_definitions(cudalib, orc):
    from paper_2202_07569_gb300 import binding as B

    assert B.abi_version() == 4
    for N, L in ((4096, 2), (8192, 4), (16384, 7)):
        assert B.default_primes(N, L).tolist() == orc.primes(N, L).tolist()
    for m, k in ((24, 2), (10, 4), (12, 5)):
        for x in range(math.comb(m, k)):
            assert B.map_perfect(x, m, k).tolist() == orc.map_perfect(x, m, k).tolist()
    assert B.code_length(65536, 4) == 37
    assert B.code_length(256, 2) == 24
    assert B.code_length(1 << 32, 8) == 64
    with pytest.raises(B.CwpirError):
        B.map_perfect(math.comb(24, 2), 24, 2)
    for m, k in ((64, 8), (9, 2), (16, 16)):
        for x in (0, 1, 12345, (1 << 64) - 1, 0x0123456789ABCDEF):
            assert B.map_lossy(x, m, k).tolist() == orc.map_lossy(x, m, k).tolist()
    with pytest.raises(B.CwpirError):
        B.map_lossy(5, 4, 5)


def test_folklore_codewords_match_definition(cudalib, orc):
    """cwpir_map_folklore: positions 2i + y[i] (the plain folklore operator,
    Eq. folklore-plain-eq), against the oracle; y >= 2^ell is rejected."""
    from paper_2202_07569_gb300 import binding as B

    for ell in (1, 2, 7, 12, 16):
        for y in sorted({0, 1, (1 << ell) - 1, 0x5A5A & ((1 << ell) - 1)}):
            got = B.map_folklore(y, ell).tolist()
            assert got == orc.folklore_codeword(y, ell).tolist()
            assert got == [2 * i + ((y >> i) & 1) for i in range(ell)]
    with pytest.raises(B.CwpirError):
        B.map_folklore(1 << 5, 5)


def test_setup_rejects_bad_parameters(cudalib):
    """cwpir_setup checks N, L, t and the primes before it touches the
    device: each bad set returns EINVAL with a message naming the problem."""
    import numpy as np

    from paper_2202_07569_gb300 import binding as B

    q8 = [int(v) for v in B.default_primes(8192, 4)]
    composite = next(x for x in range(q8[0] - 16384, 1 << 53, -16384)
                     if any(x % d == 0 for d in (3, 5, 7, 11, 13)))
    cases = [
        (1000, q8, 65537, "N must be"),
        (32768, q8, 65537, "N must be"),
        (8192, [int(v) for v in B.default_primes(8192, 9)], 65537, "L must be"),
        (8192, q8, 65536, "t must be"),
        (8192, q8, (1 << 20) + 7, "t must be"),
        (8192, q8, 2, "t must be"),
        (16384, q8, 65537, "q[2] must be"),           # not 1 mod 2N at N = 16384
        (8192, [composite] + q8[1:], 65537, "q[0] must be"),
        (8192, [q8[0], q8[0]], 65537, "distinct"),
    ]
    for N, q, t, msg in cases:
        L = max(len(q), 1)
        relin = np.zeros(L * 2 * L * N, np.uint64)
        with pytest.raises(B.CwpirError) as ei:
            B.Context(N, np.array(q, np.uint64), t, relin)
        assert ei.value.code == -1 and msg in str(ei.value), (N, len(q), t, str(ei.value))


def test_kernel_classes_match_the_header(cudalib):
    """The timing classes: the binding's count is the header's
    CWPIR_K_CLASSES, and each class name the library reports is the one the
    header documents beside its enumerator."""
    from paper_2202_07569_gb300 import binding as B

    src = open(os.path.join(ROOT, "include", "cwpir.h")).read()
    assert int(re.search(r"CWPIR_K_CLASSES\s*=\s*(\d+)", src).group(1)) == B.K_CLASSES
    documented = {}
    for m in re.finditer(r"CWPIR_K_[A-Z]+\s*=\s*(\d+),\s*/\*(.*?)\*/", src, flags=re.S):
        name = re.search(r'\("([a-z_]+)"', m.group(2))
        if name:
            documented[int(m.group(1))] = name.group(1)
    assert sorted(documented) == list(range(B.K_CLASSES))
    lib = ctypes.CDLL(cudalib)
    lib.cwpir_kernel_class_name.restype = ctypes.c_char_p
    lib.cwpir_kernel_class_name.argtypes = [ctypes.c_int]
    for i in range(B.K_CLASSES):
        assert lib.cwpir_kernel_class_name(i).decode() == documented[i], i
