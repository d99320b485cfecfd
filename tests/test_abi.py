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

    assert B.abi_version() == 2
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
