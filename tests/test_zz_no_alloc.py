"""The multiplication entry point that allocates nothing (cwpir_mul_noalloc).

It serves callers that cannot allocate device memory where they multiply;
its intermediates live in a fixed device array inside the library.  This
file runs last so that a stop at the first failure has already run every
other test; it also runs alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2202_07569_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2202_07569_gb300 import build

    build.build()


def test_mul_noalloc_matches_mul_on_two_calls_in_a_row():
    import torch

    from paper_2202_07569_gb300 import binding as B
    from tests.workloads import Client

    cl = Client(8192, 4, seed=41)
    ctx = cl.context()
    shape = ctx.ct_shape
    da = torch.empty(shape, dtype=torch.int64, device="cuda:0")
    db = torch.empty(shape, dtype=torch.int64, device="cuda:0")
    dout = torch.empty(shape, dtype=torch.int64, device="cuda:0")
    st = torch.cuda.current_stream()
    st.synchronize()
    free_after = []
    for call in range(2):
        a = syn.uniform_residues(syn.Stream(42, call), cl.q, (2,), 8192)
        b = syn.uniform_residues(syn.Stream(43, call), cl.q, (2,), 8192)
        want = ctx.mul(a, b)  # the existing, allocating entry point
        da.copy_(torch.from_numpy(a.view(np.int64)))
        db.copy_(torch.from_numpy(b.view(np.int64)))
        dout.zero_()
        st.synchronize()
        ctx.mul_noalloc(da.data_ptr(), db.data_ptr(), dout.data_ptr(), st.cuda_stream)
        got = dout.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), call  # bit-exact, the tolerance of every test
        free_after.append(torch.cuda.mem_get_info()[0])
    # the second call took no device memory
    assert free_after[1] == free_after[0]
    ctx.close()


def test_mul_noalloc_rejects_sizes_beyond_the_array():
    import torch

    from paper_2202_07569_gb300 import binding as B
    from tests.workloads import Client

    cl = Client(16384, 7, seed=44)
    ctx = cl.context()
    buf = torch.zeros(ctx.ct_shape, dtype=torch.int64, device="cuda:0")
    with pytest.raises(B.CwpirError) as ei:
        ctx.mul_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 0)
    assert ei.value.code == -1 and "scratch" in str(ei.value)
    ctx.close()
