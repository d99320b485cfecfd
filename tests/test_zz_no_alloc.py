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
    """Two calls in a row, each equal bit for bit (the tolerance of every
    test here) to the existing, allocating cwpir_mul and to the oracle's
    multiplication; the second call with residues at q_j - 1, the largest
    inputs the boundary accepts."""
    import torch

    from tests.workloads import Client

    cl = Client(8192, 4, seed=41)
    ctx = cl.context()
    shape = ctx.ct_shape
    da = torch.empty(shape, dtype=torch.int64, device="cuda:0")
    db = torch.empty(shape, dtype=torch.int64, device="cuda:0")
    dout = torch.empty(shape, dtype=torch.int64, device="cuda:0")
    st = torch.cuda.current_stream()
    st.synchronize()
    for call in range(2):
        a = syn.uniform_residues(syn.Stream(42, call), cl.q, (2,), 8192)
        b = syn.uniform_residues(syn.Stream(43, call), cl.q, (2,), 8192)
        if call == 1:
            for j, qj in enumerate(cl.q):
                a[:, j, ::3] = qj - 1
                b[:, j, 1::5] = qj - 1
        want = ctx.mul(a, b)  # the existing, allocating entry point
        assert np.array_equal(want, cl.O.bfv_mul(a, b, cl.rlk)), call
        da.copy_(torch.from_numpy(a.view(np.int64)))
        db.copy_(torch.from_numpy(b.view(np.int64)))
        dout.zero_()
        st.synchronize()
        ctx.mul_noalloc(da.data_ptr(), db.data_ptr(), dout.data_ptr(), st.cuda_stream)
        got = dout.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), call
    ctx.close()


def test_mul_noalloc_takes_no_device_memory():
    """After a first call, repeated calls alone (nothing else between them)
    leave the device's free memory and torch's allocations unchanged, and
    each call's result is still the product."""
    import torch

    from tests.workloads import Client

    cl = Client(4096, 2, seed=45)
    ctx = cl.context()
    a = syn.uniform_residues(syn.Stream(46), cl.q, (2,), 4096)
    b = syn.uniform_residues(syn.Stream(47), cl.q, (2,), 4096)
    want = cl.O.bfv_mul(a, b, cl.rlk)
    da = torch.from_numpy(a.view(np.int64)).cuda()
    db = torch.from_numpy(b.view(np.int64)).cuda()
    dout = torch.empty(ctx.ct_shape, dtype=torch.int64, device="cuda:0")
    st = torch.cuda.current_stream()
    ctx.mul_noalloc(da.data_ptr(), db.data_ptr(), dout.data_ptr(), st.cuda_stream)
    torch.cuda.synchronize()
    free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(4):
        ctx.mul_noalloc(da.data_ptr(), db.data_ptr(), dout.data_ptr(), st.cuda_stream)
        assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == torch0
    assert np.array_equal(dout.cpu().numpy().view(np.uint64), want)
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
