"""Error reporting of the device-buffer paths, the documented option
defaults and refused allocations.

None of these tests makes the GPU fault: a failed device check is raised by
the library's test hook (a host-to-device copy into the slot's flag word),
and allocations are refused by the context's memory cap before cudaMalloc.
"""
import os
import re

import numpy as np
import pytest

from tests.workloads import T, Client, database

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2202_07569_gb300 import build

    build.build()


def test_device_path_reports_a_failed_check_once():
    """cwpir_answer_device returns once enqueued; the check flag it may set
    is read (and cleared) by cwpir_device_status, so a failure is reported
    for the work that raised it and never blamed on a later call."""
    import torch

    from paper_2202_07569_gb300 import binding as B

    cl = Client(4096, 2, seed=111)
    ctx = cl.context()
    items, cw, _ = database(20, 64, T, 2, 8, seed=112)
    db = ctx.load_db(items, cw, 8)
    q = cl.query(cw[5], 8, 0, stream=1)
    want = cl.O.answer(items, cw, 8, q, cl.rlk)
    dq = torch.from_numpy(q.view(np.int64)).cuda()
    dr = torch.empty(ctx.ct_shape, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    ctx.answer_device(db, dq.data_ptr(), dr.data_ptr(), 0, st)
    assert ctx.device_status(0, st) == 0
    assert np.array_equal(dr.cpu().numpy().view(np.uint64), want)
    ctx.inject_status(0)
    ctx.answer_device(db, dq.data_ptr(), dr.data_ptr(), 0, st)
    assert ctx.device_status(0, st) == B.EINTERNAL
    assert ctx.device_status(0, st) == 0  # read once, then cleared
    # the host-buffer call reads slot 0's flag itself
    ctx.inject_status(0)
    with pytest.raises(B.CwpirError) as ei:
        ctx.answer(db, q)
    assert ei.value.code == B.EINTERNAL
    assert np.array_equal(ctx.answer(db, q), want)
    ctx.close()


def test_slot_answers_equal_slot_zero_and_slots_are_reused():
    import torch

    cl = Client(4096, 2, seed=113)
    ctx = cl.context()
    items, cw, _ = database(40, 64, T, 2, 10, seed=114)
    db = ctx.load_db(items, cw, 10)
    qs = np.stack([cl.query(cw[i], 10, 0, stream=10 + i) for i in (3, 17)])
    want = ctx.answer_batch(db, qs)
    s1, s2 = ctx.slot_create(), ctx.slot_create()
    assert (s1, s2) == (1, 2)
    dq = torch.from_numpy(qs.view(np.int64)).cuda()
    outs = [torch.empty((2,) + ctx.ct_shape, dtype=torch.int64, device="cuda") for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    for slot, out, stm in zip((s1, s2), outs, streams):
        ctx.answer_batch_slot(slot, db, 2, dq.data_ptr(), out.data_ptr(), 0, stm.cuda_stream)
    for slot, out, stm in zip((s1, s2), outs, streams):
        assert ctx.device_status(slot, stm.cuda_stream) == 0
        assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
    ctx.slot_release(s1)
    assert ctx.slot_create() == s1
    ctx.close()


def test_option_defaults_match_the_header():
    """Every option default the header documents as "(default)" is the
    value the library reports."""
    from paper_2202_07569_gb300 import binding as B

    text = open(os.path.join(ROOT, "include", "cwpir.h")).read()
    body = text[text.index("---- options ----"):text.index("int cwpir_set_option")]
    documented = {}
    for comment, name in re.findall(r"/\*(.*?)\*/\s*(CWPIR_OPT_\w+)", body, re.S):
        comment = re.sub(r"\s*\n\s*\*\s*", " ", comment)
        m = re.search(r"(\d+) \(default\)", comment)
        if m:
            documented[name] = int(m.group(1))
        elif re.search(r"0 = no cap, the default", comment):
            documented[name] = 0
        elif re.search(r"0 = the default, (\d+)", comment):
            documented[name] = int(re.search(r"0 = the default, (\d+)", comment).group(1))
    assert documented["CWPIR_OPT_USE_GRAPH"] == 0
    assert {"CWPIR_OPT_SHARE_LEVEL1", "CWPIR_OPT_KERNEL_TIMING", "CWPIR_OPT_ROW_BASIS",
            "CWPIR_OPT_MEM_LIMIT", "CWPIR_OPT_ROW_GROUP_WAVES"} <= set(documented)
    cl = Client(4096, 2, seed=115)
    ctx = cl.context()
    for name, value in documented.items():
        assert ctx.get_option(getattr(B, name.replace("CWPIR_", ""))) == value, name
    ctx.close()


def test_memory_cap_refuses_allocations_with_enomem():
    """The host-side fault "allocation refused": with a cap on the context's
    device memory, loading a database or sizing the scratch that would pass
    it fails with ENOMEM before any cudaMalloc, and the context keeps
    working once the cap is raised."""
    from paper_2202_07569_gb300 import binding as B

    cl = Client(4096, 2, seed=116)
    ctx = cl.context()
    items, cw, _ = database(60, 64, T, 2, 12, seed=117)
    used = ctx.mem_used()
    cap = used + (8 << 20)
    ctx.set_option(B.OPT_MEM_LIMIT, cap)
    assert ctx.get_option(B.OPT_MEM_LIMIT) == cap
    big = np.zeros((4096, 64), np.uint32)
    cwb = np.stack([cw[i % 60] for i in range(4096)])
    with pytest.raises(B.CwpirError) as ei:
        ctx.load_db(big, cwb, 12)  # 4096 rows x 3 x 4096 x 4 B = 192 MiB
    assert ei.value.code == -2
    db = ctx.load_db(items, cw, 12)  # 60 rows: 2.8 MiB, within the cap
    q = cl.query(cw[9], 12, 0, stream=3)
    with pytest.raises(B.CwpirError) as ei:
        ctx.answer(db, q)  # the scratch of slot 0 (GiBs) does not fit
    assert ei.value.code == -2
    assert ctx.mem_used() <= cap
    ctx.set_option(B.OPT_MEM_LIMIT, 0)
    got = ctx.answer(db, q)
    assert np.array_equal(got, cl.O.answer(items, cw, 12, q, cl.rlk))
    ctx.close()
