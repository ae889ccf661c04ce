"""The allocation-free expectation entry point (qaoa_expect_noalloc).

It serves callers that cannot allocate device memory when they evaluate
<H_C> (a framework owning all device memory, a loop that must not take the
device synchronisation of cudaMalloc/cudaFree, code with raw device pointers
and no context).  This file is collected last on purpose: the entry point
shares one fixed device array across calls, and it must give the same answer
when it runs after every other test as when it runs alone.
"""
import numpy as np
import pytest

from paper_2606_26297_b300 import instances as inst

pytestmark = pytest.mark.gpu

E_TOL = 1e-12  # same reduction in the same order as qaoa_expect: equal to rounding


@pytest.fixture(scope="module")
def q():
    from paper_2606_26297_b300 import build_lib
    build_lib.build()
    from paper_2606_26297_b300 import qaoa
    return qaoa


def _case(q, ctx, n, seed, p):
    import torch
    Q = inst.upper_int_qubo(n, seed)
    g, b = inst.ramp_angles(p, gamma_scale=0.15)
    cost = q.qaoa_build_cost(ctx, Q.H, Q.f, Q.c0, "i32")
    st = q.qaoa_forward(ctx, cost, g, b)
    info = q.qaoa_cost_info(cost)
    # the table is handed over as a caller-owned device buffer
    table = torch.from_numpy(q.qaoa_cost_copy_to_host(ctx, cost, n)).to("cuda")
    amps, count = q.qaoa_state_device_ptr(st)
    assert count == 1 << n
    return cost, st, info, table, amps


def test_noalloc_matches_qaoa_expect_two_calls(q):
    import torch
    ctx = q.qaoa_ctx_create(0)
    try:
        c1, s1, i1, t1, a1 = _case(q, ctx, 20, 7, 3)
        c2, s2, i2, t2, a2 = _case(q, ctx, 14, 8, 2)
        torch.cuda.synchronize()
        ref1 = q.qaoa_expect(ctx, c1, s1)
        ref2 = q.qaoa_expect(ctx, c2, s2)
        # two calls in a row on different states: the second must not see the first's scratch
        got1 = q.qaoa_expect_noalloc(a1, t1.data_ptr(), 20, i1["shift_bits"], i1["k_c"])
        got2 = q.qaoa_expect_noalloc(a2, t2.data_ptr(), 14, i2["shift_bits"], i2["k_c"])
        scale1 = max(1.0, float(np.abs(q.qaoa_cost_copy_to_host(ctx, c1, 20)).max()))
        scale2 = max(1.0, float(np.abs(q.qaoa_cost_copy_to_host(ctx, c2, 14)).max()))
        assert abs(got1 - ref1) <= E_TOL * scale1
        assert abs(got2 - ref2) <= E_TOL * scale2
        # and again in the other order, on a torch stream
        s = torch.cuda.Stream()
        got2b = q.qaoa_expect_noalloc(a2, t2.data_ptr(), 14, i2["shift_bits"], i2["k_c"], s.cuda_stream)
        got1b = q.qaoa_expect_noalloc(a1, t1.data_ptr(), 20, i1["shift_bits"], i1["k_c"], s.cuda_stream)
        assert got1b == got1 and got2b == got2
        for st_, co_ in ((s1, c1), (s2, c2)):
            q.qaoa_state_destroy(st_)
            q.qaoa_cost_destroy(co_)
    finally:
        q.qaoa_ctx_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_array(q):
    import torch
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    tab = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(q.QaoaError) as e:
        q.qaoa_expect_noalloc(buf.data_ptr(), tab.data_ptr(), 31, 0, 0)
    assert e.value.status == q.QAOA_ERR_INVALID_ARG
    assert "30" in str(e.value)
    with pytest.raises(q.QaoaError):
        q.qaoa_expect_noalloc(0, tab.data_ptr(), 3, 0, 0)
