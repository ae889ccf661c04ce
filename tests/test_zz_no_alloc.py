"""The allocation-free expectation entry point (qaoa_expect_noalloc).

It serves callers that cannot allocate device memory when they evaluate
<H_C> (a framework owning all device memory, a loop that must not take the
device synchronisation of cudaMalloc/cudaFree, code with raw device pointers
and no context).  This file is collected last on purpose: the entry point
shares one fixed device array across calls, and it must give the same answer
when it runs after every other test as when it runs alone.

qaoa_expect_noalloc runs the same reduction as qaoa_expect in the same order,
so the two agree exactly; against the FP64 oracle the expectation of the same
state agrees within |dE| <= 1e-5 max|F| (the complex64 tolerance).
"""
import numpy as np
import pytest

import oracle
from paper_2606_26297_b300 import instances as inst

pytestmark = pytest.mark.gpu

E_TOL = 1e-5


@pytest.fixture(scope="module")
def q():
    from paper_2606_26297_b300 import build_lib
    build_lib.build()
    from paper_2606_26297_b300 import qaoa
    return qaoa


def _case(q, ctx, Q, p, seed_scale=0.15, caller_copy=True):
    import torch
    n = Q.n
    g, b = inst.ramp_angles(p, gamma_scale=seed_scale)
    cost = q.qaoa_build_cost(ctx, Q.H, Q.f, Q.c0, "i32" if Q.dtype == "i32" else "f32")
    st = q.qaoa_forward(ctx, cost, g, b)
    info = q.qaoa_cost_info(cost)
    if caller_copy:
        # the table handed over as a caller-owned device buffer
        table = torch.from_numpy(q.qaoa_cost_copy_to_host(ctx, cost, n)).to("cuda")
        tptr = table.data_ptr()
    else:
        table = None
        tptr, count = q.qaoa_cost_device_ptr(cost)
        assert count == 1 << n
    amps, count = q.qaoa_state_device_ptr(st)
    assert count == 1 << n
    return dict(cost=cost, st=st, info=info, table=table, tptr=tptr, amps=amps, n=n, g=g, b=b)


def _noalloc(q, c, stream=None):
    return q.qaoa_expect_noalloc(c["amps"], c["tptr"], c["n"], c["info"]["shift_bits"], c["info"]["k_c"], stream)


def _drop(q, *cases):
    for c in cases:
        q.qaoa_state_destroy(c["st"])
        q.qaoa_cost_destroy(c["cost"])


def test_noalloc_matches_qaoa_expect_two_calls(q):
    """Two calls in a row on different states (integer n=20, real-valued n=14
    with fixed-point shift s > 0 and offset k_c != 0): each equals qaoa_expect
    exactly, so the second does not see the first's scratch; then in the
    other order on a torch stream."""
    import torch
    ctx = q.qaoa_ctx_create(0)
    try:
        c1 = _case(q, ctx, inst.upper_int_qubo(20, 7), 3)
        c2 = _case(q, ctx, inst.normal_qubo(14, 8), 2, seed_scale=0.5)
        assert c2["info"]["shift_bits"] > 0 and c2["info"]["k_c"] != 0
        torch.cuda.synchronize()
        ref1 = q.qaoa_expect(ctx, c1["cost"], c1["st"])
        ref2 = q.qaoa_expect(ctx, c2["cost"], c2["st"])
        got1 = _noalloc(q, c1)
        got2 = _noalloc(q, c2)
        assert got1 == ref1
        assert got2 == ref2
        s = torch.cuda.Stream()
        got2b = _noalloc(q, c2, s.cuda_stream)
        got1b = _noalloc(q, c1, s.cuda_stream)
        assert got1b == ref1 and got2b == ref2
        _drop(q, c1, c2)
    finally:
        q.qaoa_ctx_destroy(ctx)


def test_noalloc_against_oracle_small_and_real(q):
    """Against the FP64 oracle on the same seeded instances: a state below one
    chunk of 8192 amplitudes (n=9, partly masked chunk), an integer n=17 and a
    real-valued n=16 table (shift s > 0, k_c != 0), each called twice."""
    ctx = q.qaoa_ctx_create(0)
    try:
        for Q, p in ((inst.upper_int_qubo(9, 31), 2), (inst.upper_int_qubo(17, 32), 3), (inst.normal_qubo(16, 33), 2)):
            c = _case(q, ctx, Q, p, caller_copy=False)
            F = oracle.cost_table(oracle.canonical_of(Q))
            Eo = oracle.expectation(F, oracle.evolve(F, c["g"], c["b"]))
            ref = q.qaoa_expect(ctx, c["cost"], c["st"])
            for _ in range(2):
                got = _noalloc(q, c)
                assert got == ref
                assert abs(got - Eo) <= E_TOL * np.abs(F).max()
            _drop(q, c)
    finally:
        q.qaoa_ctx_destroy(ctx)


def test_noalloc_largest_size(q):
    """n=30, the largest size the fixed array holds: the partial sums fill it
    up to the final slots; equal to qaoa_expect twice in a row, on the cost
    handle's own table, and bounded by min F <= E <= max F."""
    import torch
    ctx = q.qaoa_ctx_create(0)
    try:
        Q = inst.normal_qubo(30, 1003)
        c = _case(q, ctx, Q, 1, seed_scale=0.3, caller_copy=False)
        ref = q.qaoa_expect(ctx, c["cost"], c["st"])
        assert _noalloc(q, c) == ref
        assert _noalloc(q, c) == ref
        info = c["info"]
        assert info["min_cost"] <= ref
        _drop(q, c)
        torch.cuda.synchronize()
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
    host = np.zeros(16, dtype=np.float32)
    with pytest.raises(q.QaoaError) as e:  # host memory is refused before any launch
        q.qaoa_expect_noalloc(host.ctypes.data, tab.data_ptr(), 3, 0, 0)
    assert e.value.status == q.QAOA_ERR_INVALID_ARG
