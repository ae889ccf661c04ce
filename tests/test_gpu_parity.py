"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances: integer work (objective tables, argmin, top-K indices, counts)
bit-exact; complex64 amplitudes: L2 error <= 1e-5; expectation:
|dE| / max|F| <= 1e-5; gradient: max_l |dg_l| / max(|g|_inf, 1e-12) <= 1e-4.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_26297_b300 import instances as inst

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
E_TOL = 1e-5
G_TOL = 1e-4


@pytest.fixture(scope="module")
def q():
    from paper_2606_26297_b300 import build_lib
    build_lib.build()
    from paper_2606_26297_b300 import qaoa
    return qaoa


@pytest.fixture(scope="module")
def ctx(q):
    c = q.qaoa_ctx_create(0)
    yield c
    q.qaoa_ctx_destroy(c)


def _cost(q, ctx, Q):
    return q.qaoa_build_cost(ctx, Q.H, Q.f, Q.c0, "i32" if Q.dtype == "i32" else "f32")


def _table_error_bound(n, s):
    return (1 + n + n * (n - 1) / 2) * 2.0 ** (-(s + 1))


# ---- objective table ---------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 12, 13, 14, 17, 20])
def test_cost_table_integer_bitexact(q, ctx, n):
    Q = inst.upper_int_qubo(n, 500 + n)
    cost = _cost(q, ctx, Q)
    info = q.qaoa_cost_info(cost)
    T = q.qaoa_cost_copy_to_host(ctx, cost, n).astype(np.int64)
    F = oracle.cost_table(oracle.canonical_of(Q))
    assert info["shift_bits"] == 0
    assert np.array_equal(T + info["k_c"], F.astype(np.int64))
    assert info["argmin"] == oracle.argmin(F)
    assert info["min_cost"] == F.min()
    q.qaoa_cost_destroy(cost)


def test_cost_table_nonsymmetric_input(q, ctx):
    """H with both triangles and f and c0: canonicalisation (Sec. 2.1)."""
    rng = inst.SplitMix64(4)
    n = 13
    H = np.array([[rng.randint(-7, 7) for _ in range(n)] for _ in range(n)], dtype=float)
    f = np.array([rng.randint(-7, 7) for _ in range(n)], dtype=float)
    cost = q.qaoa_build_cost(ctx, H, f, 5.0, "i32")
    info = q.qaoa_cost_info(cost)
    T = q.qaoa_cost_copy_to_host(ctx, cost, n).astype(np.int64)
    F = oracle.cost_table(oracle.canonicalize(H, f, 5.0))
    assert np.array_equal(T + info["k_c"], F.astype(np.int64))
    q.qaoa_cost_destroy(cost)


@pytest.mark.parametrize("maker,n", [(inst.normal_qubo, 14), (inst.unit_commitment_qubo, 16)])
def test_cost_table_real_within_bound(q, ctx, maker, n):
    Q = maker(n, 600 + n)
    cost = _cost(q, ctx, Q)
    info = q.qaoa_cost_info(cost)
    T = q.qaoa_cost_copy_to_host(ctx, cost, n).astype(np.float64)
    Fg = (T + info["k_c"]) * 2.0 ** (-info["shift_bits"])
    F = oracle.cost_table(oracle.canonical_of(Q))
    assert np.max(np.abs(Fg - F)) <= _table_error_bound(n, info["shift_bits"])
    assert abs(F[info["argmin"]] - F.min()) <= 2 * _table_error_bound(n, info["shift_bits"])
    q.qaoa_cost_destroy(cost)


@pytest.mark.parametrize("n,kind", [(14, "int"), (15, "big"), (18, "normal"), (22, "int"), (24, "uc"),
                                    (26, "big"), (29, "normal")])
def test_table_tensor_core_matches_simt(q, n, kind):
    """The tcgen05 build (digit-split f16 products, exact FP32 accumulation)
    against the integer SIMT build of the same fixed-point table: bit-exact
    tables, argmin and minimum.  'big' has couplings up to 5e4, which need two
    base-2^11 digits."""
    if kind == "int":
        Q = inst.upper_int_qubo(n, 900 + n)
    elif kind == "big":
        Q = inst.upper_int_qubo(n, 900 + n, lo=-50000, hi=50000)
    elif kind == "normal":
        Q = inst.normal_qubo(n, 900 + n)
    else:
        Q = inst.unit_commitment_qubo(n, 900 + n)
    dt = "i32" if Q.dtype == "i32" else "f32"
    c_tc = q.qaoa_ctx_create(0)
    c_si = q.qaoa_ctx_create(0, table_build=1)
    k_tc = q.qaoa_build_cost(c_tc, Q.H, Q.f, Q.c0, dt)
    k_si = q.qaoa_build_cost(c_si, Q.H, Q.f, Q.c0, dt)
    assert q.qaoa_cost_info(k_tc) == q.qaoa_cost_info(k_si)
    T_tc = q.qaoa_cost_copy_to_host(c_tc, k_tc, n)
    T_si = q.qaoa_cost_copy_to_host(c_si, k_si, n)
    assert np.array_equal(T_tc, T_si)
    if n <= 22:
        info = q.qaoa_cost_info(k_tc)
        F = oracle.cost_table(oracle.canonical_of(Q))
        if Q.dtype == "i32":
            assert np.array_equal(T_tc.astype(np.int64) + info["k_c"], F.astype(np.int64))
        else:
            s = info["shift_bits"]
            got = (T_tc.astype(np.float64) + info["k_c"]) * 2.0 ** (-s)
            assert np.max(np.abs(got - F)) <= _table_error_bound(n, s)
    for k, c in ((k_tc, c_tc), (k_si, c_si)):
        q.qaoa_cost_destroy(k)
        q.qaoa_ctx_destroy(c)


# ---- forward state -------------------------------------------------------------------

FWD_CASES = [
    (4, 1, "int"), (9, 2, "normal"), (12, 2, "int"),             # shared-memory resident path
    (13, 1, "int"), (13, 3, "normal"), (14, 2, "int"), (16, 3, "normal"),
    (18, 2, "maxcut"), (20, 3, "int"), (21, 2, "normal"), (23, 4, "int"),   # layer-pass path
]


def _instance(kind, n, seed):
    if kind == "int":
        return inst.upper_int_qubo(n, seed)
    if kind == "normal":
        return inst.normal_qubo(n, seed)
    return inst.regular_maxcut_qubo(n, seed)


def _angles(Q, p, kind):
    scale = 1.0 if kind != "normal" else math.sqrt(Q.n) / inst.coefficient_norm(Q)
    if kind == "int":
        scale = 0.15
    return inst.ramp_angles(p, gamma_scale=scale)


@pytest.mark.parametrize("n,p,kind", FWD_CASES)
def test_forward_amplitudes_and_expectation(q, ctx, n, p, kind):
    Q = _instance(kind, n, 700 + n + p)
    g, b = _angles(Q, p, kind)
    cost = _cost(q, ctx, Q)
    st = q.qaoa_forward(ctx, cost, g, b)
    psi = q.qaoa_state_copy_to_host(ctx, st, n).astype(np.complex128)
    F = oracle.cost_table(oracle.canonical_of(Q))
    ref = oracle.evolve(F, g, b)
    assert np.linalg.norm(psi - ref) <= AMP_TOL
    E = q.qaoa_expect(ctx, cost, st)
    assert abs(E - oracle.expectation(F, ref)) / np.max(np.abs(F)) <= E_TOL
    q.qaoa_state_destroy(st)
    q.qaoa_cost_destroy(cost)


def test_forward_fp64_state_small(q):
    """n=12, p=2 with a complex128 state (the dense integer n=12 workload)."""
    c = q.qaoa_ctx_create(0, state_fp64=True)
    Q, g, b = inst.workload_small_int()
    cost = _cost(q, c, Q)
    st = q.qaoa_forward(c, cost, g, b)
    psi = q.qaoa_state_copy_to_host(c, st, 12, fp64=True)
    F = oracle.cost_table(oracle.canonical_of(Q))
    ref = oracle.evolve(F, g, b)
    assert np.linalg.norm(psi - ref) <= 1e-12
    E, dg, db = q.qaoa_grad(c, cost, g, b)
    Eo, dgo, dbo = oracle.grad_adjoint(F, g, b)
    assert abs(E - Eo) <= 1e-10 * np.max(np.abs(F))
    sc = max(np.max(np.abs(dgo)), np.max(np.abs(dbo)))
    assert max(np.max(np.abs(dg - dgo)), np.max(np.abs(db - dbo))) <= 1e-9 * sc
    q.qaoa_state_destroy(st)
    q.qaoa_cost_destroy(cost)
    q.qaoa_ctx_destroy(c)


def test_p0_is_uniform(q, ctx):
    for n in (5, 15):
        Q = inst.upper_int_qubo(n, 3)
        cost = _cost(q, ctx, Q)
        st = q.qaoa_forward(ctx, cost, [], [])
        psi = q.qaoa_state_copy_to_host(ctx, st, n)
        assert np.max(np.abs(psi - 2.0 ** (-n / 2))) < 1e-7
        F = oracle.cost_table(oracle.canonical_of(Q))
        assert abs(q.qaoa_expect(ctx, cost, st) - F.mean()) <= E_TOL * np.max(np.abs(F))
        q.qaoa_state_destroy(st)
        q.qaoa_cost_destroy(cost)


def test_gamma_zero_global_phase(q, ctx):
    n = 16
    Q = inst.normal_qubo(n, 9)
    cost = _cost(q, ctx, Q)
    beta = [0.3, 1.1, -0.7]
    st = q.qaoa_forward(ctx, cost, [0.0, 0.0, 0.0], beta)
    psi = q.qaoa_state_copy_to_host(ctx, st, n).astype(np.complex128)
    ref = np.exp(-1j * n * sum(beta)) * 2.0 ** (-n / 2)
    assert np.linalg.norm(psi - ref) <= AMP_TOL
    q.qaoa_state_destroy(st)
    q.qaoa_cost_destroy(cost)


# ---- gradient ----------------------------------------------------------------------------

GRAD_CASES = [(8, 2, "int"), (12, 3, "normal"), (13, 1, "int"), (13, 2, "normal"), (14, 3, "maxcut"),
              (16, 4, "int"), (18, 2, "normal"), (21, 3, "int"), (22, 2, "normal")]


@pytest.mark.parametrize("n,p,kind", GRAD_CASES)
def test_gradient_vs_oracle(q, ctx, n, p, kind):
    Q = _instance(kind, n, 800 + n + p)
    g, b = _angles(Q, p, kind)
    cost = _cost(q, ctx, Q)
    E, dg, db = q.qaoa_grad(ctx, cost, g, b)
    F = oracle.cost_table(oracle.canonical_of(Q))
    Eo, dgo, dbo = oracle.grad_adjoint(F, g, b)
    assert abs(E - Eo) / np.max(np.abs(F)) <= E_TOL
    sc = max(np.max(np.abs(dgo)), np.max(np.abs(dbo)), 1e-12)
    err = max(np.max(np.abs(dg - dgo)), np.max(np.abs(db - dbo))) / sc
    assert err <= G_TOL, (err, dg, dgo, db, dbo)
    q.qaoa_cost_destroy(cost)


def test_gradient_special_cases(q, ctx):
    Q = inst.upper_int_qubo(15, 41)
    cost = _cost(q, ctx, Q)
    _, dg, db = q.qaoa_grad(ctx, cost, [0.0, 0.0], [0.4, 1.2])
    assert np.max(np.abs(db)) < 1e-4
    _, dg, db = q.qaoa_grad(ctx, cost, [0.05, 0.09], [0.0, 0.0])
    assert np.max(np.abs(dg)) < 1e-4 * max(1.0, np.max(np.abs(q.qaoa_grad(ctx, cost, [0.05, 0.09], [0.3, 0.2])[1])))
    q.qaoa_cost_destroy(cost)


def test_grad_deterministic(q, ctx):
    Q = inst.normal_qubo(19, 5)
    g, b = _angles(Q, 3, "normal")
    cost = _cost(q, ctx, Q)
    r1 = q.qaoa_grad(ctx, cost, g, b, k_top=8)
    r2 = q.qaoa_grad(ctx, cost, g, b, k_top=8)
    assert r1[0] == r2[0]
    assert np.array_equal(r1[1], r2[1]) and np.array_equal(r1[2], r2[2])
    assert np.array_equal(r1[3], r2[3]) and np.array_equal(r1[4], r2[4])
    q.qaoa_cost_destroy(cost)


# ---- top-K -------------------------------------------------------------------------------

def _cpu_topk(P, k):
    return np.lexsort((np.arange(P.shape[0]), -P))[:k]


@pytest.mark.parametrize("n,k", [(10, 8), (14, 10), (17, 16), (20, 64)])
def test_topk_bitexact_on_gpu_probabilities(q, ctx, n, k):
    Q = inst.upper_int_qubo(n, 900 + n)
    g, b = _angles(Q, 2, "int")
    cost = _cost(q, ctx, Q)
    st = q.qaoa_forward(ctx, cost, g, b)
    psi = q.qaoa_state_copy_to_host(ctx, st, n)
    res = q.qaoa_topk(ctx, cost, st, k)
    # bit-exact against a CPU selection on the GPU's own probabilities (same FP32 key)
    ref = _cpu_topk(res_prob_array(psi), k)
    assert list(res["idx"]) == list(ref)
    # against the oracle: equal as tie groups (probabilities within 1e-6 max P)
    F = oracle.cost_table(oracle.canonical_of(Q))
    Po = oracle.probabilities(oracle.evolve(F, g, b))
    thr = 1e-6 * Po.max()
    kth = np.sort(Po)[::-1][k - 1]
    for x in res["idx"]:
        assert Po[x] >= kth - thr
    assert res["argmin"] == oracle.argmin(F)
    assert np.allclose(res["cost"], F[res["idx"].astype(np.int64)])
    q.qaoa_state_destroy(st)
    q.qaoa_cost_destroy(cost)


def res_prob_array(psi):
    """|psi|^2 as the kernels form it: fmaf(re, re, im*im) in FP32 (the
    product re*re is exact in extended precision, then one rounding)."""
    re = psi.real.astype(np.float32)
    im = psi.imag.astype(np.float32)
    im2 = (im * im).astype(np.float32)
    return (re.astype(np.longdouble) * re.astype(np.longdouble) + im2.astype(np.longdouble)).astype(np.float32)


def test_fused_topk_matches_state_topk(q, ctx):
    n = 18
    Q = inst.regular_maxcut_qubo(n, 12)
    g, b = inst.ramp_angles(3)
    cost = _cost(q, ctx, Q)
    _, _, _, ti, tp = q.qaoa_grad(ctx, cost, g, b, k_top=10)
    st = q.qaoa_forward(ctx, cost, g, b)
    res = q.qaoa_topk(ctx, cost, st, 10)
    F = oracle.cost_table(oracle.canonical_of(Q))
    Po = oracle.probabilities(oracle.evolve(F, g, b))
    kth = np.sort(Po)[::-1][9]
    for x in ti:
        assert Po[x] >= kth - 1e-6 * Po.max()
    assert np.allclose(tp, res["prob"], rtol=1e-4, atol=1e-9)
    q.qaoa_state_destroy(st)
    q.qaoa_cost_destroy(cost)


# ---- DQAOA ---------------------------------------------------------------------------------

@pytest.mark.parametrize("maker,n,M", [(inst.upper_int_qubo, 16, 3), (inst.normal_qubo, 15, 4),
                                      (inst.unit_commitment_qubo, 14, 2)])
def test_factorisation_check(q, ctx, maker, n, M):
    Q = maker(n, 1100 + n)
    cost = _cost(q, ctx, Q)
    qpu_of = q.qaoa_partition(n, M)
    mism, perr = q.qaoa_check_factorisation(ctx, cost, qpu_of, 0.8)
    assert mism == 0
    assert perr < 1e-5
    loc = q.qaoa_classify(cost, qpu_of, 5)
    assert (loc["local"], loc["cross"], loc["remote_cx"]) == oracle.classify(oracle.canonical_of(Q), list(qpu_of), 5)
    q.qaoa_cost_destroy(cost)


def test_dense30_partition_counts_through_abi(q, ctx):
    """Dense n=30 (N(0,1) couplings), caps [10,10,10] contiguous: 135 local,
    300 cross, 4800 remote CX at p=8 (Sec. 3.1).  Uses a small n=30 handle."""
    Q = inst.normal_qubo(30, 1003)
    cost = _cost(q, ctx, Q)
    qpu_of = q.qaoa_partition(30, 3, caps=[10, 10, 10])
    r = q.qaoa_classify(cost, qpu_of, 8)
    assert (r["local"], r["cross"], r["remote_cx"]) == (135, 300, 4800)
    q.qaoa_cost_destroy(cost)


# ---- boundary error paths ---------------------------------------------------------------------

def test_error_paths(q, ctx):
    Q = inst.upper_int_qubo(14, 1)
    cost = _cost(q, ctx, Q)
    with pytest.raises(q.QaoaError) as e:
        q.qaoa_grad(ctx, cost, [], [])
    assert e.value.status == q.QAOA_ERR_INVALID_ARG
    with pytest.raises(q.QaoaError):
        q.qaoa_grad(ctx, cost, [0.1], [float("nan")])
    st = q.qaoa_forward(ctx, cost, [0.1], [0.2])
    with pytest.raises(q.QaoaError):
        q.qaoa_topk(ctx, cost, st, 0)
    with pytest.raises(q.QaoaError):
        q.qaoa_topk(ctx, cost, st, 65)
    Q2 = inst.upper_int_qubo(15, 1)
    cost2 = _cost(q, ctx, Q2)
    with pytest.raises(q.QaoaError):
        q.qaoa_expect(ctx, cost2, st)
    with pytest.raises(q.QaoaError) as e:
        q.qaoa_build_cost(ctx, np.zeros((34, 34)), None, 0.0, "f64")
    assert e.value.status == q.QAOA_ERR_INVALID_ARG
    with pytest.raises(q.QaoaError) as e:
        q.qaoa_build_cost(ctx, np.full((3, 3), 2 ** 30), None, 0.0, "i32")
    assert e.value.status == q.QAOA_ERR_RANGE
    # batch, optimiser, gather, tuner and option arguments
    with pytest.raises(q.QaoaError):
        q.qaoa_grad_batch(ctx, [cost], np.zeros((0, 2)), np.zeros((0, 2)))
    with pytest.raises(q.QaoaError):
        q.qaoa_grad_batch(ctx, [cost], np.zeros((2, 1)), np.zeros((2, 1)), item_cost=[0, 3])
    with pytest.raises(q.QaoaError):
        q.qaoa_optimize_adam(ctx, [cost], np.zeros((1, 2)), np.zeros((1, 2)), 0)
    with pytest.raises(q.QaoaError):
        q.qaoa_state_gather(ctx, st, [1 << 14])
    small = _cost(q, ctx, inst.upper_int_qubo(8, 2))
    with pytest.raises(q.QaoaError):
        q.qaoa_autotune(ctx, small, 2)
    q.qaoa_cost_destroy(small)
    for kw in ({"adjoint_mode": 3}, {"table_build": 2}, {"max_fused_qubits": 11}, {"max_fused_qubits": 2}):
        with pytest.raises(q.QaoaError) as e:
            q.qaoa_ctx_create(0, **kw)
        assert e.value.status == q.QAOA_ERR_INVALID_ARG
    q.qaoa_state_destroy(st)
    q.qaoa_cost_destroy(cost)
    q.qaoa_cost_destroy(cost2)


# ---- fusion depth -----------------------------------------------------------------------------

@pytest.mark.parametrize("n,p,kind", [(13, 2, "normal"), (17, 3, "int"), (22, 2, "maxcut")])
def test_fusion_depth_agrees(q, n, p, kind):
    """The mixer factorises over qubits (Eq. qaoa_mixer_unitary), so every
    grouping of the qubits into fused passes gives the same state up to
    rounding: 10, 6 and 4 qubits per pass against each other and the oracle."""
    Q = _instance(kind, n, 1200 + n)
    g, b = _angles(Q, p, kind)
    F = oracle.cost_table(oracle.canonical_of(Q))
    ref = oracle.evolve(F, g, b)
    Eo, dgo, dbo = oracle.grad_adjoint(F, g, b)
    for k in (10, 6, 4):
        c = q.qaoa_ctx_create(0, max_fused_qubits=k)
        cost = _cost(q, c, Q)
        st = q.qaoa_forward(c, cost, g, b)
        psi = q.qaoa_state_copy_to_host(c, st, n).astype(np.complex128)
        assert np.linalg.norm(psi - ref) <= AMP_TOL
        E, dg, db = q.qaoa_grad(c, cost, g, b)
        assert abs(E - Eo) / np.max(np.abs(F)) <= E_TOL
        sc = max(np.max(np.abs(dgo)), np.max(np.abs(dbo)))
        assert max(np.max(np.abs(dg - dgo)), np.max(np.abs(db - dbo))) <= G_TOL * sc
        q.qaoa_state_destroy(st)
        q.qaoa_cost_destroy(cost)
        q.qaoa_ctx_destroy(c)


@pytest.mark.parametrize("maxq", [10, 6])
def test_split_windows_n24(q, maxq):
    """From n = 24 the high groups take one 5-bit window from the lower and one
    from the upper half of the high bits; state and gradient against the
    oracle for 3 (width 10) and 4 (width 6) groups."""
    n, p = 24, 2
    Q = inst.normal_qubo(n, 1300)
    g, b = _angles(Q, p, "normal")
    c = q.qaoa_ctx_create(0, max_fused_qubits=maxq)
    cost = _cost(q, c, Q)
    F = oracle.cost_table(oracle.canonical_of(Q))
    st = q.qaoa_forward(c, cost, g, b)
    psi = q.qaoa_state_copy_to_host(c, st, n).astype(np.complex128)
    assert np.linalg.norm(psi - oracle.evolve(F, g, b)) <= AMP_TOL
    E, dg, db = q.qaoa_grad(c, cost, g, b)
    Eo, dgo, dbo = oracle.grad_adjoint(F, g, b)
    assert abs(E - Eo) / np.max(np.abs(F)) <= E_TOL
    sc = max(np.max(np.abs(dgo)), np.max(np.abs(dbo)))
    assert max(np.max(np.abs(dg - dgo)), np.max(np.abs(db - dbo))) <= G_TOL * sc
    q.qaoa_state_destroy(st)
    q.qaoa_cost_destroy(cost)
    q.qaoa_ctx_destroy(c)


@pytest.mark.parametrize("n,p,kind,maxq", [(13, 2, "normal", 10), (18, 3, "int", 10), (22, 3, "maxcut", 10),
                                          (24, 2, "normal", 10), (20, 2, "int", 6), (17, 4, "normal", 4)])
def test_adjoint_modes_agree(q, n, p, kind, maxq):
    """Stored forward states (lambda alone through mixer-only passes) and the
    uncompute sweep give the same E and gradient, both against the oracle;
    2 to 5 qubit groups."""
    Q = _instance(kind, n, 1400 + n)
    g, b = _angles(Q, p, kind)
    F = oracle.cost_table(oracle.canonical_of(Q))
    Eo, dgo, dbo = oracle.grad_adjoint(F, g, b)
    sc = max(np.max(np.abs(dgo)), np.max(np.abs(dbo)))
    res = {}
    for mode in (q.QAOA_ADJ_UNCOMPUTE, q.QAOA_ADJ_STORE):
        c = q.qaoa_ctx_create(0, adjoint_mode=mode, max_fused_qubits=maxq)
        cost = _cost(q, c, Q)
        E, dg, db, ti, tp = q.qaoa_grad(c, cost, g, b, k_top=4)
        assert abs(E - Eo) / np.max(np.abs(F)) <= E_TOL
        assert max(np.max(np.abs(dg - dgo)), np.max(np.abs(db - dbo))) <= G_TOL * sc
        Eb, dgb, dbb = q.qaoa_grad_batch(c, [cost], np.stack([g, g * 0.5]), np.stack([b, b]))
        assert abs(Eb[0] - Eo) / np.max(np.abs(F)) <= E_TOL
        assert max(np.max(np.abs(dgb[0] - dgo)), np.max(np.abs(dbb[0] - dbo))) <= G_TOL * sc
        res[mode] = (E, dg, db, ti, Eb, dgb, dbb)
        q.qaoa_cost_destroy(cost)
        q.qaoa_ctx_destroy(c)
    (E1, dg1, db1, t1, Eb1, dgb1, dbb1), (E2, dg2, db2, t2, Eb2, dgb2, dbb2) = res.values()
    assert abs(E1 - E2) <= 1e-6 * np.max(np.abs(F))
    assert max(np.abs(dg1 - dg2).max(), np.abs(db1 - db2).max()) <= 1e-5 * sc
    assert np.array_equal(t1, t2)
    assert np.max(np.abs(Eb1 - Eb2)) <= 1e-6 * np.max(np.abs(F))


@pytest.mark.parametrize("n,p,kind,maxq,mode", [(13, 2, "normal", 10, 2), (18, 3, "int", 10, 1),
                                               (24, 2, "normal", 10, 2), (24, 2, "normal", 10, 1),
                                               (20, 2, "int", 6, 1), (17, 4, "normal", 4, 2),
                                               (22, 3, "maxcut", 8, 2)])
def test_reverse_block_layouts_agree(q, n, p, kind, maxq, mode):
    """The final and reverse cost-layer passes on half blocks of 2^12
    amplitudes (two CTAs per SM) for the low group (the default), on blocks of
    2^13 (one CTA per SM) everywhere, and on half blocks everywhere give the
    same E and gradient up to summation order, all against the oracle: low and
    high groups, full and partial groups, adjacent and split windows, stored
    states and the uncompute sweep, single and batched requests."""
    Q = _instance(kind, n, 1500 + n)
    g, b = _angles(Q, p, kind)
    F = oracle.cost_table(oracle.canonical_of(Q))
    Eo, dgo, dbo = oracle.grad_adjoint(F, g, b)
    sc = max(np.max(np.abs(dgo)), np.max(np.abs(dbo)))
    res = []
    for layout in (0, 1, 2):
        c = q.qaoa_ctx_create(0, adjoint_mode=mode, max_fused_qubits=maxq, reverse_blocks=layout)
        cost = _cost(q, c, Q)
        E, dg, db = q.qaoa_grad(c, cost, g, b)
        assert abs(E - Eo) / np.max(np.abs(F)) <= E_TOL
        assert max(np.max(np.abs(dg - dgo)), np.max(np.abs(db - dbo))) <= G_TOL * sc
        Eb, dgb, dbb = q.qaoa_grad_batch(c, [cost], np.stack([g, g * 0.7, g * 1.2]), np.stack([b, b * 0.9, b]))
        assert abs(Eb[0] - Eo) / np.max(np.abs(F)) <= E_TOL
        assert max(np.max(np.abs(dgb[0] - dgo)), np.max(np.abs(dbb[0] - dbo))) <= G_TOL * sc
        res.append((E, dg, db, Eb, dgb, dbb))
        q.qaoa_cost_destroy(cost)
        q.qaoa_ctx_destroy(c)
    # the layouts give each thread different amplitudes, so the FP32 partial
    # sums round differently: agreement to FP32 rounding, well inside the bounds
    E0, dg0, db0, Eb0, dgb0, dbb0 = res[0]
    for E1, dg1, db1, Eb1, dgb1, dbb1 in res[1:]:
        assert abs(E0 - E1) <= 1e-7 * np.max(np.abs(F))
        assert max(np.abs(dg0 - dg1).max(), np.abs(db0 - db1).max()) <= 1e-5 * sc
        assert np.max(np.abs(Eb0 - Eb1)) <= 1e-7 * np.max(np.abs(F))
        assert max(np.abs(dgb0 - dgb1).max(), np.abs(dbb0 - dbb1).max()) <= 1e-5 * sc


def test_adjoint_keeps_what_fits(q):
    """Between the two adjoint forms: under a memory budget the automatic
    choice keeps the inputs of as many of the last mixer-only passes as fit and
    uncomputes the rest.  Budgets from below the uncompute sweep's need to above
    the fully stored form's: every evaluation that runs matches the oracle, the
    number of mixer-only reverse passes on lambda alone (profile kind 12) never
    falls as the budget grows, and some budget gives a mixed sweep (four qubit
    groups, n = 20, p = 3: six mixer-only passes)."""
    n, p = 20, 3
    Q = inst.normal_qubo(n, 1600)
    g, b = _angles(Q, p, "normal")
    F = oracle.cost_table(oracle.canonical_of(Q))
    Eo, dgo, dbo = oracle.grad_adjoint(F, g, b)
    sc = max(np.max(np.abs(dgo)), np.max(np.abs(dbo)))
    N8 = 8 << n
    kept = []
    for j in range(0, 24):
        budget = 40 * N8 // 8 + j * N8 // 2
        c = q.qaoa_ctx_create(0, max_fused_qubits=6, memory_budget=budget, profile=True)
        cost = None
        try:
            try:
                cost = _cost(q, c, Q)
                E, dg, db = q.qaoa_grad(c, cost, g, b)
            except q.QaoaError as e:
                assert e.status == q.QAOA_ERR_OUT_OF_MEMORY
                continue
            assert abs(E - Eo) / np.max(np.abs(F)) <= E_TOL
            assert max(np.max(np.abs(dg - dgo)), np.max(np.abs(db - dbo))) <= G_TOL * sc
            kept.append(q.qaoa_profile_read(c, 12)["launches"])
        finally:
            if cost is not None:
                q.qaoa_cost_destroy(cost)
            q.qaoa_ctx_destroy(c)
    assert kept, "no budget in the sweep ran"
    assert kept == sorted(kept)
    assert kept[0] == 0 and kept[-1] == 6
    assert any(0 < k < 6 for k in kept), kept


@pytest.mark.parametrize("n,p,maxq,mode", [(20, 3, 6, 2), (20, 3, 6, 1), (24, 2, 10, 2), (17, 2, 4, 2)])
def test_launches_follow_the_described_plan(q, n, p, maxq, mode):
    """The kernels a gradient launches are the passes qaoa_plan_describe lists
    (the CPU tests check that plan): forward passes (kinds 8, 9), the final
    pass (10, 13), reverse passes on (psi, lambda) (11, 14) and on lambda alone
    (12), one launch each."""
    Q = inst.normal_qubo(n, 1700 + n)
    g, b = _angles(Q, p, "normal")
    stored = -1 if mode == 2 else 0
    plan, _, _ = q.qaoa_plan_describe(n, p, grad=True, max_fused_qubits=maxq, stored_mids=stored)
    want = {k: sum(ps["kind"] == k for ps in plan) for k in range(4)}
    c = q.qaoa_ctx_create(0, adjoint_mode=mode, max_fused_qubits=maxq, profile=True)
    try:
        cost = _cost(q, c, Q)
        q.qaoa_grad(c, cost, g, b)
        got = {kk: q.qaoa_profile_read(c, kk)["launches"] for kk in range(8, 15)}
        assert got[8] + got[9] == want[0]
        assert got[10] + got[13] == want[1] == 1
        assert got[11] + got[14] == want[2]
        assert got[12] == want[3]
        q.qaoa_cost_destroy(cost)
    finally:
        q.qaoa_ctx_destroy(c)


def test_factorisation_noncontiguous(q, ctx):
    """A manual (non-contiguous) allocation goes through the general check."""
    n = 14
    Q = inst.normal_qubo(n, 77)
    cost = _cost(q, ctx, Q)
    manual = [(i * 7) % 3 for i in range(n)]
    qpu_of = q.qaoa_partition(n, 3, caps=[5, 5, 5], manual=manual)
    mism, perr = q.qaoa_check_factorisation(ctx, cost, qpu_of, 1.3)
    assert mism == 0 and perr < 1e-5
    q.qaoa_cost_destroy(cost)


def _int32_view(ptr, count):
    """A torch view of device memory owned by the library (for planting edits)."""
    import torch

    class _Raw:
        __cuda_array_interface__ = {"shape": (count,), "typestr": "<i4", "data": (ptr, False),
                                    "version": 3, "strides": None}
    return torch.as_tensor(_Raw(), device="cuda")


@pytest.mark.parametrize("n,caps,manual", [
    (20, [10, 10], None),            # contiguous, QPU 0 of 10 variables: tiled kernel
    (22, [11, 6, 5], None),          # contiguous, QPU 0 of 11: tiled kernel with a bit above the tile
    (16, [6, 5, 5], None),           # contiguous, QPU 0 of 6: row kernel
    (14, [5, 5, 5], [(i * 7) % 3 for i in range(14)]),  # manual: general kernel
])
def test_factorisation_check_detects_edited_entries(q, ctx, n, caps, manual):
    """Sec. 3.2, Eq. local_cross_rule: the check counts exactly the entries of
    the table that no longer split into local and cross-QPU parts.  Entries
    are edited on the host side through the table's device address (no GPU
    fault involved), counted, then restored."""
    import torch
    Q = inst.normal_qubo(n, 4200 + n)
    cost = _cost(q, ctx, Q)
    qpu_of = q.qaoa_partition(n, len(caps), caps=caps, manual=manual)
    assert q.qaoa_check_factorisation(ctx, cost, qpu_of, 0.9)[0] == 0
    ptr, count = q.qaoa_cost_device_ptr(cost)
    assert count == 1 << n
    T = _int32_view(ptr, count)
    N = 1 << n
    edits = sorted({0, 1, 2, 3, 1023, 1024, N // 2 + 5, N - 1} | set(np.random.default_rng(n).integers(0, N, 20).tolist()))
    idx = torch.tensor(edits, dtype=torch.int64, device="cuda")
    saved = T[idx].clone()
    T[idx] = saved + torch.tensor([(-1) ** k * (1 + k) for k in range(len(edits))], dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    mism, _ = q.qaoa_check_factorisation(ctx, cost, qpu_of, 0.9)
    assert mism == len(edits)
    T[idx] = saved
    torch.cuda.synchronize()
    mism, perr = q.qaoa_check_factorisation(ctx, cost, qpu_of, 0.9)
    assert mism == 0 and perr < 1e-5
    q.qaoa_cost_destroy(cost)


def test_peak_probe_rates(q):
    """The arithmetic-pipe probe returns finite positive rates for every kind
    and rejects an unknown kind; FP32 FMA runs far faster than FP64 FMA on this
    part."""
    ctx = q.qaoa_ctx_create(0)
    rates = [q.qaoa_peak_probe(ctx, k) for k in range(4)]
    for ops, flops in rates:
        assert np.isfinite(ops) and ops > 0 and flops >= ops
    assert rates[0][1] > 4 * rates[2][1]
    with pytest.raises(q.QaoaError):
        q.qaoa_peak_probe(ctx, 4)
    q.qaoa_ctx_destroy(ctx)


def test_bounded_wait_expires_and_context_survives(q):
    """Failure path of the device waits without a GPU fault: a wait on a copy
    that is never issued runs out (QAOA_ERR_TIMEOUT from the status word), and
    the same context then evaluates a gradient that matches the oracle."""
    ctx = q.qaoa_ctx_create(0)
    with pytest.raises(q.QaoaError) as ei:
        q.qaoa_wait_probe(ctx)
    assert ei.value.status == q.QAOA_ERR_TIMEOUT
    Q = inst.upper_int_qubo(14, 9090)
    cost = q.qaoa_build_cost(ctx, Q.H, Q.f, Q.c0, "i32")
    g, b = inst.ramp_angles(2, gamma_scale=0.2)
    E, dg, db = q.qaoa_grad(ctx, cost, g, b)
    F = oracle.cost_table(oracle.canonical_of(Q))
    Eo, dgo, dbo = oracle.grad_adjoint(F, g, b)
    assert abs(E - Eo) / np.max(np.abs(F)) <= 1e-5
    q.qaoa_cost_destroy(cost)
    q.qaoa_ctx_destroy(ctx)
