"""Thin Python binding of the C ABI in include/qaoa.h.

Argument marshalling only: every function has the name of its C entry point,
converts numpy / torch arguments to plain pointers, calls the library, and
raises QaoaError on a non-zero status.  All computation happens in
libqaoa.so (CUDA, sm_103a); if the library is missing, importing this module
fails loudly.  There is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqaoa.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2606_26297_b300.build_lib`")
_lib = ctypes.CDLL(LIB_PATH)

QAOA_OK, QAOA_ERR_INVALID_ARG, QAOA_ERR_OUT_OF_MEMORY, QAOA_ERR_RANGE, QAOA_ERR_CUDA, \
    QAOA_ERR_TIMEOUT, QAOA_ERR_ALLOCATION = range(7)
QAOA_I32, QAOA_F32, QAOA_F64 = 0, 1, 2
QAOA_ADJ_AUTO, QAOA_ADJ_UNCOMPUTE, QAOA_ADJ_STORE = 0, 1, 2
_DTYPES = {"i32": (QAOA_I32, np.int32), "f32": (QAOA_F32, np.float32), "f64": (QAOA_F64, np.float64)}


class QaoaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


class qaoa_qubo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("dtype", ctypes.c_int), ("H", ctypes.c_void_p),
                ("f", ctypes.c_void_p), ("c0", ctypes.c_double)]


class qaoa_options(ctypes.Structure):
    _fields_ = [("adjoint_mode", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("max_fused_qubits", ctypes.c_int32),
                ("state_fp64", ctypes.c_int32), ("table_build", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("reverse_blocks", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class qaoa_pass_info(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("group_type", ctypes.c_int32), ("loA", ctypes.c_int32),
                ("loB", ctypes.c_int32), ("mask", ctypes.c_uint32), ("pre_layer", ctypes.c_int32),
                ("cost_layer", ctypes.c_int32), ("post_layer", ctypes.c_int32), ("in_slot", ctypes.c_int32),
                ("out_slot", ctypes.c_int32), ("psi_slot", ctypes.c_int32), ("lambda_alone_out", ctypes.c_int32),
                ("interleaved_out", ctypes.c_int32), ("slot_param", ctypes.c_int32 * 8),
                ("bytes_per_amp", ctypes.c_double)]


class qaoa_adam_options(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("iterations", ctypes.c_int32), ("disable_graph", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]


class qaoa_sample_metrics(ctypes.Structure):
    _fields_ = [("shots", ctypes.c_int64), ("distinct", ctypes.c_int64), ("mean_cost", ctypes.c_double),
                ("best_cost", ctypes.c_double), ("best_index", ctypes.c_uint64), ("p_best_index", ctypes.c_double),
                ("p_best_cost", ctypes.c_double), ("low_cost_mass", ctypes.c_double),
                ("p_ref_cost", ctypes.c_double), ("p_ref_index", ctypes.c_double),
                ("best_cost_matches_ref", ctypes.c_int32), ("best_index_matches_ref", ctypes.c_int32)]


class qaoa_spsa_options(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("c", ctypes.c_double), ("c_decay", ctypes.c_double),
                ("iterations", ctypes.c_int32), ("shots", ctypes.c_int32), ("averaging", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("seed", ctypes.c_uint64), ("reserved", ctypes.c_int32 * 6)]


class qaoa_solve_options(ctypes.Structure):
    _fields_ = [("p_max", ctypes.c_int32), ("optimizer", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("shots", ctypes.c_int32), ("averaging", ctypes.c_int32), ("random_starts", ctypes.c_int32),
                ("warm_perturb", ctypes.c_int32), ("include_warm", ctypes.c_int32), ("final_shots", ctypes.c_int32),
                ("use_reference", ctypes.c_int32), ("lr", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double), ("c", ctypes.c_double),
                ("c_decay", ctypes.c_double), ("warm_sigma", ctypes.c_double), ("gamma_range", ctypes.c_double),
                ("beta_range", ctypes.c_double), ("margin", ctypes.c_double), ("tol", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("reserved", ctypes.c_int32 * 8)]


class qaoa_solve_result(ctypes.Structure):
    _fields_ = [("best_p", ctypes.c_int32), ("runs", ctypes.c_int32), ("expect", ctypes.c_double),
                ("metrics", qaoa_sample_metrics)]


class qaoa_telegate_counts(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("ops", "local_zz", "cross_zz", "remote_cx", "measurements", "resets",
                                              "feedforward")]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PF = ctypes.POINTER(ctypes.c_float)
_PU64 = ctypes.POINTER(ctypes.c_uint64)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PI32 = ctypes.POINTER(ctypes.c_int32)

_SIGS = {
    "qaoa_ctx_create": ([_I, _P, ctypes.POINTER(qaoa_options), ctypes.POINTER(_P)], _I),
    "qaoa_ctx_destroy": ([_P], None),
    "qaoa_last_error": ([], ctypes.c_char_p),
    "qaoa_build_cost": ([_P, ctypes.POINTER(qaoa_qubo), ctypes.POINTER(_P)], _I),
    "qaoa_cost_destroy": ([_P], None),
    "qaoa_cost_info": ([_P, _PI32, _PI32, _PI64, _PU64, _PD], _I),
    "qaoa_cost_copy_to_host": ([_P, _P, _P], _I),
    "qaoa_cost_device_ptr": ([_P, ctypes.POINTER(_P), _PI64], _I),
    "qaoa_forward": ([_P, _P, _I, _PD, _PD, ctypes.POINTER(_P)], _I),
    "qaoa_state_destroy": ([_P], None),
    "qaoa_state_copy_to_host": ([_P, _P, _P], _I),
    "qaoa_state_device_ptr": ([_P, ctypes.POINTER(_P), _PI64], _I),
    "qaoa_state_gather": ([_P, _P, _PU64, _I, _P], _I),
    "qaoa_expect": ([_P, _P, _P, _PD], _I),
    "qaoa_topk": ([_P, _P, _P, _I, _PU64, _PF, _PD, _PU64, _PD, _PF], _I),
    "qaoa_grad": ([_P, _P, _I, _PD, _PD, _PD, _PD, _PD, _I, _PU64, _PF], _I),
    "qaoa_grad_batch": ([_P, _I, ctypes.POINTER(_P), _PI32, _I, _I, _PD, _PD, _PD, _PD, _PD], _I),
    "qaoa_optimize_adam": ([_P, _I, ctypes.POINTER(_P), _PI32, _I, _I, _PD, _PD,
                            ctypes.POINTER(qaoa_adam_options), _PD, _PD], _I),
    "qaoa_autotune": ([_P, _P, _I, _PI32, _PD], _I),
    "qaoa_optimize_adam_resume": ([_P, _I, ctypes.POINTER(_P), _PI32, _I, _I, _PD, _PD,
                                   ctypes.POINTER(qaoa_adam_options), _PD, _PD, _PD, _PD, _PI32], _I),
    "qaoa_state_from_host": ([_P, _I, _I, _P, ctypes.POINTER(_P)], _I),
    "qaoa_sample": ([_P, _P, _P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, _PU64, _PU64, _PD, _PD], _I),
    "qaoa_sample_stats": ([ctypes.c_int64, _PU64, _PD, _D, _I, _PU64, _PD, _PI64, _I, _D, ctypes.c_uint64, _D,
                           ctypes.POINTER(qaoa_sample_metrics)], _I),
    "qaoa_optimize_spsa": ([_P, _I, ctypes.POINTER(_P), _PI32, _I, _I, _PD, _PD,
                            ctypes.POINTER(qaoa_spsa_options), _PD, _PD], _I),
    "qaoa_solve": ([_P, _P, ctypes.POINTER(qaoa_solve_options), _PD, _PD, _I, _PU64, _PD, _PI64,
                    ctypes.POINTER(qaoa_sample_metrics), ctypes.POINTER(qaoa_solve_result)], _I),
    "qaoa_partition": ([_I, _I, _PI32, _PI32, _PI32], _I),
    "qaoa_plan_describe": ([_I, _I, _I, _I, _I, ctypes.POINTER(qaoa_pass_info), _I, _PI32, _PI32, _PI32], _I),
    "qaoa_telegate_simulate": ([_P, _P, _PI32, _I, _PD, _PD, _I, ctypes.c_uint64, _PD, _PF,
                                ctypes.POINTER(qaoa_telegate_counts)], _I),
    "qaoa_partition_graph": ([ctypes.POINTER(qaoa_qubo), _I, _PI32, _PI32], _I),
    "qaoa_allocation_candidates": ([ctypes.POINTER(qaoa_qubo), _I, _PI32, _PI32, _I, _PI32, _PI32, _PI64, _PI64],
                                   _I),
    "qaoa_classify": ([_P, _PI32, _I, _PI64, _PI64, _PI64, _PI64], _I),
    "qaoa_check_factorisation": ([_P, _P, _PI32, _D, _PI64, _PD], _I),
    "qaoa_profile_read": ([_P, _I, _PI64, _PD, _PD, _I], _I),
    "qaoa_peak_probe": ([_P, _I, _PD, _PD], _I),
    "qaoa_wait_probe": ([_P], _I),
    "qaoa_expect_noalloc": ([_P, _P, _I, ctypes.c_int32, ctypes.c_int64, _P, _PD], _I),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


def _check(status: int) -> None:
    if status != QAOA_OK:
        raise QaoaError(status, _lib.qaoa_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def qaoa_last_error() -> str:
    return _lib.qaoa_last_error().decode()


# ---- context ---------------------------------------------------------------------

def qaoa_ctx_create(device: int = 0, stream: int | None = None, profile: bool = False,
                    memory_budget: int = 0, max_fused_qubits: int = 0, state_fp64: bool = False,
                    table_build: int = 0, autotune: bool = False, adjoint_mode: int = 0,
                    reverse_blocks: int = 0):
    """Create a context; `stream` is a raw cudaStream_t (e.g. torch's
    `torch.cuda.current_stream().cuda_stream`), None for the default stream."""
    opt = qaoa_options()
    opt.profile = int(profile)
    opt.memory_budget = int(memory_budget)
    opt.max_fused_qubits = int(max_fused_qubits)
    opt.state_fp64 = int(state_fp64)
    opt.table_build = int(table_build)
    opt.autotune = int(autotune)
    opt.adjoint_mode = int(adjoint_mode)
    opt.reverse_blocks = int(reverse_blocks)
    out = _P()
    _check(_lib.qaoa_ctx_create(int(device), _P(stream or 0), ctypes.byref(opt), ctypes.byref(out)))
    return out


def qaoa_ctx_destroy(ctx) -> None:
    _lib.qaoa_ctx_destroy(ctx)


# ---- objective table ---------------------------------------------------------------

def make_qubo(H, f=None, c0: float = 0.0, dtype: str = "f64"):
    """Build a qaoa_qubo struct (Sec. 2.1 input form) plus the arrays it points
    to (keep the returned tuple alive for the duration of the call)."""
    code, npt = _DTYPES[dtype]
    Hc = np.ascontiguousarray(np.asarray(H).astype(npt))
    n = Hc.shape[0]
    fc = None if f is None else np.ascontiguousarray(np.asarray(f).astype(npt))
    q = qaoa_qubo(n, code, Hc.ctypes.data, 0 if fc is None else fc.ctypes.data, float(c0))
    return q, (Hc, fc)


def qaoa_build_cost(ctx, H, f=None, c0: float = 0.0, dtype: str = "f64"):
    q, keep = make_qubo(H, f, c0, dtype)
    out = _P()
    _check(_lib.qaoa_build_cost(ctx, ctypes.byref(q), ctypes.byref(out)))
    del keep
    return out


def qaoa_cost_destroy(cost) -> None:
    _lib.qaoa_cost_destroy(cost)


def qaoa_cost_info(cost) -> dict:
    n, s = ctypes.c_int32(), ctypes.c_int32()
    kc = ctypes.c_int64()
    am = ctypes.c_uint64()
    mc = ctypes.c_double()
    _check(_lib.qaoa_cost_info(cost, ctypes.byref(n), ctypes.byref(s), ctypes.byref(kc), ctypes.byref(am),
                               ctypes.byref(mc)))
    return {"n": n.value, "shift_bits": s.value, "k_c": kc.value, "argmin": am.value, "min_cost": mc.value}


def qaoa_cost_copy_to_host(ctx, cost, n: int) -> np.ndarray:
    out = np.empty(1 << n, dtype=np.int32)
    _check(_lib.qaoa_cost_copy_to_host(ctx, cost, out.ctypes.data))
    return out


def qaoa_cost_device_ptr(cost):
    """Device address of the cost handle's int32 table and its entry count."""
    p = _P()
    cnt = ctypes.c_int64()
    _check(_lib.qaoa_cost_device_ptr(cost, ctypes.byref(p), ctypes.byref(cnt)))
    return p.value, cnt.value


# ---- forward --------------------------------------------------------------------------

def qaoa_forward(ctx, cost, gamma, beta, state=None):
    g, b = _f64(gamma), _f64(beta)
    assert g.shape == b.shape
    st = _P(state.value if isinstance(state, _P) else (state or 0))
    _check(_lib.qaoa_forward(ctx, cost, g.shape[0], _dptr(g), _dptr(b), ctypes.byref(st)))
    return st


def qaoa_state_destroy(state) -> None:
    _lib.qaoa_state_destroy(state)


def qaoa_state_copy_to_host(ctx, state, n: int, fp64: bool = False) -> np.ndarray:
    out = np.empty(1 << n, dtype=np.complex128 if fp64 else np.complex64)
    _check(_lib.qaoa_state_copy_to_host(ctx, state, out.ctypes.data))
    return out


def qaoa_state_device_ptr(state):
    p = _P()
    cnt = ctypes.c_int64()
    _check(_lib.qaoa_state_device_ptr(state, ctypes.byref(p), ctypes.byref(cnt)))
    return p.value, cnt.value


def qaoa_state_gather(ctx, state, idx, fp64: bool = False) -> np.ndarray:
    """Amplitudes at the given basis indices (complex64, or complex128)."""
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64).reshape(-1))
    out = np.zeros(ix.size, dtype=np.complex128 if fp64 else np.complex64)
    _check(_lib.qaoa_state_gather(ctx, state, ix.ctypes.data_as(_PU64), int(ix.size), out.ctypes.data))
    return out


def qaoa_expect(ctx, cost, state) -> float:
    e = ctypes.c_double()
    _check(_lib.qaoa_expect(ctx, cost, state, ctypes.byref(e)))
    return e.value


def qaoa_topk(ctx, cost, state, k: int):
    idx = np.zeros(k, dtype=np.uint64)
    prob = np.zeros(k, dtype=np.float32)
    cst = np.zeros(k, dtype=np.float64)
    am = ctypes.c_uint64()
    mc = ctypes.c_double()
    pam = ctypes.c_float()
    _check(_lib.qaoa_topk(ctx, cost, state, int(k), idx.ctypes.data_as(_PU64), prob.ctypes.data_as(_PF),
                          _dptr(cst), ctypes.byref(am), ctypes.byref(mc), ctypes.byref(pam)))
    return {"idx": idx, "prob": prob, "cost": cst, "argmin": am.value, "min_cost": mc.value,
            "prob_argmin": pam.value}


# ---- gradient ---------------------------------------------------------------------------

def qaoa_grad(ctx, cost, gamma, beta, k_top: int = 0):
    """(E, dE/dgamma, dE/dbeta[, top-K indices, probabilities])."""
    g, b = _f64(gamma), _f64(beta)
    p = g.shape[0]
    dg = np.zeros(p)
    db = np.zeros(p)
    e = ctypes.c_double()
    ti = np.zeros(max(k_top, 1), dtype=np.uint64)
    tp = np.zeros(max(k_top, 1), dtype=np.float32)
    _check(_lib.qaoa_grad(ctx, cost, p, _dptr(g), _dptr(b), ctypes.byref(e), _dptr(dg), _dptr(db), int(k_top),
                          ti.ctypes.data_as(_PU64), tp.ctypes.data_as(_PF)))
    if k_top:
        return e.value, dg, db, ti[:k_top], tp[:k_top]
    return e.value, dg, db


def qaoa_grad_batch(ctx, costs, gamma, beta, item_cost=None, grad: bool = True):
    """Batched evaluation: gamma, beta of shape (B, p)."""
    g = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(beta, dtype=np.float64))
    B, p = g.shape
    arr = (_P * len(costs))(*[c.value if isinstance(c, _P) else c for c in costs])
    ic = None if item_cost is None else np.ascontiguousarray(np.asarray(item_cost, dtype=np.int32))
    E = np.zeros(B)
    dg = np.zeros((B, p)) if grad else None
    db = np.zeros((B, p)) if grad else None
    _check(_lib.qaoa_grad_batch(ctx, len(costs), arr, None if ic is None else ic.ctypes.data_as(_PI32), B, p,
                                _dptr(g), _dptr(b), _dptr(E), None if dg is None else _dptr(dg),
                                None if db is None else _dptr(db)))
    return (E, dg, db) if grad else E


def qaoa_optimize_adam(ctx, costs, gamma, beta, iterations: int, item_cost=None, lr: float = 0.0,
                       beta1: float = 0.0, beta2: float = 0.0, eps: float = 0.0, use_graph: bool = True):
    """Adam on the exact gradient for B parameter sets (gamma, beta: (B, p)).
    Returns (gamma, beta, history (iterations, B), final E (B,))."""
    g = np.array(np.asarray(gamma, dtype=np.float64), order="C", copy=True)
    b = np.array(np.asarray(beta, dtype=np.float64), order="C", copy=True)
    B, p = g.shape
    arr = (_P * len(costs))(*[c.value if isinstance(c, _P) else c for c in costs])
    ic = None if item_cost is None else np.ascontiguousarray(np.asarray(item_cost, dtype=np.int32))
    opt = qaoa_adam_options()
    opt.lr, opt.beta1, opt.beta2, opt.eps = float(lr), float(beta1), float(beta2), float(eps)
    opt.iterations = int(iterations)
    opt.disable_graph = 0 if use_graph else 1
    hist = np.zeros((int(iterations), B))
    E = np.zeros(B)
    _check(_lib.qaoa_optimize_adam(ctx, len(costs), arr, None if ic is None else ic.ctypes.data_as(_PI32), B, p,
                                   _dptr(g), _dptr(b), ctypes.byref(opt), _dptr(hist), _dptr(E)))
    return g, b, hist, E


def qaoa_optimize_adam_resume(ctx, costs, gamma, beta, iterations: int, state=None, item_cost=None,
                              lr: float = 0.0, beta1: float = 0.0, beta2: float = 0.0, eps: float = 0.0,
                              use_graph: bool = True):
    """qaoa_optimize_adam from a saved state (None: a fresh run).  Returns
    (gamma, beta, history, final E, state) with state = {"m", "v", "step"}
    to pass to the next call."""
    g = np.array(np.asarray(gamma, dtype=np.float64), order="C", copy=True)
    b = np.array(np.asarray(beta, dtype=np.float64), order="C", copy=True)
    B, p = g.shape
    if state is None:
        state = {"m": np.zeros((B, 2 * p)), "v": np.zeros((B, 2 * p)), "step": 0}
    m = np.array(state["m"], dtype=np.float64, order="C", copy=True)
    v = np.array(state["v"], dtype=np.float64, order="C", copy=True)
    step = ctypes.c_int32(int(state["step"]))
    arr = (_P * len(costs))(*[c.value if isinstance(c, _P) else c for c in costs])
    ic = None if item_cost is None else np.ascontiguousarray(np.asarray(item_cost, dtype=np.int32))
    opt = qaoa_adam_options()
    opt.lr, opt.beta1, opt.beta2, opt.eps = float(lr), float(beta1), float(beta2), float(eps)
    opt.iterations = int(iterations)
    opt.disable_graph = 0 if use_graph else 1
    hist = np.zeros((int(iterations), B))
    E = np.zeros(B)
    _check(_lib.qaoa_optimize_adam_resume(ctx, len(costs), arr, None if ic is None else ic.ctypes.data_as(_PI32), B,
                                          p, _dptr(g), _dptr(b), ctypes.byref(opt), _dptr(hist), _dptr(E), _dptr(m),
                                          _dptr(v), ctypes.byref(step)))
    return g, b, hist, E, {"m": m, "v": v, "step": step.value}


def qaoa_autotune(ctx, cost, p: int = 2, with_modes: bool = False):
    """Time every fusion width; returns (best width, {width: ms}), and with
    with_modes also {"stored": ms, "uncompute": ms} of the two adjoint forms
    at that width."""
    k = ctypes.c_int32()
    ms = np.zeros(8)
    _check(_lib.qaoa_autotune(ctx, cost, int(p), ctypes.byref(k), _dptr(ms)))
    widths = {w: float(ms[w - 3]) for w in range(5, 11) if not np.isnan(ms[w - 3])}
    if with_modes:
        return k.value, widths, {"stored": float(ms[0]), "uncompute": float(ms[1])}
    return k.value, widths


# ---- measurement by shots and SPSA ----------------------------------------------------------

def qaoa_state_from_host(ctx, amps, n: int | None = None):
    """A device state holding `amps` (complex64, or complex128 for n <= 12)."""
    a = np.ascontiguousarray(amps)
    if a.dtype not in (np.complex64, np.complex128):
        raise TypeError("amps must be complex64 or complex128")
    nn = int(a.size).bit_length() - 1 if n is None else int(n)
    out = _P()
    _check(_lib.qaoa_state_from_host(ctx, nn, 1 if a.dtype == np.complex128 else 0, a.ctypes.data, ctypes.byref(out)))
    return out


def qaoa_sample(ctx, cost, state, shots: int, seed: int = 0, stream: int = 0, rand=None,
                want_idx: bool = True, want_cost: bool = False, want_mean: bool = False):
    """Measure `state` with `shots` shots.  Returns (idx uint64[shots] or None,
    cost float64[shots] or None, mean cost or None)."""
    S = int(shots)
    r = None if rand is None else np.ascontiguousarray(np.asarray(rand, dtype=np.uint64))
    if r is not None and r.size != S:
        raise ValueError("rand must hold one integer per shot")
    idx = np.zeros(S, dtype=np.uint64) if want_idx else None
    cst = np.zeros(S) if want_cost else None
    mean = ctypes.c_double()
    _check(_lib.qaoa_sample(ctx, cost, state, S, int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream) & 0xFFFFFFFFFFFFFFFF,
                            None if r is None else r.ctypes.data_as(_PU64),
                            None if idx is None else idx.ctypes.data_as(_PU64),
                            None if cst is None else _dptr(cst), ctypes.byref(mean) if want_mean else None))
    return idx, cst, (mean.value if want_mean else None)


def qaoa_sample_stats(idx, cost, margin: float = 0.0, elite: int = 10, ref_cost=None, ref_index=None,
                      tol: float = 1e-9) -> dict:
    """Sec. 3.6 metrics of measured indices and their costs (host)."""
    x = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    c = _f64(cost)
    m = qaoa_sample_metrics()
    ei = np.zeros(max(int(elite), 1), dtype=np.uint64)
    ec = np.zeros(max(int(elite), 1))
    en = np.zeros(max(int(elite), 1), dtype=np.int64)
    has = ref_cost is not None
    _check(_lib.qaoa_sample_stats(x.size, x.ctypes.data_as(_PU64), _dptr(c), float(margin), int(elite),
                                  ei.ctypes.data_as(_PU64), _dptr(ec), en.ctypes.data_as(_PI64), 1 if has else 0,
                                  float(ref_cost) if has else 0.0,
                                  int(ref_index) if ref_index is not None else 0xFFFFFFFFFFFFFFFF, float(tol),
                                  ctypes.byref(m)))
    out = {f: getattr(m, f) for f, _ in qaoa_sample_metrics._fields_}
    out["elite"] = [(int(ei[i]), float(ec[i]), int(en[i]), float(en[i]) / m.shots)
                    for i in range(int(elite)) if en[i] > 0]
    return out


def qaoa_optimize_spsa(ctx, costs, gamma, beta, iterations: int, item_cost=None, shots: int = 0,
                       averaging: int = 1, seed: int = 0, c: float = 0.1, c_decay: float = 0.101,
                       lr: float = 0.0, beta1: float = 0.0, beta2: float = 0.0, eps: float = 0.0):
    """SPSA-Adam (Sec. 3.4) for B parameter sets (gamma, beta: (B, p)).
    Returns (gamma, beta, history (iterations, B, 2) of (J+, J-), final exact E (B,))."""
    g = np.array(np.asarray(gamma, dtype=np.float64), order="C", copy=True)
    b = np.array(np.asarray(beta, dtype=np.float64), order="C", copy=True)
    B, p = g.shape
    arr = (_P * len(costs))(*[x.value if isinstance(x, _P) else x for x in costs])
    ic = None if item_cost is None else np.ascontiguousarray(np.asarray(item_cost, dtype=np.int32))
    o = qaoa_spsa_options()
    o.lr, o.beta1, o.beta2, o.eps = float(lr), float(beta1), float(beta2), float(eps)
    o.c, o.c_decay = float(c), float(c_decay)
    o.iterations, o.shots, o.averaging = int(iterations), int(shots), int(averaging)
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    hist = np.zeros((int(iterations), B, 2))
    E = np.zeros(B)
    _check(_lib.qaoa_optimize_spsa(ctx, len(costs), arr, None if ic is None else ic.ctypes.data_as(_PI32), B, p,
                                   _dptr(g), _dptr(b), ctypes.byref(o), _dptr(hist), _dptr(E)))
    return g, b, hist, E


def _metrics_dict(m) -> dict:
    return {f: getattr(m, f) for f, _ in qaoa_sample_metrics._fields_}


def qaoa_solve(ctx, cost, p_max: int, optimizer: str = "spsa", iterations: int = 50, shots: int = 0,
               averaging: int = 1, random_starts: int = 2, warm_perturb: int = 1, include_warm: bool = True,
               final_shots: int = 4096, use_reference: bool = True, lr: float = 0.0, beta1: float = 0.0,
               beta2: float = 0.0, eps: float = 0.0, c: float = 0.1, c_decay: float = 0.101,
               warm_sigma: float = 0.05, gamma_range: float = 0.5, beta_range: float = 1.5707963267948966,
               margin: float = 0.0, tol: float = 1e-9, seed: int = 0, elite: int = 10) -> dict:
    """Algorithm 1 (Sec. 3.5): depth progression with warm starts and random
    restarts.  Returns a dict with the selected depth, angles, metrics, elite
    set and each depth's representative metrics."""
    o = qaoa_solve_options()
    o.p_max, o.optimizer, o.iterations = int(p_max), {"spsa": 0, "adam": 1}[optimizer], int(iterations)
    o.shots, o.averaging, o.random_starts = int(shots), int(averaging), int(random_starts)
    o.warm_perturb, o.include_warm, o.final_shots = int(warm_perturb), int(bool(include_warm)), int(final_shots)
    o.use_reference = int(bool(use_reference))
    o.lr, o.beta1, o.beta2, o.eps, o.c, o.c_decay = float(lr), float(beta1), float(beta2), float(eps), float(c), \
        float(c_decay)
    o.warm_sigma, o.gamma_range, o.beta_range = float(warm_sigma), float(gamma_range), float(beta_range)
    o.margin, o.tol, o.seed = float(margin), float(tol), int(seed) & 0xFFFFFFFFFFFFFFFF
    g = np.zeros(int(p_max))
    b = np.zeros(int(p_max))
    ne = max(int(elite), 1)
    ei, ec, en = np.zeros(ne, dtype=np.uint64), np.zeros(ne), np.zeros(ne, dtype=np.int64)
    dm = (qaoa_sample_metrics * int(p_max))()
    r = qaoa_solve_result()
    _check(_lib.qaoa_solve(ctx, cost, ctypes.byref(o), _dptr(g), _dptr(b), int(elite), ei.ctypes.data_as(_PU64),
                           _dptr(ec), en.ctypes.data_as(_PI64), dm, ctypes.byref(r)))
    m = _metrics_dict(r.metrics)
    return {"best_p": r.best_p, "runs": r.runs, "expect": r.expect, "gamma": g[:r.best_p].copy(),
            "beta": b[:r.best_p].copy(), "metrics": m,
            "elite": [(int(ei[i]), float(ec[i]), int(en[i]), float(en[i]) / m["shots"])
                      for i in range(int(elite)) if en[i] > 0],
            "depth_metrics": [_metrics_dict(dm[i]) for i in range(int(p_max))]}


# ---- DQAOA ----------------------------------------------------------------------------------

def qaoa_plan_describe(n: int, p: int, grad: bool = True, max_fused_qubits: int = 10, stored_mids: int = 0):
    """The pass schedule of one evaluation (host only; no device is touched):
    a list of dicts, one per pass in execution order, and the numbers of
    stored states and of mixer-only passes."""
    cnt, ns, nm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.qaoa_plan_describe(int(n), int(p), int(bool(grad)), int(max_fused_qubits), int(stored_mids), None,
                                   0, ctypes.byref(cnt), None, None))
    arr = (qaoa_pass_info * max(cnt.value, 1))()
    _check(_lib.qaoa_plan_describe(int(n), int(p), int(bool(grad)), int(max_fused_qubits), int(stored_mids), arr,
                                   cnt.value, ctypes.byref(cnt), ctypes.byref(ns), ctypes.byref(nm)))
    passes = []
    for i in range(cnt.value):
        e = arr[i]
        d = {f: getattr(e, f) for f, _ in qaoa_pass_info._fields_ if f != "slot_param"}
        d["slot_param"] = list(e.slot_param)
        passes.append(d)
    return passes, ns.value, nm.value


def qaoa_partition(n: int, M: int, caps=None, manual=None) -> np.ndarray:
    out = np.zeros(n, dtype=np.int32)
    c = None if caps is None else np.ascontiguousarray(np.asarray(caps, dtype=np.int32))
    m = None if manual is None else np.ascontiguousarray(np.asarray(manual, dtype=np.int32))
    _check(_lib.qaoa_partition(int(n), int(M), None if c is None else c.ctypes.data_as(_PI32),
                               None if m is None else m.ctypes.data_as(_PI32), out.ctypes.data_as(_PI32)))
    return out


def qaoa_partition_graph(H, f, c0: float, caps, dtype: str = "f64") -> np.ndarray:
    """Graph-aware allocation of the QUBO (H, f, c0) for the capacities caps."""
    qb, keep = make_qubo(H, f, c0, dtype)
    n = qb.n
    c = np.ascontiguousarray(np.asarray(caps, dtype=np.int32))
    out = np.zeros(n, dtype=np.int32)
    _check(_lib.qaoa_partition_graph(ctypes.byref(qb), len(c), c.ctypes.data_as(_PI32), out.ctypes.data_as(_PI32)))
    return out


def qaoa_allocation_candidates(H, f, c0: float, caps, manual=None, p: int = 1, dtype: str = "f64") -> dict:
    """Contiguous, graph-aware and manual candidates scored by cross-QPU
    couplings; returns the selected allocation and every candidate's counts."""
    qb, keep = make_qubo(H, f, c0, dtype)
    n = qb.n
    c = np.ascontiguousarray(np.asarray(caps, dtype=np.int32))
    m = None if manual is None else np.ascontiguousarray(np.asarray(manual, dtype=np.int32))
    out = np.zeros(n, dtype=np.int32)
    kind = ctypes.c_int32()
    cross = np.zeros(3, dtype=np.int64)
    rcx = np.zeros(3, dtype=np.int64)
    _check(_lib.qaoa_allocation_candidates(ctypes.byref(qb), len(c), c.ctypes.data_as(_PI32),
                                           None if m is None else m.ctypes.data_as(_PI32), int(p),
                                           out.ctypes.data_as(_PI32), ctypes.byref(kind),
                                           cross.ctypes.data_as(_PI64), rcx.ctypes.data_as(_PI64)))
    k = 3 if manual is not None else 2
    return {"qpu_of": out, "kind": kind.value, "cross": [int(v) for v in cross[:k]],
            "remote_cx": [int(v) for v in rcx[:k]]}


def qaoa_telegate_simulate(ctx, cost, qpu_of, gamma, beta, trajectories: int = 1, seed: int = 0,
                           want_amps: bool = False):
    """Gate-level TeleGate simulation (Sec. 3.3).  Returns (fidelity per
    trajectory, data states (trajectories, 2^n) complex64 or None, counts)."""
    q = np.ascontiguousarray(np.asarray(qpu_of, dtype=np.int32))
    g, b = _f64(gamma), _f64(beta)
    T = int(trajectories)
    fid = np.zeros(T)
    n = q.size
    amps = np.zeros((T, 1 << n), dtype=np.complex64) if want_amps else None
    cnt = qaoa_telegate_counts()
    _check(_lib.qaoa_telegate_simulate(ctx, cost, q.ctypes.data_as(_PI32), len(g), _dptr(g), _dptr(b), T,
                                       int(seed) & 0xFFFFFFFFFFFFFFFF, _dptr(fid),
                                       None if amps is None else amps.ctypes.data_as(_PF), ctypes.byref(cnt)))
    return fid, amps, {f: getattr(cnt, f) for f, _ in qaoa_telegate_counts._fields_}


def qaoa_classify(cost, qpu_of, p: int):
    q = np.ascontiguousarray(np.asarray(qpu_of, dtype=np.int32))
    a, b, c, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.qaoa_classify(cost, q.ctypes.data_as(_PI32), int(p), ctypes.byref(a), ctypes.byref(b),
                              ctypes.byref(c), ctypes.byref(d)))
    return {"local": a.value, "cross": b.value, "remote_cx": c.value, "cross_all_pairs": d.value}


def qaoa_check_factorisation(ctx, cost, qpu_of, gamma_probe: float = 0.7):
    q = np.ascontiguousarray(np.asarray(qpu_of, dtype=np.int32))
    mm = ctypes.c_int64()
    pe = ctypes.c_double()
    _check(_lib.qaoa_check_factorisation(ctx, cost, q.ctypes.data_as(_PI32), float(gamma_probe), ctypes.byref(mm),
                                         ctypes.byref(pe)))
    return mm.value, pe.value


def qaoa_expect_noalloc(amps_ptr: int, table_ptr: int, n: int, shift_bits: int, k_c: int,
                        stream: int | None = None) -> float:
    """<H_C> from raw device pointers, without any device allocation (the
    library keeps this call's scratch in a fixed device array; n <= 30)."""
    e = ctypes.c_double()
    _check(_lib.qaoa_expect_noalloc(_P(amps_ptr), _P(table_ptr), int(n), int(shift_bits), int(k_c),
                                    _P(stream or 0), ctypes.byref(e)))
    return e.value


def qaoa_profile_read(ctx, kind: int, reset: bool = False):
    n = ctypes.c_int64()
    ms, by = ctypes.c_double(), ctypes.c_double()
    _check(_lib.qaoa_profile_read(ctx, int(kind), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by), int(reset)))
    return {"launches": n.value, "ms": ms.value, "bytes": by.value}


def qaoa_peak_probe(ctx, kind: int):
    """Sustained (ops/s, flop/s) of one arithmetic pipe: 0 FP32 FMA, 1 f32x2
    FMA, 2 FP64 FMA, 3 sin/cos pairs."""
    o, f = ctypes.c_double(), ctypes.c_double()
    _check(_lib.qaoa_peak_probe(ctx, int(kind), ctypes.byref(o), ctypes.byref(f)))
    return o.value, f.value


def qaoa_wait_probe(ctx) -> None:
    """Make one bounded device wait expire; raises QaoaError with status
    QAOA_ERR_TIMEOUT, which is the expected outcome."""
    _check(_lib.qaoa_wait_probe(ctx))


PROFILE_KINDS = {"fwd_pass": 0, "rev_pass": 1, "cost_build": 2, "small_resident": 3, "factorisation": 4,
                 "sample_weights": 6, "sample_shots": 7}
# one kernel each (a layer pass is counted in its aggregate kind above and here)
PROFILE_KERNEL_KINDS = {"fwd_pass_kernel": 8, "fwd_cost_tma_kernel": 9, "final_pass_kernel": 10,
                        "rev_pass_kernel": 11, "rev_mid_tma_kernel": 12, "final_pass_half_kernel": 13,
                        "rev_pass_half_kernel": 14}
PROFILE_ALL_LAUNCHES = 5


def bitstring(x: int, n: int) -> str:
    """Logical QUBO bitstring z_1..z_n of basis index x (Sec. 3.6): bit i of x
    is z_{i+1}, printed first to last."""
    return "".join("1" if (int(x) >> i) & 1 else "0" for i in range(n))
