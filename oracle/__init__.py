"""FP64 CPU oracle for the QAOA statevector hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its Python binding) never imports it, and this
package never imports the product; the two share only the seeded instance
generator (``paper_2606_26297_b300.instances``), which holds no QAOA
arithmetic.

The heavy loops (objective table, state evolution, adjoint gradient) are plain
C in ``qaoa_oracle.c``, compiled here with gcc and loaded with ctypes; the rest
is numpy or plain Python.  Each function names the passage of the paper it
follows.

Pins: every function is checked by ``tests/test_oracle_pins.py`` against an
independent fact (a closed form, brute force, a special case, or a published
analytic result); see the docstrings there.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from itertools import combinations

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qaoa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_U64 = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_canonicalize.argtypes = [ctypes.c_int, _D, _D, _D, _D]
        lib.oracle_cost_one.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D, ctypes.c_uint64]
        lib.oracle_cost_one.restype = ctypes.c_double
        lib.oracle_cost_table.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D, _D]
        lib.oracle_cost_sampled.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D, _U64,
                                            ctypes.c_int64, _D]
        lib.oracle_evolve.argtypes = [ctypes.c_int, _D, ctypes.c_int, _D, _D, _D]
        lib.oracle_expectation.argtypes = [ctypes.c_int, _D, _D]
        lib.oracle_expectation.restype = ctypes.c_double
        lib.oracle_grad_adjoint.argtypes = [ctypes.c_int, _D, ctypes.c_int, _D, _D, _D, _D]
        lib.oracle_grad_adjoint.restype = ctypes.c_double
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


# ---- Sec. 2.1 ---------------------------------------------------------------

class Canonical:
    """Canonical QUBO (Eq. qubo_canonical_work): c0, l (n), b (n x n, i<j)."""

    def __init__(self, n: int, c0: float, ell: np.ndarray, b: np.ndarray):
        self.n, self.c0, self.ell, self.b = n, float(c0), ell, b


def canonicalize(H: np.ndarray, f: np.ndarray | None, c0: float) -> Canonical:
    """l_i = f_i + H_ii and b_ij = H_ij + H_ji, i<j (Eqs. canonical_linear,
    canonical_quadratic)."""
    lib = _load()
    H = np.ascontiguousarray(H, dtype=np.float64)
    n = H.shape[0]
    fv = np.ascontiguousarray(f if f is not None else np.zeros(n), dtype=np.float64)
    ell = np.zeros(n)
    b = np.zeros((n, n))
    lib.oracle_canonicalize(n, _dp(H), _dp(fv), _dp(ell), _dp(b))
    return Canonical(n, c0, ell, b)


def canonical_of(q) -> Canonical:
    """Canonical form of an instance from paper_2606_26297_b300.instances."""
    return canonicalize(q.H, q.f, q.c0)


def cost_table(cq: Canonical) -> np.ndarray:
    """F(x) for all 2^n basis indices (Eq. qubo_canonical_work; the eigenvalues
    of H_C, Eq. cost_hamiltonian_raw)."""
    lib = _load()
    F = np.empty(1 << cq.n)
    lib.oracle_cost_table(cq.n, cq.c0, _dp(cq.ell), _dp(cq.b), _dp(F))
    return F


def cost_at(cq: Canonical, xs) -> np.ndarray:
    """F at sampled indices xs (uint64)."""
    lib = _load()
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    out = np.empty(xs.shape[0])
    lib.oracle_cost_sampled(cq.n, cq.c0, _dp(cq.ell), _dp(cq.b),
                            xs.ctypes.data_as(_U64), xs.shape[0], _dp(out))
    return out


# ---- Sec. 2.3 ---------------------------------------------------------------

def evolve(F: np.ndarray, gamma, beta) -> np.ndarray:
    """The depth-p state of Eq. qaoa_state as a complex128 array of 2^n."""
    lib = _load()
    F = np.ascontiguousarray(F, dtype=np.float64)
    n = int(round(math.log2(F.shape[0])))
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    assert g.shape == b.shape
    psi = np.empty(2 << n)
    lib.oracle_evolve(n, _dp(F), g.shape[0], _dp(g), _dp(b), _dp(psi))
    return psi.view(np.complex128)


def expectation(F: np.ndarray, psi: np.ndarray) -> float:
    """sum_z P(z) F(z) (Eq. qaoa_expectation_expanded)."""
    lib = _load()
    n = int(round(math.log2(F.shape[0])))
    pv = np.ascontiguousarray(psi, dtype=np.complex128).view(np.float64)
    return float(lib.oracle_expectation(n, _dp(np.ascontiguousarray(F)), _dp(pv)))


def probabilities(psi: np.ndarray) -> np.ndarray:
    """P(z) = |<z|gamma,beta>|^2."""
    return psi.real ** 2 + psi.imag ** 2


def topk(P: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k most probable bitstrings, ordered by probability
    descending and, among equal probabilities, by index ascending (the elite
    set of Sec. 3.6, ranked by exact probability)."""
    order = np.lexsort((np.arange(P.shape[0]), -P))
    return order[:k]


def argmin(F: np.ndarray) -> int:
    """Brute-force minimiser of F, smallest index among ties (the brute-force
    mode of Sec. 3.7)."""
    return int(np.argmin(F))  # numpy returns the first occurrence


def grad_adjoint(F: np.ndarray, gamma, beta):
    """(E, dE/dgamma, dE/dbeta) by the textbook adjoint sweep in FP64."""
    lib = _load()
    F = np.ascontiguousarray(F, dtype=np.float64)
    n = int(round(math.log2(F.shape[0])))
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    dg = np.zeros_like(g)
    db = np.zeros_like(b)
    E = lib.oracle_grad_adjoint(n, _dp(F), g.shape[0], _dp(g), _dp(b), _dp(dg), _dp(db))
    return float(E), dg, db


def grad_fd(F: np.ndarray, gamma, beta, h: float = 1e-5):
    """Central finite differences of E in FP64, one parameter at a time (the
    coordinate-wise scheme that Sec. 4.2 replaces with SPSA)."""
    g = np.array(gamma, dtype=np.float64)
    b = np.array(beta, dtype=np.float64)

    def E(gg, bb):
        return expectation(F, evolve(F, gg, bb))

    dg = np.zeros_like(g)
    db = np.zeros_like(b)
    for l in range(g.shape[0]):
        gp, gm = g.copy(), g.copy()
        gp[l] += h
        gm[l] -= h
        dg[l] = (E(gp, b) - E(gm, b)) / (2 * h)
        bp, bm = b.copy(), b.copy()
        bp[l] += h
        bm[l] -= h
        db[l] = (E(g, bp) - E(g, bm)) / (2 * h)
    return dg, db


def interleave(gamma, beta) -> np.ndarray:
    """x = [gamma_1, beta_1, ..., gamma_p, beta_p] (Sec. 3.4)."""
    return np.stack([np.asarray(gamma), np.asarray(beta)], axis=1).reshape(-1)


# ---- Sec. 3.1-3.2: allocation and coupling classification -----------------

def balanced_capacities(n: int, M: int) -> list[int]:
    """Capacities as even as possible (make_balanced_capacities, Sec. 3.1):
    c_m = floor(n/M) + [m < n mod M]."""
    return [n // M + (1 if m < n % M else 0) for m in range(M)]


def contiguous_allocation(n: int, caps: list[int]) -> list[int]:
    """Fill QPU 1 with the first c_1 variables, then QPU 2, ... (the default
    contiguous allocation of Sec. 3.1)."""
    q = []
    for m, c in enumerate(caps):
        q.extend([m] * c)
    return q[:n]


def validate_allocation(qpu_of: list[int], caps: list[int]) -> bool:
    """Every variable on exactly one QPU, no capacity exceeded, every QPU used
    (validate_allocation, Sec. 3.1)."""
    M = len(caps)
    if any(q < 0 or q >= M for q in qpu_of):
        return False
    counts = [qpu_of.count(m) for m in range(M)]
    return all(counts[m] <= caps[m] for m in range(M)) and all(c > 0 for c in counts)


def classify(cq: Canonical, qpu_of: list[int], p: int):
    """Local vs cross-QPU couplings (Eq. local_cross_rule) over the pairs with
    b_ij != 0, and the remote-CX estimate 2 * cross * p (Sec. 3.1)."""
    n_local = n_cross = 0
    for i, j in combinations(range(cq.n), 2):
        if cq.b[i, j] == 0.0:
            continue
        if qpu_of[i] == qpu_of[j]:
            n_local += 1
        else:
            n_cross += 1
    return n_local, n_cross, 2 * n_cross * p
