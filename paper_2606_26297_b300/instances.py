"""Seeded synthetic QUBO instances and angle schedules.

This module holds only input generation (random numbers and problem
construction); none of the QAOA arithmetic lives here.  Both the CUDA path
(bench, tests) and the FP64 oracle consume the instances it produces, so the
two sides always see bit-identical inputs.

Every instance is given in the paper's input form (Sec. 2.1, Eq.
qubo_input_form): F(z) = c0 + f^T z + z^T H z with H a dense n x n matrix
(row-major), f a length-n vector and c0 a scalar.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), implemented here from its
published definition on Python integers.  Integers are drawn uniformly by
rejection, reals uniformly from the top 53 bits, normals by the Box-Muller
transform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream: state advances by the golden-ratio increment and each
    output is the state passed through the published 64-bit finaliser."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] by rejection (no modulo bias)."""
        r = hi - lo + 1
        limit = (1 << 64) - ((1 << 64) % r)
        while True:
            u = self.next_u64()
            if u < limit:
                return lo + (u % r)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def normal_pair(self) -> tuple[float, float]:
        """Two independent N(0,1) draws by Box-Muller."""
        u1 = self.uniform()
        u2 = self.uniform()
        rad = math.sqrt(-2.0 * math.log(1.0 - u1))
        return rad * math.cos(2.0 * math.pi * u2), rad * math.sin(2.0 * math.pi * u2)

    def normals(self, count: int) -> list[float]:
        out: list[float] = []
        while len(out) < count:
            a, b = self.normal_pair()
            out.append(a)
            out.append(b)
        return out[:count]


@dataclass
class Qubo:
    """A QUBO in the paper's input form (Sec. 2.1).

    ``dtype`` names the coefficient type handed to the C-ABI: "i32" for
    integer instances (results are bit-exact), "f32" for real instances given
    in single precision.  ``H`` and ``f`` hold the exact values in float64
    (for "f32" they are float32-representable)."""

    n: int
    H: np.ndarray
    f: np.ndarray
    c0: float
    dtype: str
    name: str = ""
    meta: dict = field(default_factory=dict)


def upper_int_qubo(n: int, seed: int, lo: int = -10, hi: int = 10) -> Qubo:
    """Dense integer QUBO: upper-triangular Q (diagonal included) with entries
    uniform in [lo, hi]; f = 0, c0 = 0."""
    rng = SplitMix64(seed)
    H = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        for j in range(i, n):
            H[i, j] = rng.randint(lo, hi)
    return Qubo(n, H, np.zeros(n), 0.0, "i32", f"int-upper-n{n}-s{seed}")


def normal_qubo(n: int, seed: int) -> Qubo:
    """Dense real QUBO: couplings Q_ij (i<j) and linear terms h_i drawn N(0,1)
    and rounded to float32; H strictly upper, f = h, c0 = 0."""
    rng = SplitMix64(seed)
    m = n * (n - 1) // 2
    vals = np.array(rng.normals(m + n), dtype=np.float64).astype(np.float32).astype(np.float64)
    H = np.zeros((n, n), dtype=np.float64)
    k = 0
    for i in range(n):
        for j in range(i + 1, n):
            H[i, j] = vals[k]
            k += 1
    f = vals[m:m + n].copy()
    return Qubo(n, H, f, 0.0, "f32", f"normal-n{n}-s{seed}")


def random_regular_graph(n: int, d: int, seed: int, max_tries: int = 100000) -> list[tuple[int, int]]:
    """Random d-regular simple graph by the pairing (configuration) model:
    n*d half-edges are matched by a Fisher-Yates shuffle; matchings with a loop
    or a repeated edge are rejected and redrawn."""
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    rng = SplitMix64(seed)
    for _ in range(max_tries):
        pts = [v for v in range(n) for _ in range(d)]
        for i in range(len(pts) - 1, 0, -1):
            j = rng.randint(0, i)
            pts[i], pts[j] = pts[j], pts[i]
        edges = set()
        ok = True
        for k in range(0, len(pts), 2):
            u, v = pts[k], pts[k + 1]
            if u == v:
                ok = False
                break
            e = (min(u, v), max(u, v))
            if e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)
    raise RuntimeError("no simple regular graph found")


def maxcut_qubo(n: int, edges: list[tuple[int, int]], name: str = "") -> Qubo:
    """MaxCut as a minimisation QUBO with unit weights: H_ij = +2 on each edge
    (i<j), f_i = -deg(i), c0 = 0, so that F(z) = -cut(z)."""
    H = np.zeros((n, n), dtype=np.float64)
    f = np.zeros(n, dtype=np.float64)
    for (u, v) in edges:
        H[min(u, v), max(u, v)] = 2.0
        f[u] -= 1.0
        f[v] -= 1.0
    return Qubo(n, H, f, 0.0, "i32", name or f"maxcut-n{n}", {"edges": edges})


def regular_maxcut_qubo(n: int, seed: int, d: int = 3) -> Qubo:
    edges = random_regular_graph(n, d, seed)
    return maxcut_qubo(n, edges, f"maxcut{d}reg-n{n}-s{seed}")


def unit_commitment_qubo(n: int, seed: int, lam: float = 10.0) -> Qubo:
    """Unit-commitment-shaped QUBO: unit costs c_i ~ U[50, 500], outputs
    P_i ~ U[10, 100], demand D = 0.5 * sum(P), and the penalty
    lam * (sum_i P_i z_i - D)^2.  Expanded with z_i^2 = z_i:
      linear  f_i  = c_i + lam * (P_i^2 - 2 D P_i)
      coupling H_ij = 2 lam P_i P_j  (i<j, upper)
      constant c0  = lam * D^2.
    Coefficients are rounded to float32."""
    rng = SplitMix64(seed)
    cost = np.array([50.0 + 450.0 * rng.uniform() for _ in range(n)])
    P = np.array([10.0 + 90.0 * rng.uniform() for _ in range(n)])
    D = 0.5 * float(P.sum())
    f = cost + lam * (P * P - 2.0 * D * P)
    H = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        for j in range(i + 1, n):
            H[i, j] = 2.0 * lam * P[i] * P[j]
    f = f.astype(np.float32).astype(np.float64)
    H = H.astype(np.float32).astype(np.float64)
    c0 = float(np.float32(lam * D * D))
    return Qubo(n, H, f, c0, "f32", f"uc-n{n}-s{seed}", {"cost": cost, "P": P, "D": D})


def block_diagonal_qubo(blocks: list[Qubo]) -> Qubo:
    """Direct sum of QUBOs on disjoint variable ranges (zero couplings between
    blocks); the constants add."""
    n = sum(b.n for b in blocks)
    H = np.zeros((n, n))
    f = np.zeros(n)
    off = 0
    for b in blocks:
        H[off:off + b.n, off:off + b.n] = b.H
        f[off:off + b.n] = b.f
        off += b.n
    dtype = "i32" if all(b.dtype == "i32" for b in blocks) else "f32"
    return Qubo(n, H, f, float(sum(b.c0 for b in blocks)), dtype, "blockdiag")


def ramp_angles(p: int, gamma_scale: float = 1.0, amp: float = 0.8) -> tuple[np.ndarray, np.ndarray]:
    """Linear-ramp schedule: gamma_l = amp*(l-1/2)/p * gamma_scale and
    beta_l = amp*(1-(l-1/2)/p), l = 1..p."""
    t = (np.arange(1, p + 1) - 0.5) / p
    return amp * t * gamma_scale, amp * (1.0 - t)


def random_angles(p: int, batch: int, seed: int, gamma_scale: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Multi-start points: gamma ~ U[0, pi)*gamma_scale, beta ~ U[0, pi/2);
    arrays of shape (batch, p)."""
    rng = SplitMix64(seed)
    g = np.array([[math.pi * rng.uniform() * gamma_scale for _ in range(p)] for _ in range(batch)])
    b = np.array([[0.5 * math.pi * rng.uniform() for _ in range(p)] for _ in range(batch)])
    return g, b


def coefficient_norm(q: Qubo) -> float:
    """Plain size statistic of the input coefficients, sqrt(sum H^2 + sum f^2);
    used only to pick angle scales for real-valued instances."""
    return float(math.sqrt(float((q.H * q.H).sum() + (q.f * q.f).sum())))


# ---- the named workloads -------------------------------------------------

def workload_small_int() -> tuple[Qubo, np.ndarray, np.ndarray]:
    """Dense integer QUBO, n=12, p=2, gamma=(0.4,0.8), beta=(0.7,0.3)."""
    return upper_int_qubo(12, 1001), np.array([0.4, 0.8]), np.array([0.7, 0.3])


def workload_maxcut26() -> tuple[Qubo, np.ndarray, np.ndarray]:
    """MaxCut on a random 3-regular graph, n=26, p=4, ramp angles."""
    g, b = ramp_angles(4)
    return regular_maxcut_qubo(26, 1002), g, b


def workload_dense30(n: int = 30, p: int = 8) -> tuple[Qubo, np.ndarray, np.ndarray]:
    """Dense N(0,1) float32 QUBO, n=30, p=8, ramp angles scaled by
    sqrt(n)/coefficient_norm."""
    q = normal_qubo(n, 1003)
    g, b = ramp_angles(p, gamma_scale=math.sqrt(n) / coefficient_norm(q))
    return q, g, b


def workload_batch20(batch: int = 256, p: int = 4) -> tuple[Qubo, np.ndarray, np.ndarray]:
    """One n=20 integer QUBO and `batch` random multi-start angle sets, p=4."""
    q = upper_int_qubo(20, 1004)
    g, b = random_angles(p, batch, 2004, gamma_scale=1.0 / math.sqrt(q.n))
    return q, g, b


def workload_ragged(count: int = 64, nmin: int = 10, nmax: int = 22, p: int = 4):
    """`count` integer QUBOs with n uniform in [nmin, nmax]; one angle set each."""
    rng = SplitMix64(3004)
    qs = [upper_int_qubo(rng.randint(nmin, nmax), 1004 + 1 + i) for i in range(count)]
    g, b = random_angles(p, count, 4004, gamma_scale=0.25)
    return qs, g, b


def workload_uc32(n: int = 32, p: int = 6) -> tuple[Qubo, np.ndarray, np.ndarray]:
    """Unit-commitment-shaped float32 QUBO, n=32, p=6, ramp angles scaled by
    sqrt(n)/coefficient_norm."""
    q = unit_commitment_qubo(n, 1005)
    g, b = ramp_angles(p, gamma_scale=math.sqrt(n) / coefficient_norm(q))
    return q, g, b


def random_state(n: int, seed: int, zero_mask=None, dtype=np.complex64) -> np.ndarray:
    """A normalised random statevector of 2^n amplitudes (independent complex
    normals), with the amplitudes where zero_mask (bool, 2^n) is true set to
    zero; for measuring states of a chosen shape."""
    rng = np.random.default_rng(seed)
    N = 1 << n
    a = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    if zero_mask is not None:
        a[np.asarray(zero_mask, dtype=bool)] = 0.0
    a /= np.linalg.norm(a)
    return a.astype(dtype)


def random_u64(count: int, seed: int) -> np.ndarray:
    """count uniform 64-bit integers (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, np.iinfo(np.uint64).max, size=count, dtype=np.uint64, endpoint=True)
