"""Closed forms from the literature used as pins by the tests (test
infrastructure; no library or oracle code)."""
import math


def maxcut_p1_closed_form(n, edges, gamma, beta):
    """Wang, Hadfield, Jiang, Rieffel, PRA 97, 022304 (2018), Thm. 1: for the
    cut operator C = sum (1 - Z_u Z_v)/2 and |g,b> = e^{-ibB}e^{-igC}|+>,
      <C_uv> = 1/2 + 1/4 sin4b sing (cos^du g + cos^dv g)
               - 1/4 sin^2 2b cos^{du+dv-2t} g (1 - cos^t 2g),
    du = deg(u)-1, dv = deg(v)-1, t = #triangles on (u,v).
    The QUBO here has F = -cut, so exp(-i g F) = exp(-i (-g) C) and
    E_F(g, b) = -E_cut(-g, b)."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    g = -gamma
    tot = 0.0
    for u, v in edges:
        du, dv = len(adj[u]) - 1, len(adj[v]) - 1
        t = len(adj[u] & adj[v])
        val = 0.5 + 0.25 * math.sin(4 * beta) * math.sin(g) * (math.cos(g) ** du + math.cos(g) ** dv)
        val -= 0.25 * math.sin(2 * beta) ** 2 * math.cos(g) ** (du + dv - 2 * t) * (1 - math.cos(2 * g) ** t)
        tot += val
    return -tot
