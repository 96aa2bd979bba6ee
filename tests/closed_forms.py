"""Closed forms used as pins at sizes the oracle cannot reach.

qaoa_p1_maxcut: the expected cut of depth-1 QAOA on any graph, from the
analysis of Wang, Hadfield, Jiang and Rieffel (Phys. Rev. A 97, 022304, 2018,
the p = 1 formula for an edge (u, v) with degrees d_u, d_v and f triangles
through the edge). Their ansatz is exp(-i beta B) exp(-i gamma' C) with
C = sum_edges (1 - Z_u Z_v) / 2; the cost layer here is
prod_edges exp(-i gamma Z_u Z_v) = exp(-i gamma |E|) exp(2 i gamma C), so
gamma' = -2 gamma (the global phase drops out of <C>).
"""
import numpy as np


def qaoa_p1_maxcut(n, edges, gamma, beta):
    nb = [set() for _ in range(n)]
    for u, v in edges:
        nb[u].add(v)
        nb[v].add(u)
    g = -2.0 * gamma
    c, s = np.cos(g), np.sin(g)
    total = 0.0
    for u, v in edges:
        f = len(nb[u] & nb[v])
        du, dv = len(nb[u]) - 1, len(nb[v]) - 1
        total += (0.5 + 0.25 * np.sin(4 * beta) * s * (c ** du + c ** dv)
                  - 0.25 * np.sin(2 * beta) ** 2 * c ** (du + dv - 2 * f) * (1 - np.cos(2 * g) ** f))
    return total
