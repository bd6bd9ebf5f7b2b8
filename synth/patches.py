"""Fixed dictionaries for the overlapping-patch prior (inputs; no method
arithmetic).  The paper's learned basis is not published; an over-complete
separable DCT stands in for it."""
from __future__ import annotations

import numpy as np


def overcomplete_dct(m: int, k: int) -> np.ndarray:
    """k^2 atoms of m x m pixels ([k*k, m*m], float64): outer products of k
    one-dimensional atoms cos(pi (2n + 1) u / (2k)), n < m, u < k (k >= m:
    over-complete), each with its mean removed for u > 0 and unit norm."""
    n = np.arange(m)
    one = []
    for u in range(k):
        a = np.cos(np.pi * (2 * n + 1) * u / (2 * k))
        if u > 0:
            a = a - a.mean()
        one.append(a / np.linalg.norm(a))
    return np.stack([np.outer(a, b).ravel() for a in one for b in one])
