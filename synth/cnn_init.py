"""Seeded initial parameters of the residual CNN prox (an input of training,
shared by the oracle tests and the GPU trainer; no network arithmetic)."""
from __future__ import annotations

import numpy as np

CHANNELS = (1, 32, 32, 32, 32, 32, 32, 32, 1)


def init_params(seed: int, channels=CHANNELS) -> np.ndarray:
    """Flat float32 vector in the layer order W_1, b_1, ..., W_8, b_8 with
    W_l [C_l][C_{l-1}][3][3]: He-normal weights (std sqrt(2 / (9 C_{l-1}))),
    zero biases, the last layer's weights scaled by 0.1 so that the untrained
    network stays close to z -> z."""
    g = np.random.default_rng(seed)
    parts = []
    n = len(channels) - 1
    for l in range(1, n + 1):
        cin, cout = channels[l - 1], channels[l]
        std = np.sqrt(2.0 / (9 * cin)) * (0.1 if l == n else 1.0)
        parts.append(g.standard_normal(cout * cin * 9) * std)
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)
