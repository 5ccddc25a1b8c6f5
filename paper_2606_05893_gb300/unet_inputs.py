"""Seeded inputs of the learned warm start's network: initial weights and test
volumes. Random numbers only (numpy PCG64 seeded by the caller): no network
arithmetic lives here, so the CUDA library's binding and the CPU oracle may
both consume these arrays.
"""
from __future__ import annotations

import numpy as np


def init_weights(shapes, seed=0):
    """He-normal initial weights: one FP64 array per shape, drawn in order,
    standard deviation sqrt(2 / fan_in) with fan_in = prod(shape[1:])."""
    rng = np.random.default_rng(seed)
    out = []
    for s in shapes:
        fan_in = int(np.prod(s[1:]))
        out.append(rng.standard_normal(s) * np.sqrt(2.0 / fan_in))
    return out


def random_volume(channels, D, H, W, seed=0, smooth=0):
    """A (channels, D, H, W) FP64 volume of standard normal values, optionally
    smoothed by `smooth` passes of a periodic 3-point box average per axis (test
    inputs with some spatial correlation, like a charge density)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((channels, D, H, W))
    for _ in range(smooth):
        for ax in (1, 2, 3):
            x = (np.roll(x, 1, ax) + x + np.roll(x, -1, ax)) / 3.0
    return x
