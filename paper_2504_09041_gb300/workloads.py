"""Seeded synthetic workloads: the parameter draws of the benchmark problems.

Nothing here computes any part of the method; the module only draws reproducible parameters
(box sizes, Rayleigh and Prandtl numbers, wall-temperature profiles) that the tests, the
benchmark and users share.
"""
from __future__ import annotations

import math

import numpy as np

# Side lengths of the square cavities of the ensemble workload.
ENSEMBLE_SIDES = (64, 96, 128, 192, 256, 384, 512)


def ensemble_2d(seed: int = 4, count: int = 64, sides=ENSEMBLE_SIDES, Ra_range=(1e3, 1e7),
                Pr_range=(0.71, 7.0)):
    """An ensemble of independent square cavities: side drawn uniformly from `sides`, Ra
    log-uniform in Ra_range, Pr uniform in Pr_range, all from one seeded PCG64 stream.
    Returns (sizes [(nx, ny)], Ra [count], Pr [count])."""
    rng = np.random.default_rng(seed)
    side = rng.choice(np.asarray(sides), size=count)
    Ra = 10.0 ** rng.uniform(math.log10(Ra_range[0]), math.log10(Ra_range[1]), count)
    Pr = rng.uniform(Pr_range[0], Pr_range[1], count)
    return [(int(s), int(s)) for s in side], Ra.tolist(), Pr.tolist()


def sine_profile(seed: int, n: int, base: float = 1.0, amp: float = 0.05, modes: int = 4):
    """base + amp * sum_k a_k sin(pi k (j + 1/2) / n), a_k uniform in [-1, 1], j = 0..n-1."""
    a = np.random.default_rng(seed).uniform(-1.0, 1.0, modes)
    j = np.arange(n) + 0.5
    return base + amp * sum(a[k] * np.sin(math.pi * (k + 1) * j / n) for k in range(modes))
