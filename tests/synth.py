"""Seeded synthetic inputs shared by the oracle side and the CUDA side of the parity tests.

This module holds no arithmetic of the method: it only draws reproducible random numbers and
scales given arrays with them.
"""

import numpy as np

from paper_2504_09041_gb300.workloads import ensemble_2d, sine_profile  # noqa: F401 (shared draws)


def perturbed(base: np.ndarray, seed: int, scale: float) -> np.ndarray:
    """base * (1 + scale * U(-1, 1)), elementwise, from a seeded PCG64 stream."""
    rng = np.random.default_rng(seed)
    return base * (1.0 + scale * rng.uniform(-1.0, 1.0, base.shape))


def rates(seed: int, n: int, lo: float = 0.6, hi: float = 1.9) -> np.ndarray:
    """n relaxation rates drawn uniformly in [lo, hi)."""
    return np.random.default_rng(seed).uniform(lo, hi, n)




def sample_nodes(seed: int, shape, count: int, include_corners: bool = True):
    """count distinct (z, y, x) nodes of a box, always including its 8 corners and face centres."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    pts = set()
    if include_corners:
        for z in {0, nz - 1}:
            for y in {0, ny - 1}:
                for x in {0, nx - 1}:
                    pts.add((z, y, x))
        for p in [(nz // 2, ny // 2, 0), (nz // 2, ny // 2, nx - 1), (nz // 2, 0, nx // 2),
                  (nz // 2, ny - 1, nx // 2), (0, ny // 2, nx // 2), (nz - 1, ny // 2, nx // 2)]:
            pts.add(p)
    while len(pts) < count:
        pts.add((int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx))))
    return sorted(pts)
