"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and the benchmark.

This module only draws random numbers.  It holds none of the FMM's arithmetic, so both the
FP64 oracle and the CUDA path can take their inputs from it without sharing any method code.

The paper benchmarks only synthetic point clouds (Section 5): points uniform in a volume and
points uniform on the surface of the unit sphere.  The workloads below follow those two
families.  Every array is drawn in FP64 with NumPy's PCG64 generator and then cast to FP32,
so the oracle (which widens the FP32 values back to FP64) and the GPU see identical values.

Seed convention: 0 for points, 1 for charges, 2 for cotangents, 3 for sampled targets.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_POINTS = 0
SEED_CHARGES = 1
SEED_COTANGENT = 2
SEED_SAMPLE = 3


def cube_points(n: int, seed: int = SEED_POINTS) -> np.ndarray:
    """n points i.i.d. uniform in [0,1)^3, float32, shape (n, 3), row-major."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 3)).astype(np.float32)


def sphere_points(n: int, seed: int = SEED_POINTS) -> np.ndarray:
    """n points uniform on the unit sphere surface (normalised Gaussian 3-vectors), float32."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g.astype(np.float32)


def mixed_points(n: int, seed: int = SEED_POINTS, radius: float = 0.15) -> np.ndarray:
    """n points of the two families in one cube, for strongly non-uniform trees: the first n // 2
    uniform in [0,1)^3, the rest uniform on the sphere of the given radius centred at
    (0.5, 0.5, 0.5).  float32, shape (n, 3)."""
    rng = np.random.default_rng(seed)
    a = rng.random((n // 2, 3))
    g = rng.standard_normal((n - n // 2, 3))
    g = 0.5 + radius * g / np.linalg.norm(g, axis=1, keepdims=True)
    return np.concatenate([a, g]).astype(np.float32)


def charges(n: int, kind: str, seed: int = SEED_CHARGES) -> np.ndarray:
    """n charges, float32.  kind: 'u01' (U[0,1)), 'u11' (U[-1,1)) or 'normal' (N(0,1))."""
    rng = np.random.default_rng(seed)
    if kind == "u01":
        q = rng.random(n)
    elif kind == "u11":
        q = 2.0 * rng.random(n) - 1.0
    elif kind == "normal":
        q = rng.standard_normal(n)
    else:
        raise ValueError(f"unknown charge distribution {kind!r}")
    return q.astype(np.float32)


def sample_indices(n: int, m: int, seed: int = SEED_SAMPLE) -> np.ndarray:
    """m distinct indices in [0, n), sorted, int64 (the sampled check targets)."""
    rng = np.random.default_rng(seed)
    m = min(m, n)
    return np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named workload: point family, size, expansion order, tree depth, domain."""

    name: str
    n: int
    dist: str          # 'cube', 'sphere' or 'mixed'
    charge: str        # 'u01', 'u11', 'normal'
    p: int             # expansion order; surface size 6(p-1)^2+2
    depth: int         # uniform octree depth
    origin: tuple      # bounding cube corner
    side: float        # bounding cube side
    gradient: bool

    def points(self, seed: int = SEED_POINTS) -> np.ndarray:
        if self.dist == "mixed":
            return mixed_points(self.n, seed)
        return cube_points(self.n, seed) if self.dist == "cube" else sphere_points(self.n, seed)

    def charges(self, seed: int = SEED_CHARGES) -> np.ndarray:
        return charges(self.n, self.charge, seed)


CUBE = ((0.0, 0.0, 0.0), 1.0)
BALL = ((-1.0, -1.0, -1.0), 2.0)

# The five workloads: a small plain case, a 1M cube, the 8M sphere (the headline),
# the differentiation case and the 33.5M scale case; and a 2M sphere at depth 6, the quarter-
# size stand-in of the headline (the same ~112 points per non-empty leaf) for timed CPU samples
# and for profiler captures that must stay small.
WORKLOADS = {
    "cube20k_p4_d3": Workload("cube20k_p4_d3", 20_000, "cube", "u01", 4, 3, *CUBE, False),
    "cube1m_p6_d5": Workload("cube1m_p6_d5", 1_048_576, "cube", "u11", 6, 5, *CUBE, True),
    "sphere8m_p6_d7": Workload("sphere8m_p6_d7", 8_388_608, "sphere", "u01", 6, 7, *BALL, True),
    "cube262k_p6_d4": Workload("cube262k_p6_d4", 262_144, "cube", "normal", 6, 4, *CUBE, True),
    "cube33m_p8_d8": Workload("cube33m_p8_d8", 33_554_432, "cube", "u01", 8, 8, *CUBE, True),
    "sphere2m_p6_d6": Workload("sphere2m_p6_d6", 2_097_152, "sphere", "u01", 6, 6, *BALL, True),
    # p = 8 at a size where both forms of the M2L (dense and FFT) run in a bench step: the scale
    # case's order and cube family at an eighth of its points and depth 6 (16 points per leaf)
    "cube4m_p8_d6": Workload("cube4m_p8_d6", 4_194_304, "cube", "u01", 8, 6, *CUBE, True),
    # strongly non-uniform points for the adaptive tree: half uniform in the unit cube, half on a
    # sphere of radius 0.15 inside it, refined to depth 9
    "mixed1m_p6_d9": Workload("mixed1m_p6_d9", 1_048_576, "mixed", "u01", 6, 9, *CUBE, True),
}


def scaled(w: Workload, n: int, depth: int | None = None, p: int | None = None) -> Workload:
    """A smaller copy of workload w (same family and charges) for quick tests."""
    return dataclasses.replace(w, name=f"{w.name}@{n}", n=n,
                               depth=w.depth if depth is None else depth,
                               p=w.p if p is None else p)
