"""Seeded synthetic inputs shared by the GPU path's tests, the oracle's tests and
the benchmark.

This module holds none of the method's arithmetic: it only draws random numbers
(numpy PCG64) in the shapes the paper's workloads have.

* Initial conformations: a random walk of unit bonds from r_0 = 0 with each
  bond direction uniform on the sphere (z ~ U(-1, 1), phi ~ U(0, 2 pi)).  The
  paper draws its initial configurations with cuRAND uniform numbers (Sec. 4,
  random-number paragraph); the freely-jointed walk is the equilibrium
  distribution of the chain without HI.
* Noise: i.i.d. N(0, 1) per bead component per step, [n_steps][sum N][3].
* Uneven batches: chain lengths drawn uniformly from an integer range.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def random_walk(n_beads, seed: int, stretched: bool = False) -> np.ndarray:
    """Packed positions [sum N][3] for chains of the given lengths.

    ``stretched`` places every chain on the x axis instead (a fully extended
    start, used for relaxation tests)."""
    n_beads = np.atleast_1d(np.asarray(n_beads, dtype=np.int64))
    g = rng(seed)
    out = []
    for N in n_beads:
        N = int(N)
        if stretched:
            r = np.zeros((N, 3))
            r[:, 0] = np.arange(N, dtype=np.float64)
        else:
            z = g.uniform(-1.0, 1.0, size=N - 1)
            phi = g.uniform(0.0, 2.0 * np.pi, size=N - 1)
            s = np.sqrt(1.0 - z * z)
            u = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
            r = np.concatenate([np.zeros((1, 3)), np.cumsum(u, axis=0)], axis=0)
        out.append(r)
    return np.ascontiguousarray(np.concatenate(out, axis=0))


def gaussian_noise(n_steps: int, total_beads: int, seed: int,
                   dtype=np.float64) -> np.ndarray:
    """[n_steps][total_beads][3] i.i.d. standard normal numbers."""
    g = rng(seed)
    return np.ascontiguousarray(
        g.standard_normal((int(n_steps), int(total_beads), 3)).astype(dtype, copy=False))


def uneven_lengths(n_chains: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Chain lengths drawn uniformly from {lo, ..., hi}."""
    g = rng(seed)
    return g.integers(lo, hi + 1, size=int(n_chains)).astype(np.int32)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: its chain lengths and physical parameters."""
    name: str
    n_chains: int
    n_beads: int            # 0 when lengths are drawn (uneven batch)
    hstar: float
    dt: float
    flow: int               # 0 none, 1 shear, 2 uniaxial
    Wi: float
    n_steps: int
    precision: int          # 0 fp64, 1 mixed (TF32 panel solves, FP16-operand updates)
    seed: int
    uneven: tuple = ()      # (lo, hi) for drawn lengths
    constraint: int = 0     # 0 rigid rods (tension solve), 1 Fraenkel springs
    kspring: float = 1e4    # Fraenkel spring constant K*

    def lengths(self) -> np.ndarray:
        if self.uneven:
            return uneven_lengths(self.n_chains, self.uneven[0], self.uneven[1], self.seed)
        return np.full(self.n_chains, self.n_beads, dtype=np.int32)


# The workloads of the measurement plan (seed = 1234 + id): five rigid-rod
# workloads and one with the paper's Fraenkel springs.
WORKLOADS = {
    "n16_fp64_eq": Workload("n16_fp64_eq", 1, 16, 0.25, 1e-4, 0, 0.0, 1000, 0, 1235),
    "n100x256_fp64_uniaxial": Workload("n100x256_fp64_uniaxial", 256, 100, 0.25, 1e-4, 2,
                                       10.0, 2000, 0, 1236),
    "n1000x64_mixed_shear": Workload("n1000x64_mixed_shear", 64, 1000, 0.25, 1e-4, 1,
                                     100.0, 500, 1, 1237),
    "n4000x4_mixed_uniaxial": Workload("n4000x4_mixed_uniaxial", 4, 4000, 0.25, 5e-5, 2,
                                       50.0, 100, 1, 1238),
    "uneven50to500x128_fp64": Workload("uneven50to500x128_fp64", 128, 0, 0.25, 1e-4, 2,
                                       5.0, 200, 0, 1239, (50, 500)),
    # the paper's own constraint mode (Fraenkel springs, K* = 1e4 at dt = 1e-4)
    "n1000x64_mixed_fraenkel_shear": Workload("n1000x64_mixed_fraenkel_shear", 64, 1000, 0.25, 1e-4,
                                              1, 100.0, 500, 1, 1240, (), 1, 1e4),
}
