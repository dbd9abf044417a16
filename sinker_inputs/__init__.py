"""Seeded synthetic inputs for the sinker benchmark (Section 3.2).

This module is shared by the CPU oracle, the tests and the benchmark. It holds
no arithmetic of the method itself: only a counter-based random stream, the
sinker parameters drawn from it, and the workload configurations.

The random stream is splitmix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output i (0-based) of the
stream with seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15 mod 2^64), with
mix the published 64-bit finaliser. A uniform double in [0, 1) is the top 53
bits times 2^-53. The CUDA library implements the same definition to draw the
start vector of its Lanczos eigenvalue estimate.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the splitmix64 stream with `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): top 53 bits of splitmix64 outputs times 2^-53."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, count, offset)


def lanczos_seed(level: int) -> int:
    """Seed of the Lanczos start vector on multigrid level `level` (0 = coarsest)."""
    return 1907_000 + level


@dataclass
class SinkerProblem:
    """Sinker benchmark parameters (Section 3.2).

    mu(x) = X(x) mu_min + (1 - X(x)) mu_max with
    X(x) = prod_i [1 - exp(-delta max(0, |c_i - x| - omega/2)^2)],
    f(x) = (0, 0, beta (X(x) - 1)), homogeneous Dirichlet velocity on the unit cube.
    """
    n: int                      # cells per axis on the finest level
    n_levels: int               # multigrid levels; coarsest has n / 2^(n_levels-1) cells per axis
    centres: np.ndarray         # (n_sinkers, 3)
    mu_min: float
    mu_max: float
    delta: float = 200.0
    omega: float = 0.1
    beta: float = 10.0
    name: str = ""
    seed: int = 0

    @property
    def n_sinkers(self) -> int:
        return int(self.centres.shape[0])

    @property
    def coarse_n(self) -> int:
        return self.n >> (self.n_levels - 1)


def sinker_centres(seed: int, n_sinkers: int) -> np.ndarray:
    """Sinker centres i.i.d. uniform in [0.2, 0.8]^3 from the seeded stream."""
    u = uniform01(seed, 3 * n_sinkers)
    return (0.2 + 0.6 * u).reshape(n_sinkers, 3)


def dr_problem(n: int, n_levels: int, n_sinkers: int, dr: float, seed: int, name: str = "") -> SinkerProblem:
    """Sinker problem with viscosity ratio DR: mu_min = DR^-1/2, mu_max = DR^1/2."""
    return SinkerProblem(n=n, n_levels=n_levels, centres=sinker_centres(seed, n_sinkers),
                         mu_min=dr ** -0.5, mu_max=dr ** 0.5, name=name, seed=seed)


def workload(name: str) -> SinkerProblem:
    """The named synthetic workloads.

    cube8   : 8^3 Q2-Q1 cells, 4 levels, 1 sinker, mu_min = 1, mu_max = 100 (14,739 velocity + 729 pressure DoFs)
    cube64  : 64^3 cells, 7 levels, 8 sinkers, viscosity ratio 1e4 (~6.4M velocity DoFs)
    cube128 : 128^3 cells, 8 levels, 16 sinkers, viscosity ratio 1e6 (~51M velocity DoFs)
    Smaller parity cases: cube16 (16^3, 5 levels, 4 sinkers, DR 1e4), cube32 (32^3, 6 levels, 8 sinkers, DR 1e4).
    Profiling case: cube96 (96^3, 6 levels, 8 sinkers, DR 1e4; FP32 vectors of 86 MB exceed L2).
    Largest case: cube192 (192^3, 7 levels down to 3^3, 16 sinkers, DR 1e6; ~171M velocity DoFs);
    seq24, seq48, seq96: the same sinkers, viscosity ratio and 3^3 coarse grid on 24^3 .. 96^3
    cells (iteration counts under mesh refinement at a fixed problem).
    Sinker centres come from splitmix64 with seed 1907 + k (k = 1, 2, 3 for cube8, cube64, cube128).
    """
    if name == "cube8":
        return SinkerProblem(n=8, n_levels=4, centres=sinker_centres(1908, 1), mu_min=1.0, mu_max=100.0,
                             name=name, seed=1908)
    if name == "cube64":
        return dr_problem(64, 7, 8, 1e4, 1909, name)
    if name == "cube128":
        return dr_problem(128, 8, 16, 1e6, 1910, name)
    if name == "cube192":
        return dr_problem(192, 7, 16, 1e6, 1916, name)
    if name == "cube96":
        return dr_problem(96, 6, 8, 1e4, 1915, name)
    if name in ("seq24", "seq48", "seq96"):   # cube192's problem on coarser meshes (3^3 coarsest)
        n = int(name[3:])
        return dr_problem(n, {24: 4, 48: 5, 96: 6}[n], 16, 1e6, 1916, name)
    if name == "cube16":
        return dr_problem(16, 5, 4, 1e4, 1911, name)
    if name == "cube32":
        return dr_problem(32, 6, 8, 1e4, 1912, name)
    if name == "cube4":
        return dr_problem(4, 3, 1, 1e2, 1913, name)
    if name == "cube2":
        return dr_problem(2, 2, 1, 1e2, 1914, name)
    raise KeyError(name)


@dataclass
class OctreeProblem:
    """Adaptive sinker problem: an octree refined in shells around the sinkers.

    The base mesh is the uniform 2^base_level grid of the unit cube. A leaf is split while
    its level is below its sinker's maximum level and its distance interval to the sinker
    centre meets the shell shell_radius - shell_half_width < |x - c| < shell_radius +
    shell_half_width; then the tree is 2:1 balanced (faces, edges and vertices). The
    coefficients are those of SinkerProblem (Section 3.2). The multigrid hierarchy runs from
    the finest leaf level down to coarsest_level (uniform, <= base_level).
    """
    base_level: int
    coarsest_level: int
    centres: np.ndarray
    max_levels: np.ndarray      # one per sinker
    mu_min: float
    mu_max: float
    shell_radius: float = 0.05
    shell_half_width: float = 0.02
    delta: float = 200.0
    omega: float = 0.1
    beta: float = 10.0
    name: str = ""
    seed: int = 0

    @property
    def n_sinkers(self) -> int:
        return int(self.centres.shape[0])


def octree_problem(base_level, coarsest_level, n_sinkers, level_choices, dr, seed, name=""):
    """Centres from splitmix64(seed) as for the uniform problems; each sinker's maximum
    level drawn uniformly from level_choices with the stream of seed + 1."""
    u = uniform01(seed + 1, n_sinkers)
    lv = np.array([level_choices[min(int(x * len(level_choices)), len(level_choices) - 1)] for x in u])
    return OctreeProblem(base_level=base_level, coarsest_level=coarsest_level,
                         centres=sinker_centres(seed, n_sinkers), max_levels=lv,
                         mu_min=dr ** -0.5, mu_max=dr ** 0.5, name=name, seed=seed)


def octree_workload(name: str) -> OctreeProblem:
    """The named adaptive workloads.

    octree   : base 8^3, 12 sinkers refined to levels 7-9 (drawn per sinker), viscosity ratio 1e6,
               multigrid down to 4^3 (~20M velocity DoFs); seed 1911
    oct_l    : base 8^3, 6 sinkers, levels 7-8, ratio 1e6 (profiling case, a few million DoFs)
    oct_m    : base 8^3, 4 sinkers, levels 5-6, ratio 1e4 (parity case)
    oct_s    : base 4^3, 2 sinkers, levels 4-5, ratio 1e4 (parity case)
    oct_xs   : base 2^3, 1 sinker, level 4, ratio 1e2 (dense-solve case)
    """
    if name == "octree":
        return octree_problem(3, 2, 12, (7, 8, 9), 1e6, 1911, name)
    if name == "oct_l":
        return octree_problem(3, 2, 6, (7, 8), 1e6, 1924, name)
    if name == "oct_m":
        return octree_problem(3, 2, 4, (5, 6), 1e4, 1921, name)
    if name == "oct_s":
        return octree_problem(2, 2, 2, (4, 5), 1e4, 1922, name)
    if name == "oct_xs":
        return octree_problem(1, 1, 1, (4,), 1e2, 1923, name)
    raise KeyError(name)


def adaptive_loop_workload(name: str):
    """(OctreeProblem, cycles) of a solve-estimate-refine loop: the start mesh is the uniform grid
    2^base_level (every sinker's maximum level equals base_level, so no shell is refined) and each
    cycle refines by the gradient indicator.

    adapt    : 16^3 start (4 global refinements, as in Section 3.3), 4 sinkers, viscosity ratio 1e4,
               multigrid down to 4^3, 5 cycles; seed 1926
    adapt_xs : 4^3 start, 1 sinker, ratio 1e2, down to 2^3, 2 cycles (oracle-sized)
    """
    if name == "adapt":
        return octree_problem(4, 2, 4, (4,), 1e4, 1926, name), 5
    if name == "adapt_xs":
        return octree_problem(2, 1, 1, (2,), 1e2, 1927, name), 2
    raise KeyError(name)


# (cells per axis, levels): coarsest 1, 3 or 5 cells per axis
BATCH_SIZES = ((16, 5), (20, 3), (24, 4), (32, 6), (40, 4), (48, 5))
# the small end of the same range: many problems that each leave most of the GPU idle
BATCH_SIZES_SMALL = ((16, 5), (20, 3), (24, 4))


def batch_workload(count: int = 64, seed: int = 1907 + 5, sizes=BATCH_SIZES):
    """Batched sinker problems: size drawn uniformly from BATCH_SIZES ({16, 20, 24, 32, 40, 48}^3
    with a coarsest mesh of at most 5^3 cells), 1-8 sinkers, viscosity ratio log-uniform in [1e2, 1e6];
    all draws from splitmix64 with `seed` (problem i uses seed * 1000 + i for its centres)."""
    u = uniform01(seed, 3 * count)
    probs = []
    for i in range(count):
        n, L = sizes[min(int(u[3 * i] * len(sizes)), len(sizes) - 1)]
        k = 1 + min(int(u[3 * i + 1] * 8), 7)
        dr = 10.0 ** (2.0 + 4.0 * u[3 * i + 2])
        probs.append(dr_problem(n, L, k, dr, seed * 1000 + i, "batch%d" % i))
    return probs


def n_velocity(n: int) -> int:
    return 3 * (2 * n + 1) ** 3


def n_pressure(n: int) -> int:
    return (n + 1) ** 3
