"""The seeded synthetic workloads: graphs plus initial states and parameters.

Each builder returns plain numpy arrays.  Floating-point inputs of the FP32
workloads are rounded to FP32-representable values before they are returned,
so that the FP64 oracle and the FP32 device path start from identical numbers.

Workloads (sizes, distributions and integrator settings):

* ``kuramoto_sbm_small``: N=1000, 5 planted communities of 200, p_in=0.9,
  p_out=0.01, omega ~ N(0,1), theta0 ~ U[0, 2pi), K=4, RK4 dt=0.01, 100
  steps, FP64.
* ``kuramoto_lognormal``: N=262144, 256 communities with lognormal sizes
  (mean 1024, sigma 0.5), p_in=0.95, inter-community Erdos-Renyi links of mean
  degree 8, omega ~ Cauchy(0, 0.5), K=2, RK4 dt=0.01, 2000 steps, FP32 state.
* ``kuramoto_ho``: N=65536, 64 communities of 1024, p_in=0.9, inter degree 4,
  pairwise K1=1 plus triadic K2=2, omega ~ N(0,1), dt=0.005, 1000 steps.
* ``cucker_smale``: N=131072, 128 communities of 1024, p_in=0.9, inter degree
  6, s ~ U[0,10]^2, v ~ N(0,1)^2, dt=0.01, 1000 steps.
* ``kuramoto_ensemble``: independent Kuramoto networks, per instance
  N_i ~ U{256..16384}, M_i ~ U{2..32} communities of equal size (+-1),
  p_in ~ U[0.7, 1.0], integer inter degree ~ U{2..10}, omega ~ N(0,1),
  theta0 ~ U[0, 2pi), K=4, RK4 dt=0.01, 500 steps, FP32, 4096 instances.
  Its graphs come from the row-parallel hash generator (node ids in block
  order), so that all 4096 (about 34 M nodes and 33 G directed links) are
  generated in seconds, one instance at a time.

``scale`` shrinks the node count and community sizes for tests; the structure
(p_in, degree, distributions) is unchanged.
"""
from __future__ import annotations

import dataclasses
import functools

import numpy as np

from .graphs import Graph, equal_sizes, hash_sbm_graph, lognormal_sizes, rng_for, sbm_graph

SEED_BASE = 2203166570


@dataclasses.dataclass
class KuramotoWorkload:
    """Phase oscillators with coupling h(x) = sum_k d_sin[k] sin kx + d_cos[k] cos kx."""

    name: str
    graph: Graph
    theta0: np.ndarray          # float64[n] (FP32-representable for fp32 workloads)
    omega: np.ndarray           # float64[n] (same)
    K: float
    d_sin: np.ndarray           # float64[p]
    d_cos: np.ndarray           # float64[p]
    dt: float
    steps: int
    precision: str              # "fp64" or "fp32"
    K2: float = 0.0             # triadic coupling (higher-order workload)


@dataclasses.dataclass
class CuckerSmaleWorkload:
    name: str
    graph: Graph
    s0: np.ndarray              # float64[n, 2]
    v0: np.ndarray              # float64[n, 2]
    K: float
    sigma: float
    beta: float
    dt: float
    steps: int
    precision: str


def as_fp32_values(x: np.ndarray) -> np.ndarray:
    """Round to the nearest FP32 value, returned as float64."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def _phases(rng, n):
    return rng.uniform(0.0, 2.0 * np.pi, size=n)


def kuramoto_sbm_small(scale: float = 1.0) -> KuramotoWorkload:
    m = 5
    size = max(2, int(round(200 * scale)))
    seed = SEED_BASE + 0
    g = sbm_graph([size] * m, 0.9, p_out=0.01, seed=seed)
    rng = rng_for(seed + 1_000_003)
    omega = rng.normal(0.0, 1.0, size=g.n)
    theta0 = _phases(rng, g.n)
    return KuramotoWorkload("kuramoto_sbm_small", g, theta0, omega, 4.0,
                            np.array([1.0]), np.array([0.0]), 0.01, 100, "fp64")


def kuramoto_lognormal(scale: float = 1.0, steps: int = 2000) -> KuramotoWorkload:
    m = max(2, int(round(256 * scale)))
    n = m * 1024
    seed = SEED_BASE + 1
    rng_sizes = rng_for(seed + 7)
    sizes = lognormal_sizes(n, m, 1024.0, 0.5, rng_sizes)
    g = sbm_graph(sizes, 0.95, inter_degree=8.0, seed=seed)
    rng = rng_for(seed + 1_000_003)
    omega = as_fp32_values(0.5 * rng.standard_cauchy(size=g.n))
    theta0 = as_fp32_values(_phases(rng, g.n))
    return KuramotoWorkload("kuramoto_lognormal", g, theta0, omega, 2.0,
                            np.array([1.0]), np.array([0.0]), 0.01, steps, "fp32")


def kuramoto_ho(scale: float = 1.0, steps: int = 1000) -> KuramotoWorkload:
    m = max(2, int(round(64 * scale)))
    size = 1024 if scale >= 1.0 else max(8, int(round(1024 * scale)))
    seed = SEED_BASE + 2
    g = sbm_graph(equal_sizes(m * size, m), 0.9, inter_degree=4.0, seed=seed)
    rng = rng_for(seed + 1_000_003)
    omega = as_fp32_values(rng.normal(0.0, 1.0, size=g.n))
    theta0 = as_fp32_values(_phases(rng, g.n))
    return KuramotoWorkload("kuramoto_ho", g, theta0, omega, 1.0,
                            np.array([1.0]), np.array([0.0]), 0.005, steps, "fp32", K2=2.0)


def cucker_smale(scale: float = 1.0, steps: int = 1000) -> CuckerSmaleWorkload:
    m = max(2, int(round(128 * scale)))
    size = 1024 if scale >= 1.0 else max(8, int(round(1024 * scale)))
    seed = SEED_BASE + 3
    g = sbm_graph(equal_sizes(m * size, m), 0.9, inter_degree=6.0, seed=seed)
    rng = rng_for(seed + 1_000_003)
    s0 = as_fp32_values(rng.uniform(0.0, 10.0, size=(g.n, 2)))
    v0 = as_fp32_values(rng.normal(0.0, 1.0, size=(g.n, 2)))
    return CuckerSmaleWorkload("cucker_smale", g, s0, v0, 1.0, 1.0, 0.4, 0.01, steps, "fp32")


@dataclasses.dataclass
class EnsembleWorkload:
    """Independent Kuramoto networks evaluated together (one plan, one launch per stage)."""

    name: str
    instances: list             # KuramotoWorkload per instance
    K: float
    dt: float
    steps: int
    precision: str


ENSEMBLE_SEED = SEED_BASE + 4


def ensemble_instance_shape(i: int, n_range=(256, 16384)) -> tuple[int, int, float, int]:
    """(N_i, M_i, p_in, inter degree) of ensemble instance i, without building it."""
    rng = rng_for(ENSEMBLE_SEED + 7919 * (i + 1))
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    m = min(int(rng.integers(2, 33)), n // 2)
    p_in = float(rng.uniform(0.7, 1.0))
    deg = int(rng.integers(2, 11))
    return n, m, p_in, deg


def ensemble_instance(i: int, n_range=(256, 16384), steps: int = 500) -> KuramotoWorkload:
    """Instance i of the seeded ensemble (the same network whatever else is built)."""
    seed = ENSEMBLE_SEED + 7919 * (i + 1)
    rng = rng_for(seed)
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    m = min(int(rng.integers(2, 33)), n // 2)
    p_in = float(rng.uniform(0.7, 1.0))
    deg = int(rng.integers(2, 11))
    g = hash_sbm_graph(equal_sizes(n, m), p_in, inter_degree=float(deg), seed=seed + 1)
    omega = as_fp32_values(rng.normal(0.0, 1.0, size=g.n))
    theta0 = as_fp32_values(_phases(rng, g.n))
    return KuramotoWorkload("kuramoto_ensemble[%d]" % i, g, theta0, omega, 4.0,
                            np.array([1.0]), np.array([0.0]), 0.01, steps, "fp32")


def kuramoto_ensemble(instances: int = 4096, n_range=(256, 16384), steps: int = 500,
                      first: int = 0) -> EnsembleWorkload:
    """Instances first .. first + instances - 1 of the seeded ensemble; n_range
    bounds N_i for tests."""
    out = [ensemble_instance(i, n_range, steps) for i in range(first, first + instances)]
    return EnsembleWorkload("kuramoto_ensemble", out, 4.0, 0.01, steps, "fp32")


@functools.lru_cache(maxsize=4)
def cached(builder: str, scale: float = 1.0):
    """Build a workload once per process (full-size graphs take seconds)."""
    return globals()[builder](scale)
