"""Seeded synthetic correspondence generators.

This module is shared by the tests, the benchmark and the oracle's callers.
It holds none of the voting method's arithmetic: it only draws random unit
vectors, a random ground-truth rotation and Gaussian noise, following the
synthetic protocol of Sec. 5.2 / Sec. 5.3.1 of the paper (random rotation,
random unit observations, Gaussian perturbation of the targets followed by
re-normalisation, and a chosen fraction of targets replaced by random
directions to act as mismatches).

The ground-truth rotation is built from an axis and an angle with the
Rodrigues formula, so that nothing here shares a formula with the
quaternion-to-matrix map the method (and its oracle) use.

All arithmetic is float64; the returned observation arrays are float32,
row-major [n, 3], which is the input format of the library.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem",
    "make_problem",
    "rodrigues",
    "config_problem",
    "batched_problems",
    "serving_stream",
    "MultiProblem",
    "make_multi_problem",
    "PoseProblem",
    "make_pose_problem",
    "make_bundle_problem",
    "SEED_BASE",
]

SEED_BASE = 1000


@dataclasses.dataclass
class Problem:
    """One synthetic rotation problem: b_i ~ R a_i for the inliers."""

    a: np.ndarray          # float32 [n, 3], unit rows
    b: np.ndarray          # float32 [n, 3], unit rows
    q_true: np.ndarray     # float64 [4], (w, x, y, z), w >= 0
    R_true: np.ndarray     # float64 [3, 3]
    outlier: np.ndarray    # bool [n], True where b_i was replaced
    delta: float           # vote tolerance (radians on S^3)
    sigma: float
    rho: float

    @property
    def n(self) -> int:
        return int(self.a.shape[0])


def _normalize_rows(x: np.ndarray) -> np.ndarray:
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def rodrigues(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rotation by `angle` about unit `axis`: I + sin(t) K + (1 - cos(t)) K^2."""
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def _random_rotation(rng: np.random.Generator):
    """Uniform random rotation: a uniform unit quaternion drawn as a normalised
    4-D Gaussian, with w >= 0, returned with its axis-angle matrix."""
    g = rng.standard_normal(4)
    g /= np.linalg.norm(g)
    if g[0] < 0:
        g = -g
    w = min(1.0, float(g[0]))
    angle = 2.0 * math.acos(w)
    v = g[1:]
    nv = np.linalg.norm(v)
    axis = v / nv if nv > 0 else np.array([1.0, 0.0, 0.0])
    return g, rodrigues(axis, angle)


def make_problem(n: int, rho: float, sigma: float, delta: float, seed: int,
                 same_axis_frac: float = 0.0) -> Problem:
    """Synthetic correspondences.

    a_i uniform on S^2; b_i = normalize(R a_i + sigma * N(0, I3)); an exact
    round(rho * n) subset chosen by a seeded permutation has b_i replaced by a
    uniform direction. With `same_axis_frac` > 0, that fraction of the n pairs
    (taken from the outlier subset) instead follows a rotation about the true
    axis by a random different angle: the structured "same-axis" mismatches
    of the paper's Table I experiment.
    """
    rng = np.random.default_rng(seed)
    q, R = _random_rotation(rng)
    a = _normalize_rows(rng.standard_normal((n, 3)))
    b = a @ R.T
    if sigma > 0:
        b = b + sigma * rng.standard_normal((n, 3))
    b = _normalize_rows(b)
    n_out = int(round(rho * n))
    perm = rng.permutation(n)
    out_idx = perm[:n_out]
    outlier = np.zeros(n, dtype=bool)
    outlier[out_idx] = True
    b[out_idx] = _normalize_rows(rng.standard_normal((n_out, 3)))
    n_same = min(n_out, int(round(same_axis_frac * n)))
    if n_same > 0:
        v = q[1:]
        axis = v / np.linalg.norm(v) if np.linalg.norm(v) > 0 else np.array([1.0, 0.0, 0.0])
        sel = out_idx[:n_same]
        for i in sel:
            Ri = rodrigues(axis, float(rng.uniform(-math.pi, math.pi)))
            b[i] = Ri @ a[i]
    return Problem(a=a.astype(np.float32), b=b.astype(np.float32), q_true=q,
                   R_true=R, outlier=outlier, delta=float(delta),
                   sigma=float(sigma), rho=float(rho))


def make_bundle_problem(n: int, spread: float, seed: int, about_axis: bool = False) -> Problem:
    """Noise-free correspondences whose observations a_i form a narrow bundle:
    a_i = normalize(a0 + spread * N(0, I3)), b_i = R a_i.  With a bundle the
    rotation about a0 is barely constrained, so the inlier set is close to the
    degenerate case of all-parallel observations (the smaller the spread, the
    closer).  about_axis=True takes a0 along the rotation axis itself, where
    b_i ~ a_i (the pairs of the paper's same-axis setting, Table I); otherwise
    a0 is a uniform direction."""
    rng = np.random.default_rng(seed)
    q, R = _random_rotation(rng)
    if about_axis:
        v = q[1:]
        a0 = v / np.linalg.norm(v)
    else:
        a0 = _normalize_rows(rng.standard_normal((1, 3)))[0]
    a = _normalize_rows(a0[None, :] + spread * rng.standard_normal((n, 3)))
    b = _normalize_rows(a @ R.T)
    return Problem(a=a.astype(np.float32), b=b.astype(np.float32), q_true=q, R_true=R,
                   outlier=np.zeros(n, dtype=bool), delta=0.03, sigma=0.0, rho=0.0)


# Synthetic workload shapes (Sec. 5.3.1 of the paper: N up to 1e6, outlier
# ratio up to 0.99, noise 0.005 .. 0.02).
_CONFIGS = {
    # name: (n, rho, sigma, delta, grid_n, levels)
    "small_n1e3_32": (1000, 0.90, 0.010, 0.03, 32, 0),
    "fp32_n1e5_64L3": (100000, 0.99, 0.010, 0.03, 64, 3),
    "lowp_n1e6_128L3": (1000000, 0.99, 0.005, 0.03, 128, 3),
}


def config_problem(name: str, rep: int = 0):
    """(Problem, grid_n, levels) of a named single-problem workload."""
    n, rho, sigma, delta, grid_n, levels = _CONFIGS[name]
    idx = list(_CONFIGS).index(name)
    p = make_problem(n, rho, sigma, delta, seed=SEED_BASE + idx + 100 * rep)
    return p, grid_n, levels


def batched_problems(count: int = 4096, seed: int = SEED_BASE + 3,
                     n_lo: int = 50, n_hi: int = 20000):
    """Independent problems with N log-uniform in [n_lo, n_hi], outlier ratio
    uniform in [0.5, 0.95], noise uniform in [0.001, 0.02] and delta = 3 sigma."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count)).astype(np.int64)
    rhos = rng.uniform(0.5, 0.95, size=count)
    sigmas = rng.uniform(0.001, 0.02, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    out = []
    for k in range(count):
        out.append(make_problem(int(ns[k]), float(rhos[k]), float(sigmas[k]),
                                3.0 * float(sigmas[k]), seed=int(seeds[k])))
    return out


def serving_stream(count: int, rate_hz: float = 2000.0, seed: int = SEED_BASE + 4,
                   n_lo: int = 100, n_hi: int = 100000, delta: float = 0.03):
    """Poisson arrivals at `rate_hz`; N log-uniform in [n_lo, n_hi]; outlier
    ratio uniform in [0.8, 0.99]; sigma = 0.01. Returns (arrival_s, problems)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count)).astype(np.int64)
    rhos = rng.uniform(0.8, 0.99, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    probs = [make_problem(int(ns[k]), float(rhos[k]), 0.01, delta, seed=int(seeds[k]))
             for k in range(count)]
    return t, probs


@dataclasses.dataclass
class MultiProblem:
    """Correspondences from several rotation motions in one scene (Sec. 4.4)."""

    a: np.ndarray          # float32 [n, 3]
    b: np.ndarray          # float32 [n, 3]
    q_true: np.ndarray     # float64 [models, 4], w >= 0
    label: np.ndarray      # int [n]: the motion of each pair, -1 for outliers

    @property
    def n(self) -> int:
        return int(self.a.shape[0])


def make_multi_problem(models: int, per_model: int, sigma: float = 0.01, outlier_frac: float = 0.0,
                       seed: int = SEED_BASE + 5) -> MultiProblem:
    """`models` uniform random rotations with `per_model` pairs each (a uniform on
    S^2, b = normalize(R_m a + sigma N(0, I3))), plus round(outlier_frac * total)
    pairs with b uniform, shuffled by a seeded permutation: the multiple-rotation
    protocol of the paper's Sec. 5.5.1."""
    rng = np.random.default_rng(seed)
    qs, aa, bb, lab = [], [], [], []
    for m in range(models):
        q, R = _random_rotation(rng)
        a = _normalize_rows(rng.standard_normal((per_model, 3)))
        b = a @ R.T
        if sigma > 0:
            b = b + sigma * rng.standard_normal((per_model, 3))
        qs.append(q)
        aa.append(a)
        bb.append(_normalize_rows(b))
        lab.append(np.full(per_model, m))
    n_out = int(round(outlier_frac * models * per_model))
    if n_out:
        aa.append(_normalize_rows(rng.standard_normal((n_out, 3))))
        bb.append(_normalize_rows(rng.standard_normal((n_out, 3))))
        lab.append(np.full(n_out, -1))
    a, b, label = np.concatenate(aa), np.concatenate(bb), np.concatenate(lab)
    perm = rng.permutation(len(label))
    return MultiProblem(a=a[perm].astype(np.float32), b=b[perm].astype(np.float32), q_true=np.array(qs),
                        label=label[perm])


@dataclasses.dataclass
class PoseProblem:
    """Point correspondences under a rigid motion y = R x + t (Sec. 4.5)."""

    x: np.ndarray          # float32 [n, 3]
    y: np.ndarray          # float32 [n, 3]
    q_true: np.ndarray     # float64 [4], w >= 0
    R_true: np.ndarray     # float64 [3, 3]
    t_true: np.ndarray     # float64 [3]
    outlier: np.ndarray    # bool [n]

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def make_pose_problem(n: int, rho: float, sigma: float, seed: int = SEED_BASE + 6) -> PoseProblem:
    """The paper's rigid-pose protocol (Sec. 5.4.1): x_i uniform in [-1, 1]^3,
    y_i = R x_i + t + sigma N(0, I3) with t uniform in [-1, 1]^3; an exact
    round(rho n) subset (seeded permutation) has x_i and y_i both uniform in
    [-1, 1]^3."""
    rng = np.random.default_rng(seed)
    q, R = _random_rotation(rng)
    t = rng.uniform(-1.0, 1.0, 3)
    x = rng.uniform(-1.0, 1.0, (n, 3))
    y = x @ R.T + t
    if sigma > 0:
        y = y + sigma * rng.standard_normal((n, 3))
    n_out = int(round(rho * n))
    perm = rng.permutation(n)
    out = np.zeros(n, dtype=bool)
    out[perm[:n_out]] = True
    x[out] = rng.uniform(-1.0, 1.0, (n_out, 3))
    y[out] = rng.uniform(-1.0, 1.0, (n_out, 3))
    return PoseProblem(x=x.astype(np.float32), y=y.astype(np.float32), q_true=q, R_true=R, t_true=t, outlier=out)
