"""The seeded input generators (the recipe of the synthetic workloads): unit
float32 vectors the library accepts, exact outlier counts, the true rotation's
matrix from its quaternion, noise-free inliers on b = R a, the per-config seeds,
determinism, and the batched, pose and multi-motion shapes."""
import math

import numpy as np

from paper_2506_11547_gb300 import synth


def _R_of_q(q):
    """Rotation matrix of the unit quaternion (w, x, y, z), written out here."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _unit32(v):
    n2 = np.sum(v.astype(np.float64) ** 2, axis=1)
    return v.dtype == np.float32 and np.all(np.abs(n2 - 1.0) <= 1e-6)


def test_problem_recipe():
    for n, rho, sigma, seed in ((1000, 0.9, 0.01, 1), (777, 0.0, 0.0, 2), (501, 0.5, 0.02, 3), (64, 1.0, 0.01, 4)):
        p = synth.make_problem(n, rho, sigma, 0.03, seed=seed)
        assert p.a.shape == p.b.shape == (n, 3) and _unit32(p.a) and _unit32(p.b)
        assert p.outlier.sum() == int(round(rho * n))
        assert abs(np.linalg.norm(p.q_true) - 1) < 1e-12 and p.q_true[0] >= 0
        assert np.allclose(p.R_true, _R_of_q(p.q_true), atol=1e-12)
        inl = ~p.outlier
        res = np.linalg.norm(p.b[inl].astype(np.float64) - p.a[inl].astype(np.float64) @ p.R_true.T, axis=1)
        if sigma == 0:
            assert res.max() < 1e-6
        elif inl.any():
            assert np.median(res) < 3 * sigma  # tangent part of sigma N(0, I3): median ~ 1.18 sigma


def test_determinism_and_config_seeds():
    p1 = synth.make_problem(500, 0.8, 0.01, 0.03, seed=7)
    p2 = synth.make_problem(500, 0.8, 0.01, 0.03, seed=7)
    p3 = synth.make_problem(500, 0.8, 0.01, 0.03, seed=8)
    assert np.array_equal(p1.a, p2.a) and np.array_equal(p1.b, p2.b) and np.array_equal(p1.outlier, p2.outlier)
    assert not np.array_equal(p1.a, p3.a)
    # config k, repetition r: seed SEED_BASE + k + 100 r
    p, grid_n, levels = synth.config_problem("small_n1e3_32", rep=2)
    q = synth.make_problem(1000, 0.9, 0.01, 0.03, seed=synth.SEED_BASE + 0 + 200)
    assert (grid_n, levels) == (32, 0) and np.array_equal(p.a, q.a) and np.array_equal(p.b, q.b)


def test_batched_problem_ranges():
    ps = synth.batched_problems(64)
    assert len(ps) == 64
    for p in ps:
        assert 50 <= p.n <= 20000 and 0.5 <= p.rho <= 0.95 and 0.001 <= p.sigma <= 0.02
        assert math.isclose(p.delta, 3 * p.sigma) and _unit32(p.a) and _unit32(p.b)


def test_pose_and_multi_motion_recipes():
    p = synth.make_pose_problem(400, 0.6, 0.0, seed=11)
    assert p.x.dtype == p.y.dtype == np.float32 and p.outlier.sum() == 240
    assert np.all(np.abs(p.x) <= 1) and np.all(np.abs(p.t_true) <= 1)
    assert np.allclose(p.R_true, _R_of_q(p.q_true), atol=1e-12)
    inl = ~p.outlier
    assert np.abs(p.y[inl] - (p.x[inl].astype(np.float64) @ p.R_true.T + p.t_true)).max() < 1e-6
    m = synth.make_multi_problem(3, 200, sigma=0.0, outlier_frac=0.5, seed=12)
    assert m.n == 900 and (m.label == -1).sum() == 300 and all((m.label == k).sum() == 200 for k in range(3))
    assert np.all(m.q_true[:, 0] >= 0) and _unit32(m.a) and _unit32(m.b)
    for k in range(3):
        sel = m.label == k
        Rk = _R_of_q(m.q_true[k])
        assert np.abs(m.b[sel] - m.a[sel].astype(np.float64) @ Rk.T).max() < 1e-6
