"""Pins for the oracle's rigid-pose front end (Sec. 4.5): the pairwise length
check and unit pairs against a numpy evaluation written here, the invariance
that keeps every pair of a noise-free rigid motion, the translation vote with the
true rotation, and recovery of (R, t) on the paper's synthetic protocol."""
import numpy as np

from paper_2506_11547_gb300 import synth


def _numpy_pairs(x, y, mu, lmin):
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    n = len(x)
    i, j = np.triu_indices(n, 1)  # lexicographic i < j
    m, v = x64[i] - x64[j], y64[i] - y64[j]
    lm, ln = np.linalg.norm(m, axis=1), np.linalg.norm(v, axis=1)
    keep = (lm > lmin) & (ln > lmin) & (np.abs(lm - ln) <= mu)
    return ((m[keep] / lm[keep, None]).astype(np.float32), (v[keep] / ln[keep, None]).astype(np.float32),
            np.abs(lm - ln), keep)


def test_kept_pairs_equal_a_direct_evaluation(oracle_mod):
    p = synth.make_pose_problem(300, 0.5, 0.01, seed=51)
    x, y = p.x.copy(), p.y.copy()
    x[7], y[7] = x[3], y[3]  # a duplicated correspondence: |m| = |n| = 0, never kept
    for mu, lmin in ((0.04, 0.0), (0.1, 0.2), (1e-3, 0.0)):
        a, b = oracle_mod.pose_pairs(x, y, mu, lmin)
        na, nb, d, keep = _numpy_pairs(x, y, mu, lmin)
        # decisions within 1e-12 of mu may differ by the numpy reduction order
        close = np.abs(d - mu) < 1e-12
        assert abs(len(a) - keep.sum()) <= close.sum()
        if not close.any():
            assert np.array_equal(a, na) and np.array_equal(b, nb)
        assert np.all(np.abs(np.sum(a.astype(np.float64) ** 2, 1) - 1) < 1e-6)


def test_noise_free_rigid_motion_keeps_every_pair(oracle_mod):
    """|R m| = |m|: with no noise or outliers every pair passes any mu above float rounding."""
    p = synth.make_pose_problem(200, 0.0, 0.0, seed=52)
    k = oracle_mod.pose_pairs(p.x, p.y, 1e-5, want_pairs=False)
    assert k == 200 * 199 // 2


def test_translation_vote_with_the_true_rotation(oracle_mod):
    """Noise-free inliers all give t_i = t_true: the winning cell is the one holding
    t_true and its count is the number of inliers (up to float32 rounding of y)."""
    for seed in (53, 54, 55):
        p = synth.make_pose_problem(400, 0.6, 0.0, seed=seed)
        L, G = 5.0, 400
        s = 2 * L / G
        c = np.floor((p.t_true + L) / s)
        if np.any(np.abs((p.t_true + L) / s - np.round((p.t_true + L) / s)) < 1e-4):
            continue  # t_true on a cell boundary: float32 rounding may split the inliers
        t, cell, cnt = oracle_mod.pose_translation(p.x, p.y, p.R_true, L, G)
        assert cell == (c[2] * G + c[1]) * G + c[0]
        assert cnt == (~p.outlier).sum()
        assert np.allclose(t, -L + (c + 0.5) * s)


def test_pose_pipeline_recovers_rotation_and_translation(oracle_mod):
    """The paper's synthetic protocol (Sec. 5.4.1) at N = 600, 50% outliers, noise 0.01."""
    from tests._util import quat_angle
    p = synth.make_pose_problem(600, 0.5, 0.01, seed=56)
    r, t, cell, cnt, K = oracle_mod.pose(p.x, p.y, 0.04, 0.03, 32, 2, nthreads=8)
    assert quat_angle(r.q, p.q_true) < 0.01
    assert np.linalg.norm(t - p.t_true) < 0.05
    assert K >= 300 * 299 // 2 * 0.9
