"""Pins for the oracle's Alg. 1 (Sec. 4.3.2): the circle basis, the samples,
the stereographic projection and the argmax, each checked against something
other than the Alg. 1 code itself -- the rotation matrix of App. A, the
S-matrix of the pair step, the inverse projection, Rodrigues' formula and a
noise-free ground truth."""
import numpy as np
import pytest

from paper_2506_11547_gb300 import synth


def _oracle():
    import oracle
    return oracle


def _unit(rng, n):
    x = rng.standard_normal((n, 3))
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def _rodrigues_R(q):
    """Rotation matrix of a unit quaternion (w, x, y, z) by Rodrigues' formula
    R = I + 2w [v]x + 2 [v]x^2 (written here independently of the oracle)."""
    w, v = q[0], np.asarray(q[1:])
    K = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    return np.eye(3) + 2 * w * K + 2 * K @ K


def test_basis_is_orthonormal_and_q_b1_is_the_minimal_rotation():
    o = _oracle()
    rng = np.random.default_rng(1)
    a, b = _unit(rng, 50), _unit(rng, 50)
    for i in range(50):
        ok, q1, q2 = o.alg1_basis(a[i], b[i])
        assert ok
        # unit up to the float32 rounding of a and b (|a|^2 - 1 ~ 1e-7); orthogonal exactly
        assert abs(q1 @ q1 - 1) < 1e-6 and abs(q2 @ q2 - 1) < 1e-6 and abs(q1 @ q2) < 1e-14
        ai, bi = a[i].astype(np.float64), b[i].astype(np.float64)
        # q_b1 maps a to b, and its axis is perpendicular to both (minimal rotation)
        assert np.allclose(_rodrigues_R(q1) @ ai, bi, atol=1e-6)
        assert abs(q1[1:] @ ai) < 1e-6 and abs(q1[1:] @ bi) < 1e-6


def test_every_sample_lies_on_the_pairs_quaternion_circle():
    """R(q(alpha)) a = b for every alpha, and q(alpha)^T S q(alpha) = 0 with S the
    pair step's App. A matrix: the sampled curve is the circle of Lemma 1."""
    o = _oracle()
    rng = np.random.default_rng(2)
    a, b = _unit(rng, 20), _unit(rng, 20)
    cs = o.alg1_table(36)
    for i in range(20):
        ok, q1, q2 = o.alg1_basis(a[i], b[i])
        S = o.pair_S(a[i], b[i])
        for cj, sj in cs:
            q = q1 * cj + q2 * sj
            assert abs(np.linalg.norm(q) - 1) < 1e-6
            assert np.allclose(_rodrigues_R(q) @ a[i].astype(np.float64), b[i], atol=2e-6)
            assert abs(q @ S @ q) < 1e-6


def test_table_is_the_uniform_discretisation_of_minus_pi_to_pi():
    o = _oracle()
    J = 180
    cs = o.alg1_table(J)
    alpha = -np.pi + 2 * np.pi * np.arange(J) / J
    assert np.allclose(cs[:, 0], np.cos(alpha / 2), atol=1e-15)
    assert np.allclose(cs[:, 1], np.sin(alpha / 2), atol=1e-15)


def test_projection_of_the_lower_half_lands_in_the_unit_ball_and_inverts():
    """Cell of a sample vs the inverse projection of Sec. 4.3.1: the sample's cell
    centre maps back (P') to within the cell's reach of the sample itself."""
    o = _oracle()
    rng = np.random.default_rng(3)
    n = 64
    h = 2.0 / n
    a, b = _unit(rng, 30), _unit(rng, 30)
    cs = o.alg1_table(24)
    for i in range(30):
        _, q1, q2 = o.alg1_basis(a[i], b[i])
        for cj, sj in cs:
            q = q1 * cj + q2 * sj
            if q[3] > 0:
                q = -q
            p = q[:3] / (1 - q[3])
            assert np.linalg.norm(p) <= 1 + 1e-6  # |q| = 1 up to the float32 inputs
            pp = p @ p
            q_back = np.concatenate([2 * p, [pp - 1]]) / (1 + pp)  # P'(P(q)) = q
            assert np.allclose(q_back, q, atol=1e-6)
            idx = o.alg1_cell(q1, q2, cj, sj, n)
            ix, iy, iz = idx % n, (idx // n) % n, idx // (n * n)
            centre = -1 + (np.array([ix, iy, iz]) + 0.5) * h
            assert np.all(np.abs(centre - p) <= h / 2 + 1e-12)


def test_counts_sum_to_samples_and_noise_free_argmax_finds_the_rotation():
    o = _oracle()
    for seed in (11, 12, 13):
        p = synth.make_problem(400, rho=0.0, sigma=0.0, delta=0.03, seed=seed)
        n, J = 48, 90
        acc, bi, bc, q, cast = o.alg1(p.a, p.b, J, n)
        assert cast == 400 * J and acc.sum() == cast and acc[bi] == bc == acc.max()
        assert np.argmax(acc) == bi  # ties to the smallest index
        # the winner's centre is within the cell's reach of the true rotation
        qt = p.q_true if p.q_true[3] <= 0 else -p.q_true
        pt = qt[:3] / (1 - qt[3])
        ix, iy, iz = bi % n, (bi // n) % n, bi // (n * n)
        centre = -1 + (np.array([ix, iy, iz]) + 0.5) * (2.0 / n)
        assert np.all(np.abs(centre - pt) <= 2.0 / n)
        assert min(np.linalg.norm(q - p.q_true), np.linalg.norm(q + p.q_true)) < 4.0 / n


def test_outliers_do_not_move_the_noise_free_winner():
    o = _oracle()
    p = synth.make_problem(2000, rho=0.8, sigma=0.0, delta=0.03, seed=21)
    clean = synth.make_problem(2000, rho=0.0, sigma=0.0, delta=0.03, seed=21)
    _, bi, _, _, _ = o.alg1(p.a, p.b, 120, 40)
    ins = ~p.outlier
    _, bi2, _, _, _ = o.alg1(p.a[ins], p.b[ins], 120, 40)
    assert bi == bi2


# ---- multiple rotations (Sec. 4.4): peaks by greedy non-maximum suppression ----

def _angle(q1, q2):
    from tests._util import quat_angle
    return quat_angle(q1, q2)


def test_one_peak_is_the_argmax():
    o = _oracle()
    p = synth.make_problem(1500, rho=0.7, sigma=0.01, delta=0.03, seed=31)
    acc, bi, bc, q, _ = o.alg1(p.a, p.b, 180, 64)
    idx, cnt, qs, T = o.alg1_peaks(acc, 64, 1, 0.1)
    assert list(idx) == [bi] and list(cnt) == [bc] and np.array_equal(qs[0], q)


def test_peaks_obey_the_greedy_suppression_invariants():
    """Independently of how the oracle orders its work: (i) T is the rule's value;
    (ii) peaks come in (count desc, index asc) order, pairwise farther apart than
    theta; (iii) every candidate ranked before the last peak that is not a peak lies
    within theta of an earlier-ranked peak; (iv) with fewer than M peaks, every
    candidate is a peak or suppressed."""
    o = _oracle()
    mp = synth.make_multi_problem(4, 800, sigma=0.01, outlier_frac=0.5, seed=32)
    n, theta = 60, 0.15
    acc, *_ = o.alg1(mp.a, mp.b, 180, n)
    for M, kmax, min_count in ((6, 16384, 1), (40, 300, 1), (6, 16384, 25)):
        idx, cnt, qs, T = o.alg1_peaks(acc, n, M, theta, min_count=min_count, kmax=kmax)
        ge = lambda t: int(np.sum(acc >= t))
        t0 = 1
        while ge(t0) > kmax:
            t0 += 1
        assert T == max(t0, min_count)
        cand = np.nonzero(acc >= T)[0]
        order = sorted(cand, key=lambda c: (-acc[c], c))
        rank = {c: r for r, c in enumerate(order)}
        assert [rank[c] for c in idx] == sorted(rank[c] for c in idx)
        centre = {c: o.alg1_centre(n, c) for c in order}
        for i in range(len(idx)):
            assert np.allclose(qs[i], centre[idx[i]])
            for j in range(i):
                assert _angle(qs[i], qs[j]) > theta - 1e-9
        last = rank[idx[-1]] if len(idx) == M else len(order) - 1
        picked = set(idx.tolist())
        for c in order[: last + 1]:
            if c in picked:
                continue
            assert any(rank[pk] < rank[c] and _angle(centre[c], centre[pk]) <= theta + 1e-9 for pk in idx)


def test_peaks_recover_every_rotation_of_a_multi_motion_scene():
    """Noise-free scene of three motions with 1000 pairs each and 50% extra outliers:
    the three highest peaks are the three rotations, each within its cell's reach."""
    o = _oracle()
    mp = synth.make_multi_problem(3, 1000, sigma=0.0, outlier_frac=0.5, seed=33)
    n = 120
    acc, *_ = o.alg1(mp.a, mp.b, 540, n)
    idx, cnt, qs, T = o.alg1_peaks(acc, n, 3, 0.2)
    assert len(idx) == 3
    for qt in mp.q_true:
        assert min(_angle(q, qt) for q in qs) < 2 * 4.0 / n
