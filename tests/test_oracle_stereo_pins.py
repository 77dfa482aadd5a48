"""Pins for the oracle's stereographic chart (Sec. 4.3.1) of the dense cell test:
the cell centre is the inverse projection of the box centre, the covering radius
covers the box, votes equal an independent evaluation, noise-free inliers vote
for the true rotation's cell, and the radius varies by at most the chart's
conformal factor of 2.  Every map here is written out in the test from the
paper's P and P' formulas, not taken from the oracle."""
import math

import numpy as np

from paper_2506_11547_gb300 import synth

STEREO = 1


def P(q):
    """Sec. 4.3.1 projection of (q0, q1, q2, q3) from the pole (0, 0, 0, 1)."""
    q = np.asarray(q, np.float64)
    return q[..., :3] / (1.0 - q[..., 3:4])


def P_inv(p):
    """Sec. 4.3.1 inverse projection P'(p) = (2p, |p|^2 - 1) / (1 + |p|^2)."""
    p = np.asarray(p, np.float64)
    s = np.sum(p * p, axis=-1, keepdims=True)
    return np.concatenate([2 * p, s - 1], axis=-1) / (1 + s)


def box(n, idx):
    ix, iy, iz = idx % n, (idx // n) % n, idx // (n * n)
    h = 2.0 / n
    lo = np.array([-1 + ix * h, -1 + iy * h, -1 + iz * h])
    return (ix, iy, iz), lo, h


def R_of(q):
    """Rotation matrix of a unit quaternion by Rodrigues' formula (independent of the oracle)."""
    w, v = q[0], np.asarray(q[1:])
    s = np.linalg.norm(v)
    if s == 0:
        return np.eye(3)
    return synth.rodrigues(v / s, 2 * math.atan2(s, w))


def test_stereo_centre_is_the_inverse_projection(oracle_mod):
    for n in (2, 5, 16, 64):
        cells = oracle_mod.level_cells(n)
        for idx in cells[:: max(1, len(cells) // 50)]:
            (ix, iy, iz), lo, h = box(n, idx)
            q, _ = oracle_mod.cell_geom(n, ix, iy, iz, chart=STEREO)
            c = lo + h / 2
            assert abs(np.linalg.norm(q) - 1) < 1e-14
            assert np.allclose(q, P_inv(c), atol=1e-15)
            assert np.allclose(P(q), c, atol=1e-12)


def test_stereo_radius_covers_the_box_and_is_not_loose(oracle_mod):
    """Every point of the box (inside the ball or not) maps within r = 2 asin(chord/2)
    of the centre on S^3, and the farthest sampled point reaches over half of r."""
    rng = np.random.default_rng(41)
    for n in (2, 4, 8, 32):
        cells = oracle_mod.level_cells(n)
        pick = cells if len(cells) <= 64 else rng.choice(cells, 64, replace=False)
        for idx in pick:
            (ix, iy, iz), lo, h = box(n, idx)
            q, chord = oracle_mod.cell_geom(n, ix, iy, iz, chart=STEREO)
            r = 2 * math.asin(min(1.0, chord / 2))
            corners = lo + h * np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float)
            pts = np.vstack([lo + h * rng.uniform(0, 1, size=(3000, 3)), corners])
            ang = 2 * np.arcsin(np.clip(np.linalg.norm(P_inv(pts) - q, axis=1) / 2, 0, 1))
            assert ang.max() <= r + 1e-12
            assert ang.max() >= 0.5 * r


def test_stereo_radius_varies_by_the_conformal_factor_only(oracle_mod):
    """|dP'| = 2 |dp| / (1 + |p|^2) lies in [1, 2] |dp| on the unit ball, so cell radii
    of one level differ by about a factor of 2 at most (orthographic cells near the
    rim are far larger)."""
    n = 32
    h = 2.0 / n
    cells = oracle_mod.level_cells(n)
    rs = []
    for idx in cells:
        (ix, iy, iz), _, _ = box(n, idx)
        _, chord = oracle_mod.cell_geom(n, ix, iy, iz, chart=STEREO)
        rs.append(chord)
    rs = np.array(rs)
    assert rs.max() / rs.min() <= 2.3
    # the eight cells at the origin: 2 x half-diagonal / sqrt(1 + |c|^2), |c|^2 = 3 h^2 / 4
    assert abs(rs.max() - math.sqrt(3) * h / math.sqrt(1 + 0.75 * h * h)) < 1e-12


def test_stereo_votes_are_brute_force_and_conservative(oracle_mod):
    """Tiny grids: counts equal an independent evaluation of |b - R(q_c) a|^2/4 <= tau
    with q_c = P'(c); every pair whose circle passes within delta of a sampled point
    of the box is a voter."""
    rng = np.random.default_rng(42)
    for n in (4, 6):
        p = synth.make_problem(16, rho=0.5, sigma=0.01, delta=0.08, seed=43 + n)
        cells = oracle_mod.level_cells(n)
        cnt, _, tau_ = oracle_mod.vote_cells(p.a, p.b, p.delta, n, cells, chart=STEREO)
        a64, b64 = p.a.astype(np.float64), p.b.astype(np.float64)
        cterm = (np.sum(a64 * a64, 1) + np.sum(b64 * b64, 1) - 2) / 4
        for c, idx in enumerate(cells):
            (ix, iy, iz), lo, h = box(n, idx)
            q = P_inv(lo + h / 2)
            _, chord = oracle_mod.cell_geom(n, ix, iy, iz, chart=STEREO)
            v = np.sum((b64 - a64 @ R_of(q).T) ** 2, axis=1) / 4 - cterm
            r = 2 * math.asin(min(1.0, chord / 2))
            t = 1.0 if p.delta + r >= math.pi / 2 else math.sin(p.delta + r) ** 2
            assert abs(t - tau_[c]) < 1e-14
            decided = np.abs(v - t) > 1e-9
            assert np.sum((v <= t) & decided) <= cnt[c] <= np.sum((v <= t) | ~decided)
            qp = P_inv(lo + h * rng.uniform(0, 1, size=(300, 3)))
            for i in range(p.n):
                S = oracle_mod.pair_S(p.a[i], p.b[i])
                d = np.arcsin(np.sqrt(np.clip(np.einsum("kj,jl,kl->k", qp, S, qp), 0, 1)))
                if d.min() <= p.delta:
                    assert oracle_mod.quad(S, q) <= t + 1e-12


def test_stereo_noise_free_inliers_vote_for_the_true_cell_at_every_level(oracle_mod):
    p = synth.make_problem(400, rho=0.7, sigma=0.0, delta=0.01, seed=44)
    inl = ~p.outlier
    q = p.q_true if p.q_true[3] <= 0 else -p.q_true  # the lower-half representative: |P(q)| <= 1
    pt = P(q)
    assert np.linalg.norm(pt) <= 1 + 1e-12
    for n in (8, 16, 32, 64, 128, 256):
        idx = oracle_mod.cell_of_point(n, pt)
        (ix, iy, iz), _, _ = box(n, idx)
        assert oracle_mod.cell_exists(n, ix, iy, iz)
        cnt_in, _, _ = oracle_mod.vote_cells(p.a[inl], p.b[inl], p.delta, n, [idx], chart=STEREO)
        assert cnt_in[0] == inl.sum()


def test_stereo_chart_recovers_rotations_near_w_zero(oracle_mod):
    """Rotations by nearly pi (w ~ 0.05) sit at the rim of the orthographic chart,
    where its cells are widest; in the stereographic chart they are ordinary cells.
    The full solve (32^3 + 2 levels) recovers them."""
    from tests._util import quat_angle
    errs = []
    for seed in range(3):
        rng = np.random.default_rng(500 + seed)
        axis = rng.standard_normal(3)
        axis /= np.linalg.norm(axis)
        ang = 2 * math.acos(0.05)
        p = synth.make_problem(1000, rho=0.9, sigma=0.01, delta=0.03, seed=600 + seed)
        R = synth.rodrigues(axis, ang)
        q = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])
        inl = ~p.outlier
        b = p.a.astype(np.float64) @ R.T + 0.01 * rng.standard_normal((p.n, 3))
        b /= np.linalg.norm(b, axis=1, keepdims=True)
        bb = p.b.copy()
        bb[inl] = b[inl].astype(np.float32)
        r = oracle_mod.solve(p.a, bb, p.delta, grid_n=32, levels=2, chart=STEREO, nthreads=4, trace=False)
        errs.append(quat_angle(r.q, q))
    assert max(errs) < 0.01, errs
