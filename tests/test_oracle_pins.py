"""Pins for the FP64 oracle: each test checks the oracle against something other
than itself -- a formula or value printed in the paper, a closed form, an
invariant, a library routine, or brute force on a tiny input."""
import math
import os

import numpy as np
import pytest

from paper_2506_11547_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _unit(rng, n=1):
    x = rng.standard_normal((n, 3))
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def _rand_q(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    return q


def _quat_mul(p, q):
    w1, v1 = p[0], np.asarray(p[1:])
    w2, v2 = q[0], np.asarray(q[1:])
    return np.concatenate([[w1 * w2 - v1 @ v2], w1 * v2 + w2 * v1 + np.cross(v1, v2)])


# --------------------------------------------------------------------------
# 1. pair step
# --------------------------------------------------------------------------

def test_M_eigenvalues_are_pm1(oracle_mod):
    """App. A: det(M - lambda I) = (lambda^2 - 1)^2, eigenvalues (1, 1, -1, -1)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        a, b = _unit(rng)[0], _unit(rng)[0]
        M = oracle_mod.pair_M(a, b)
        assert np.allclose(M, M.T, atol=1e-15)
        ev = np.linalg.eigvalsh(M)
        assert np.allclose(ev, [-1, -1, 1, 1], atol=1e-6)  # float32 inputs: |a|,|b| = 1 +- 1e-7


def test_quadform_is_bRa_with_rodrigues_rotation(oracle_mod):
    """q^T M q = b^T R(q) a (App. A) with R built independently by Rodrigues'
    axis-angle formula, for q = (cos t/2, sin t/2 k)."""
    rng = np.random.default_rng(2)
    for _ in range(30):
        k = rng.standard_normal(3)
        k /= np.linalg.norm(k)
        t = rng.uniform(-math.pi, math.pi)
        q = np.concatenate([[math.cos(t / 2)], math.sin(t / 2) * k])
        R = synth.rodrigues(k, t)
        assert np.allclose(oracle_mod.quat_to_R(q), R, atol=1e-14)
        a, b = _unit(rng)[0], _unit(rng)[0]
        M = oracle_mod.pair_M(a, b)
        assert abs(q @ M @ q - b.astype(np.float64) @ R @ a.astype(np.float64)) < 1e-14


def test_S_equals_appD_AtA_over_4(oracle_mod):
    """App. D: A = [[0, (a-b)^T], [-(a-b), [a+b]x]] with A q = 0 on the circle;
    S = (I - M)/2 equals A^T A / 4 (for unit a, b)."""
    rng = np.random.default_rng(3)
    for _ in range(30):
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        b = rng.standard_normal(3)
        b /= np.linalg.norm(b)
        a32, b32 = a.astype(np.float32), b.astype(np.float32)
        a64, b64 = a32.astype(np.float64), b32.astype(np.float64)
        d, p = a64 - b64, a64 + b64
        A = np.zeros((4, 4))
        A[0, 1:] = d
        A[1:, 0] = -d
        A[1:, 1:] = [[0, -p[2], p[1]], [p[2], 0, -p[0]], [-p[1], p[0], 0]]
        S = oracle_mod.pair_S(a32, b32)
        # A^T A/4 - S = (|a|^2 + |b|^2 - 2)/4 I exactly (a float32 non-unit term)
        c = (a64 @ a64 + b64 @ b64 - 2) / 4
        assert np.allclose(A.T @ A / 4 - S, c * np.eye(4), atol=1e-15)
        # the four rows of A are -1 eigenvectors of M (App. D)
        M = oracle_mod.pair_M(a32, b32)
        assert np.allclose(M @ A.T, -A.T, atol=1e-6)


def _load_special_eigvecs():
    cols = {}
    with open(os.path.join(HERE, "golden", "appA_special_eigvecs.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x) for x in line.split()]
            cols.setdefault(v[0], {})[v[1]] = np.array(v[2:], dtype=np.float64)
    return cols


def test_S_from_appA_special_example(oracle_mod):
    """App. A 'Special Example': the printed e1..e4 are eigenvectors of M with
    eigenvalues (1, 1, -1, -1); Gram-Schmidt of e1, e2 gives beta1, beta2 and
    S = I - (beta1 beta1^T + beta2 beta2^T)."""
    cols = _load_special_eigvecs()
    rng = np.random.default_rng(4)
    for _ in range(30):
        a32, b32 = _unit(rng)[0], _unit(rng)[0]
        var = np.concatenate([a32, b32]).astype(np.float64)
        e = {k: np.array([cols[k][r] @ var for r in range(4)]) for k in cols}
        M = oracle_mod.pair_M(a32, b32)
        for k, lam in ((1, 1.0), (2, 1.0), (3, -1.0), (4, -1.0)):
            assert np.allclose(M @ e[k], lam * e[k], atol=1e-6)
        b1 = e[1] / np.linalg.norm(e[1])
        bt = e[2] - (e[2] @ b1) * b1
        b2 = bt / np.linalg.norm(bt)
        P = np.outer(b1, b1) + np.outer(b2, b2)
        assert np.allclose(oracle_mod.pair_S(a32, b32), np.eye(4) - P, atol=1e-6)


def test_S_is_projector_and_vanishes_at_true_q(oracle_mod):
    """S^2 = S, trace S = 2 (rank 2), S q_true = 0 for noise-free pairs."""
    p = synth.make_problem(64, rho=0.0, sigma=0.0, delta=0.03, seed=5)
    for i in range(p.n):
        S = oracle_mod.pair_S(p.a[i], p.b[i])
        assert np.allclose(S @ S, S, atol=1e-6)
        assert abs(np.trace(S) - 2.0) < 1e-6
        assert np.linalg.norm(S @ p.q_true) < 1e-6
        # (1 - b.Ra)/2 with float32 |a|, |b| = 1 +- 6e-8
        assert abs(oracle_mod.quad(S, p.q_true)) < 2e-7


def test_quad_equals_residual_over_4(oracle_mod):
    """q^T S q = |b - R(q) a|^2 / 4 = sin^2(theta/2), theta = angle(R a, b),
    with R from Rodrigues' formula (independent of App. A)."""
    rng = np.random.default_rng(6)
    for _ in range(50):
        k = rng.standard_normal(3)
        k /= np.linalg.norm(k)
        t = rng.uniform(-math.pi, math.pi)
        q = np.concatenate([[math.cos(t / 2)], math.sin(t / 2) * k])
        R = synth.rodrigues(k, t)
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        b = rng.standard_normal(3)
        b /= np.linalg.norm(b)
        v = oracle_mod.quad(oracle_mod.pair_S(a.astype(np.float32), b.astype(np.float32)), q)
        a64, b64 = a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
        ra = R @ a64
        theta = math.atan2(np.linalg.norm(np.cross(ra, b64)), ra @ b64)
        assert abs(v - math.sin(theta / 2) ** 2) < 3e-7  # float32 inputs: |a|^2-1 ~ 1e-7
        exact = (1 - b64 @ ra) / 2   # bilinear closed form, exact for any input norm
        assert abs(v - exact) < 1e-15


def _circle_basis(a, b):
    """Sec. 4.1: q_b1 = quaternion of the minimal-geodesic rotation a -> b,
    q_b2 = [-b^T q123, q0 b + b x q123]."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    a = a / np.linalg.norm(a)
    b = b / np.linalg.norm(b)
    th = math.acos(max(-1.0, min(1.0, a @ b)))
    c = np.cross(a, b)
    c /= np.linalg.norm(c)
    qb1 = np.concatenate([[math.cos(th / 2)], math.sin(th / 2) * c])
    q0, q123 = qb1[0], qb1[1:]
    qb2 = np.concatenate([[-(b @ q123)], q0 * b + np.cross(b, q123)])
    return qb1, qb2


def test_vote_value_is_sin2_of_distance_to_circle(oracle_mod):
    """Brute force: the S^3 angle from q to the nearest point of the quaternion
    circle q(alpha) = q_b1 cos(alpha/2) + q_b2 sin(alpha/2) (Sec. 4.1), found by
    dense sampling plus golden-section refinement, equals asin(sqrt(q^T S q))."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        a, b = _unit(rng)[0], _unit(rng)[0]
        qb1, qb2 = _circle_basis(a, b)
        # the sampled circle really is the solution set: R(q(alpha)) a = b
        for al in np.linspace(-math.pi, math.pi, 7):
            qa = qb1 * math.cos(al / 2) + qb2 * math.sin(al / 2)
            assert np.allclose(oracle_mod.quat_to_R(qa) @ a.astype(np.float64), b, atol=1e-6)
        q = _rand_q(rng)
        al = np.linspace(-2 * math.pi, 2 * math.pi, 200001)
        pts = np.outer(np.cos(al / 2), qb1) + np.outer(np.sin(al / 2), qb2)
        ang = np.arccos(np.clip(np.abs(pts @ q), -1, 1))
        j = int(np.argmin(ang))
        lo, hi = al[max(j - 1, 0)], al[min(j + 1, len(al) - 1)]
        f = lambda x: math.acos(min(1.0, abs((qb1 * math.cos(x / 2) + qb2 * math.sin(x / 2)) @ q)))
        g = (math.sqrt(5) - 1) / 2
        for _ in range(200):
            c1, c2 = hi - g * (hi - lo), lo + g * (hi - lo)
            if f(c1) < f(c2):
                hi = c2
            else:
                lo = c1
        dmin = f((lo + hi) / 2)
        v = oracle_mod.quad(oracle_mod.pair_S(a, b), q)
        assert abs(math.asin(math.sqrt(max(v, 0.0))) - dmin) < 2e-6


# --------------------------------------------------------------------------
# 2-4. grid, radius, threshold
# --------------------------------------------------------------------------

def test_level_cell_counts_match_lattice_count(oracle_mod):
    with open(os.path.join(HERE, "golden", "level_cell_counts.txt")) as f:
        rows = [tuple(int(x) for x in l.split()) for l in f if l.strip() and not l.startswith("#")]
    for n, cnt in rows:
        if n > 64:
            continue
        idx = oracle_mod.level_cells(n)
        assert len(idx) == cnt
        assert np.all(np.diff(idx) > 0)


def test_tau_closed_form(oracle_mod):
    """tau(chord) = sin^2(delta + 2 asin(chord/2)), and 1 once delta + r >= pi/2."""
    rng = np.random.default_rng(8)
    for _ in range(2000):
        d = rng.uniform(1e-4, 0.5)
        ch = rng.uniform(0, 2.2)
        r = 2 * math.asin(min(1.0, ch / 2))
        want = 1.0 if d + r >= math.pi / 2 else math.sin(d + r) ** 2
        got = oracle_mod.tau(d, ch)
        if abs(d + r - math.pi / 2) > 1e-9:
            assert abs(got - want) < 1e-14


def test_cell_radius_covers_cell(oracle_mod):
    """Every hemisphere point whose vector part lies in (box cap ball) is within
    r_cell = 2 asin(chord/2) of q_cell on S^3 (sampled densely, incl. corners)."""
    rng = np.random.default_rng(9)
    for n in (2, 4, 8, 32):
        h = 2.0 / n
        cells = oracle_mod.level_cells(n)
        pick = cells if len(cells) <= 64 else rng.choice(cells, 64, replace=False)
        for idx in pick:
            ix, iy, iz = idx % n, (idx // n) % n, idx // (n * n)
            q, chord = oracle_mod.cell_geom(n, ix, iy, iz)
            assert abs(np.linalg.norm(q) - 1) < 1e-12 and q[0] >= 0
            r = 2 * math.asin(min(1.0, chord / 2))
            lo = np.array([-1 + ix * h, -1 + iy * h, -1 + iz * h])
            pts = lo + h * rng.uniform(0, 1, size=(4000, 3))
            corners = lo + h * np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float)
            pts = np.vstack([pts, corners])
            nr = np.linalg.norm(pts, axis=1)
            pts = pts[nr <= 1.0]
            if len(pts) == 0:
                continue
            w = np.sqrt(np.maximum(0.0, 1 - np.sum(pts * pts, axis=1)))
            qp = np.hstack([w[:, None], pts])
            ang = 2 * np.arcsin(np.clip(np.linalg.norm(qp - q, axis=1) / 2, 0, 1))
            assert ang.max() <= r + 1e-12


def test_cell_exists_matches_box_ball_test(oracle_mod):
    for n in (3, 5, 8):
        h = 2.0 / n
        for ix in range(n):
            for iy in range(n):
                for iz in range(n):
                    lo = np.array([-1 + ix * h, -1 + iy * h, -1 + iz * h])
                    closest = np.clip(0.0, lo, lo + h)
                    want = float(closest @ closest) <= 1.0
                    assert oracle_mod.cell_exists(n, ix, iy, iz) == want


# --------------------------------------------------------------------------
# 5. vote
# --------------------------------------------------------------------------

def test_vote_counts_are_brute_force_and_conservative(oracle_mod):
    """Tiny grids, N <= 16: (i) counts equal an independent numpy evaluation of
    |b - R(q_cell) a|^2/4 <= sin^2(delta + r); (ii) every pair whose circle passes
    within delta of a densely sampled point of the cell is a voter."""
    rng = np.random.default_rng(10)
    for n in (4, 6, 8):
        p = synth.make_problem(16, rho=0.5, sigma=0.01, delta=0.08, seed=11 + n)
        cells = oracle_mod.level_cells(n)
        cnt, amb, tau_ = oracle_mod.vote_cells(p.a, p.b, p.delta, n, cells)
        h = 2.0 / n
        a64, b64 = p.a.astype(np.float64), p.b.astype(np.float64)
        cterm = (np.sum(a64 * a64, 1) + np.sum(b64 * b64, 1) - 2) / 4
        for c, idx in enumerate(cells):
            ix, iy, iz = idx % n, (idx // n) % n, idx // (n * n)
            q, chord = oracle_mod.cell_geom(n, ix, iy, iz)
            R = synth.rodrigues(q[1:] if np.linalg.norm(q[1:]) > 0 else np.array([1.0, 0, 0]),
                                2 * math.atan2(np.linalg.norm(q[1:]), q[0]))
            v = np.sum((b64 - a64 @ R.T) ** 2, axis=1) / 4 - cterm
            r = 2 * math.asin(min(1.0, chord / 2))
            t = 1.0 if p.delta + r >= math.pi / 2 else math.sin(p.delta + r) ** 2
            assert abs(t - tau_[c]) < 1e-14
            decided = np.abs(v - t) > 1e-9
            assert np.sum((v <= t) & decided) <= cnt[c] <= np.sum((v <= t) | ~decided)
            # conservativeness on sampled points of the cell
            lo = np.array([-1 + ix * h, -1 + iy * h, -1 + iz * h])
            pts = lo + h * rng.uniform(0, 1, size=(300, 3))
            pts = pts[np.linalg.norm(pts, axis=1) <= 1]
            if len(pts) == 0:
                continue
            qp = np.hstack([np.sqrt(np.maximum(0, 1 - np.sum(pts * pts, 1)))[:, None], pts])
            voters = 0
            for i in range(p.n):
                S = oracle_mod.pair_S(p.a[i], p.b[i])
                d = np.arcsin(np.sqrt(np.clip(np.einsum("kj,jl,kl->k", qp, S, qp), 0, 1)))
                if d.min() <= p.delta:
                    assert oracle_mod.quad(S, q) <= t + 1e-12
                voters += oracle_mod.quad(S, q) <= t
            assert voters == cnt[c]


def test_noise_free_inliers_vote_for_true_cell_at_every_level(oracle_mod):
    p = synth.make_problem(400, rho=0.7, sigma=0.0, delta=0.01, seed=12)
    inl = ~p.outlier
    for n in (8, 16, 32, 64, 128, 256):
        idx = oracle_mod.cell_of_point(n, p.q_true[1:])
        ix, iy, iz = idx % n, (idx // n) % n, idx // (n * n)
        assert oracle_mod.cell_exists(n, ix, iy, iz)
        cnt_in, _, _ = oracle_mod.vote_cells(p.a[inl], p.b[inl], p.delta, n, [idx])
        assert cnt_in[0] == inl.sum()


def test_pure_outlier_counts_are_binomial(oracle_mod):
    """For b independent of a, q^T S q ~ Uniform[0, 1] (Archimedes), so a cell's
    count is Binomial(N, tau): standardised counts have mean ~0, variance ~1."""
    rng = np.random.default_rng(13)
    N = 4000
    a = _unit(rng, N)
    b = _unit(rng, N)
    cells = oracle_mod.level_cells(8)
    cnt, _, tau_ = oracle_mod.vote_cells(a, b, 0.05, 8, cells, nthreads=4)
    z = (cnt - N * tau_) / np.sqrt(N * tau_ * (1 - tau_))
    assert abs(z.mean()) < 4 / math.sqrt(len(z)) + 0.15
    assert 0.5 < z.var() < 1.6


# --------------------------------------------------------------------------
# 6-7. rank and children
# --------------------------------------------------------------------------

def test_rank_fixtures(oracle_mod):
    count = np.array([10, 12, 12, 9, 12], np.int32)
    tau_ = np.array([0.0, 0.01, 0.01, 0.0, 0.02])
    idx = np.array([5, 9, 3, 1, 7], np.int64)
    pos, sc = oracle_mod.rank(count, tau_, idx, n_pairs=100, rank_mode=1, k=5)
    assert list(idx[pos]) == [3, 7, 9, 5, 1]          # RAW: ties by idx asc
    pos, sc = oracle_mod.rank(count, tau_, idx, n_pairs=100, rank_mode=0, k=3)
    # EXCESS: 10-0=10, 12-1=11 (idx 9), 12-1=11 (idx 3), 9, 12-2=10 (idx 7)
    assert list(idx[pos]) == [3, 9, 5]
    assert np.allclose(sc, [11, 11, 10])
    pos, _ = oracle_mod.rank(count, tau_, idx, n_pairs=100, rank_mode=0, k=50)
    assert len(pos) == 5


def test_children_partition_parent(oracle_mod):
    """The oracle's level-l+1 table is exactly the ball-meeting octants of the
    kept level-l cells: check via a traced 2-level solve."""
    p = synth.make_problem(300, rho=0.8, sigma=0.01, delta=0.05, seed=14)
    r = oracle_mod.solve(p.a, p.b, p.delta, grid_n=8, levels=2, top_k=4)
    for lev in range(2):
        n = 8 << lev
        kids = []
        for pidx in r.levels[lev]["topk_idx"]:
            ix, iy, iz = pidx % n, (pidx // n) % n, pidx // (n * n)
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        cx, cy, cz = 2 * ix + dx, 2 * iy + dy, 2 * iz + dz
                        if oracle_mod.cell_exists(2 * n, cx, cy, cz):
                            kids.append((cz * 2 * n + cy) * 2 * n + cx)
        assert sorted(kids) == sorted(r.levels[lev + 1]["idx"].tolist())


# --------------------------------------------------------------------------
# 8. fit
# --------------------------------------------------------------------------

def test_jacobi_matches_eigh(oracle_mod):
    rng = np.random.default_rng(15)
    for _ in range(200):
        X = rng.standard_normal((4, 4))
        A = X @ X.T if rng.uniform() < 0.5 else X + X.T
        ev, V = oracle_mod.jacobi4(A)
        ev_np, V_np = np.linalg.eigh(A)
        assert np.allclose(ev, ev_np, atol=1e-12 * max(1, np.abs(ev_np).max()))
        assert np.allclose(V.T @ V, np.eye(4), atol=1e-12)
        assert np.allclose(A @ V, V * ev, atol=1e-11 * max(1, np.abs(ev_np).max()))


def _svd_rotation(a, b):
    """Sec. 2.1 closed form: B = sum y x^T = U S V^T, R = U diag(1,1,det(U V^T)) V^T."""
    B = b.T @ a
    U, _, Vt = np.linalg.svd(B)
    D = np.diag([1.0, 1.0, np.linalg.det(U @ Vt)])
    return U @ D @ Vt


def _rot_angle(R1, R2):
    c = (np.trace(R1.T @ R2) - 1) / 2
    s = np.linalg.norm([R1.T @ R2 - (R1.T @ R2).T]) / (2 * math.sqrt(2))
    return math.atan2(s, c)


def test_fit_equals_svd_closed_form(oracle_mod):
    """The oracle's fit on an outlier-free problem (all pairs are inliers at
    delta = pi/4) equals the SVD method on the same pairs (the paper reports the
    two closed forms agree up to round-off, Sec. 5.2)."""
    for seed in range(5):
        p = synth.make_problem(500, rho=0.0, sigma=0.05, delta=0.7, seed=20 + seed)
        r = oracle_mod.solve(p.a, p.b, p.delta, grid_n=4, levels=0, refit_iters=8)
        assert r.status == 0
        a64, b64 = p.a.astype(np.float64), p.b.astype(np.float64)
        # refit with sin^2(0.7) keeps every pair: residual angles are ~0.05
        assert r.inliers == p.n
        R_svd = _svd_rotation(a64, b64)
        assert abs(_rot_angle(r.R, R_svd)) < 1e-9


def test_noise_free_fit_recovers_truth(oracle_mod):
    p = synth.make_problem(2000, rho=0.5, sigma=0.0, delta=0.02, seed=30)
    r = oracle_mod.solve(p.a, p.b, p.delta, grid_n=16, levels=2)
    qe = r.q
    ang = 2 * math.acos(min(1.0, abs(qe @ p.q_true)))
    assert ang < 1e-6
    assert r.inliers >= (~p.outlier).sum()


def test_degenerate_fit_returns_cell_centre(oracle_mod):
    rng = np.random.default_rng(31)
    a = _unit(rng, 5)
    b = _unit(rng, 5)
    r = oracle_mod.solve(a, b, 1e-4, grid_n=8, levels=0)
    if r.inliers < 2:
        assert r.status == -6
        n = 8
        ix, iy, iz = r.best_cell % n, (r.best_cell // n) % n, r.best_cell // (n * n)
        qc, _ = oracle_mod.cell_geom(n, ix, iy, iz)
        assert np.allclose(r.q, oracle_mod.canonical(qc))


def test_canonical_sign(oracle_mod):
    assert np.allclose(oracle_mod.canonical([-0.5, 0.5, -0.5, 0.5]), [0.5, -0.5, 0.5, -0.5])
    assert np.allclose(oracle_mod.canonical([0.0, -1.0, 0.0, 0.0]), [0.0, 1.0, 0.0, 0.0])
    assert np.allclose(oracle_mod.canonical([0.0, 0.0, 0.6, -0.8]), [0.0, 0.0, 0.6, -0.8])


def test_incompatible_pairs_have_no_common_point(oracle_mod):
    """App. E: two pairs related by rotations about the same axis with different
    angles have circles that do not meet; no q makes both vote values ~0."""
    k = np.array([0.0, 0.0, 1.0])
    a1 = np.array([1.0, 0.0, 0.0])
    a2 = np.array([0.0, 1.0, 0.0])
    b1 = synth.rodrigues(k, 0.3) @ a1
    b2 = synth.rodrigues(k, 1.1) @ a2
    S1 = oracle_mod.pair_S(a1.astype(np.float32), b1.astype(np.float32))
    S2 = oracle_mod.pair_S(a2.astype(np.float32), b2.astype(np.float32))
    ev = np.linalg.eigvalsh(S1 + S2)
    assert ev[0] > 1e-3   # min over unit q of q^T (S1+S2) q is bounded away from 0


def _appD_A(a32, b32):
    """App. D's A for one pair (written out here): A q = 0 on the pair's circle."""
    a64, b64 = a32.astype(np.float64), b32.astype(np.float64)
    d, p = a64 - b64, a64 + b64
    A = np.zeros((4, 4))
    A[0, 1:] = d
    A[1:, 0] = -d
    A[1:, 1:] = [[0, -p[2], p[1]], [p[2], 0, -p[0]], [-p[1], p[0], 0]]
    return A, (a64 @ a64 + b64 @ b64 - 2) / 4


def test_refit_converges_to_a_fixed_point(oracle_mod):
    """The refit rule (reading C9): when the refit stops because the inlier set
    repeats, the returned q is a fixed point -- the smallest eigenvector of
    sum_{i in I(q)} S_i with I(q) = {i : q^T S_i q <= sin^2(delta)} -- and the
    reported inlier count is |I(q)|.  S_i = A_i^T A_i / 4 - c_i I from App. D,
    evaluated here in numpy (eigh), independently of the oracle."""
    checked = 0
    for seed in range(6):
        p = synth.make_problem(800, rho=0.7, sigma=0.01, delta=0.03, seed=700 + seed)
        delta = float(np.float32(p.delta))
        r = oracle_mod.solve(p.a, p.b, delta, grid_n=16, levels=2, refit_iters=8, trace=False)
        if r.status != 0 or r.refits >= 8:
            continue  # stopped by the iteration cap, not by a repeated set
        As = [_appD_A(p.a[i], p.b[i]) for i in range(p.n)]
        v = np.array([np.sum((A @ r.q) ** 2) / 4 - c for A, c in As])
        thr = np.sin(delta) ** 2
        near = np.abs(v - thr) < 1e-12
        inl = v <= thr
        assert abs(inl.sum() - r.inliers) <= near.sum()
        if near.any():
            continue
        Ssum = sum(A.T @ A / 4 - c * np.eye(4) for (A, c), k in zip(As, inl) if k)
        w, V = np.linalg.eigh(Ssum)
        e = V[:, 0]
        assert w[1] - w[0] > 1e-9 * abs(w).max()
        assert min(np.linalg.norm(e - r.q), np.linalg.norm(e + r.q)) < 1e-9
        checked += 1
    assert checked >= 3


def test_refit_each_step_follows_the_rule(oracle_mod):
    """Every refit step (reading C9), including a refit stopped by the iteration
    cap: the fit from a cell with cap T returns the T-th iterate, so for each T
    up to the step where the inlier set repeats, q_T is the smallest eigenvector
    of sum S_i over I(q_{T-1}) = {i : q_{T-1}^T S_i q_{T-1} <= sin^2(delta)} and
    the reported inlier count is |I(q_{T-1})|, with S_i from App. D and the
    eigenvector from numpy eigh.  Past that step the iterate no longer moves."""
    steps = 0
    for seed in (900, 902, 910):
        p = synth.make_problem(1500, rho=0.8, sigma=0.03, delta=0.04, seed=seed)
        delta = float(np.float32(p.delta))
        cell = oracle_mod.solve(p.a, p.b, delta, grid_n=24, levels=0, refit_iters=0, trace=False).best_cell
        rs = [oracle_mod.fit_cell(p.a, p.b, delta, 24, cell, refit_iters=T) for T in range(8)]
        As = [_appD_A(p.a[i], p.b[i]) for i in range(p.n)]
        Ss = np.array([A.T @ A / 4 - c * np.eye(4) for A, c in As])
        thr = np.sin(delta) ** 2
        for T in range(1, 8):
            prev, cur = rs[T - 1], rs[T]
            assert cur.status == 0
            if cur.refits < T:  # the set repeated: the iterate stays
                assert cur.refits == prev.refits and np.array_equal(cur.q, prev.q)
                continue
            assert cur.refits == T
            v = np.einsum("j,ijk,k->i", prev.q, Ss, prev.q)
            assert not (np.abs(v - thr) < 1e-12).any()
            inl = v <= thr
            assert inl.sum() == cur.inliers
            w, V = np.linalg.eigh(Ss[inl].sum(0))
            assert w[1] - w[0] > 1e-9 * abs(w).max()
            e = V[:, 0]
            assert min(np.linalg.norm(e - cur.q), np.linalg.norm(e + cur.q)) < 1e-9
            steps += 1
    assert steps >= 9
