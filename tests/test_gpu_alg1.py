"""GPU parity of Alg. 1 (Sec. 4.3.2) through the C ABI against the FP64 oracle.

The bar is bit-exact: the library decides every sample's cell as the IEEE
double evaluation of the formulas does (FP32 first, FP64 again near a cell
boundary or near q3 = 0), so the whole n^3 accumulator, the winner, its count
and the number of samples cast equal the oracle's, and so does the rotation
(the same IEEE operations on the same cell centre).  The counter-wrap cases
also check the vote path: the return-less vote, then the vote with the wrap
record exactly when a cell reached 65536 votes, or the recording vote alone
after a problem with wraps.
"""
import numpy as np
import pytest

from paper_2506_11547_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

from paper_2506_11547_gb300 import rot_vote as rv  # noqa: E402


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def edge_pairs():
    """Pairs that exercise the special cases: axis-aligned a = b (samples on
    cell boundaries: p_1 = p_2 = 0 exactly), a = -b (w = 0: no circle), and
    near-antipodal pairs with |a| slightly above 1, whose basis norms are far
    from 1 (every sample on the FP64 path).  Along a diagonal, such a pair's
    samples reach |p| of about 3 and clamp onto the cube's edges, far outside
    the unit ball."""
    a, b = [], []
    for k in range(3):
        e = np.zeros(3, np.float32)
        e[k] = 1.0
        a += [e, e, e]
        b += [e, -e, np.roll(e, 1)]
    s = np.float32(1.0 + 4e-6)  # | |a|^2 - 1 | = 8e-6: valid
    for th in (3e-3, 4e-3, 6e-3):
        a.append(np.array([s, 0.0, 0.0], np.float32))
        b.append(np.array([-np.cos(th), np.sin(th), 0.0], np.float32))
        for ux, uy in ((1, 1), (1, -1)):
            u = np.array([ux, uy, 0.0]) / np.sqrt(2)
            a.append((s * u).astype(np.float32))
            c, sn = np.cos(th), np.sin(th)
            b.append(np.array([-(u[0] * c - u[1] * sn), -(u[0] * sn + u[1] * c), 0.0], np.float32))
    return np.array(a, np.float32), np.array(b, np.float32)


def with_edges(p):
    ea, eb = edge_pairs()
    return np.concatenate([p.a, ea]), np.concatenate([p.b, eb])


def run_both(a, b, J, side, device=True, acc_on_device=False):
    import oracle
    cells = side ** 3
    acc = torch.zeros(cells, dtype=torch.int32, device="cuda") if acc_on_device else np.zeros(cells, np.int32)
    with rv.Context() as ctx:
        r = ctx.alg1([((dev(a), dev(b)) if device else (a, b)) + (J, side, acc)])[0]
    acc = acc.cpu().numpy() if acc_on_device else acc
    o = oracle.alg1(a, b, J, side)
    return r, acc, o


def wrapped_words(acc):
    """Counter words (cells 2w, 2w + 1) holding a count of 65536 or more."""
    hot = np.nonzero(acc >= 65536)[0]
    return len(np.unique(hot // 2))


def box_distance(side):
    """Distance from the origin to each cell's box, in linear-index order."""
    h = 2.0 / side
    lo = -1 + np.arange(side) * h
    d = np.where(lo > 0, lo, np.where(lo + h < 0, -(lo + h), 0.0))
    return np.sqrt(d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2).reshape(-1)


def expected_vote_paths(acc, side):
    """Vote paths a fresh context may take.  Path 1 (the recording re-vote) is
    certain when a counter wrapped.  With n a multiple of 8 the return-less pass
    scans the cells within 1.01 of the origin (plus a margin of up to eight
    cells along x), so counts in cells beyond 1.0005 may also send a problem to
    path 1, and counts beyond that margin must."""
    if wrapped_words(acc):
        return {1}
    if side % 8:
        return {0}
    D, voted = box_distance(side), acc > 0
    if not (voted & (D > 1.0005)).any():
        return {0}
    if (voted & (D > 1.01 + 9 * 2.0 / side)).any():
        return {1}
    return {0, 1}


def check(r, acc, o):
    o_acc, o_bi, o_bc, o_q, o_cast = o
    assert r.status == rv.OK
    d = np.nonzero(acc != o_acc)[0]
    assert len(d) == 0, f"{len(d)} accumulator cells differ, e.g. {d[:5]}: {acc[d[:5]]} vs {o_acc[d[:5]]}"
    assert (r.best_cell, r.best_count, r.samples_cast) == (o_bi, o_bc, o_cast)
    assert np.array_equal(r.q, o_q), (r.q, o_q)
    # a word wraps exactly when one of its two cells holds 65536 or more votes;
    # a fresh context takes the return-less vote first and re-votes with the
    # wrap record when a counter wrapped or a count fell outside the scanned region
    assert r.wrapped_words == wrapped_words(o_acc)
    side = round(len(o_acc) ** (1 / 3))
    assert r.vote_path in expected_vote_paths(o_acc, side), (r.vote_path, expected_vote_paths(o_acc, side))
    import oracle
    assert np.allclose(r.R, oracle.quat_to_R(o_q), rtol=0, atol=1e-15)


def test_alg1_small_with_edge_cases():
    p = synth.make_problem(1000, 0.9, 0.01, 0.03, seed=2101)
    a, b = with_edges(p)
    r, acc, o = run_both(a, b, 180, 64)
    check(r, acc, o)
    # the axis-aligned samples sit on cell boundaries and the near-antipodal
    # pairs take the FP64 path for every sample
    assert r.rechecked >= 3 * 180
    # the a = -b pairs cast nothing
    assert r.samples_cast == 180 * (len(a) - 3)


@pytest.mark.parametrize("J,side,device", [(1, 8, True), (7, 37, False), (256, 90, True), (257, 360, False),
                                           (540, 128, True), (180, 2, True)])
def test_alg1_samples_and_sides(J, side, device):
    p = synth.make_problem(3000, 0.8, 0.01, 0.03, seed=2200 + J + side)
    a, b = with_edges(p)
    r, acc, o = run_both(a, b, J, side, device=device, acc_on_device=(J % 2 == 0))
    check(r, acc, o)


def test_alg1_paper_default_n1e5():
    """The paper's default resolution (1/180 -> a 360^3 accumulator) and J = 180
    on 1e5 pairs with 99% outliers."""
    p = synth.make_problem(100000, 0.99, 0.01, 0.03, seed=2301)
    r, acc, o = run_both(p.a, p.b, 180, 360)
    check(r, acc, o)
    # FP64 re-evaluations are the rare boundary cases
    assert r.rechecked < 0.05 * r.samples_cast


def test_alg1_n1e6():
    """1e6 pairs, 99% outliers (the paper's large-scale claim), full accumulator."""
    p = synth.make_problem(1000000, 0.99, 0.005, 0.03, seed=2302)
    r, acc, o = run_both(p.a, p.b, 180, 360)
    check(r, acc, o)


def test_alg1_batch_equals_single_calls():
    ps = [synth.make_problem(n, 0.9, 0.01, 0.03, seed=2400 + n) for n in (50, 777, 4096)]
    with rv.Context() as ctx:
        many = ctx.alg1([(dev(p.a), dev(p.b), 90, 48) for p in ps])
        one = [ctx.alg1([(dev(p.a), dev(p.b), 90, 48)])[0] for p in ps]
    for x, y in zip(many, one):
        assert (x.best_cell, x.best_count, x.samples_cast) == (y.best_cell, y.best_count, y.samples_cast)
        assert np.array_equal(x.q, y.q)


def test_alg1_invalid_inputs_and_arguments():
    p = synth.make_problem(500, 0.5, 0.01, 0.03, seed=2500)
    bad = p.a.copy()
    bad[7] *= 1.01  # not unit
    nan = p.a.copy()
    nan[3, 1] = np.nan
    with rv.Context() as ctx:
        r = ctx.alg1([(dev(bad), dev(p.b)), (dev(nan), dev(p.b)), (dev(p.a), dev(p.b), 0, 1),
                      (dev(p.a), dev(p.b), 70000, 16), (dev(p.a[:1]), dev(p.b[:1])), (dev(p.a), dev(p.b), 0, 24)])
    assert [x.status for x in r[:5]] == [rv.EINVAL] * 5
    assert r[5].status == rv.OK and r[5].samples_cast == 180 * 500  # J = 0 selects 180


def test_alg1_noise_free_winner_is_the_true_rotation_cell():
    """Noise-free inliers: every circle passes through the true rotation, so
    the winner's centre is within one cell of it (chart distortion <= 2)."""
    from tests._util import quat_angle
    p = synth.make_problem(2000, 0.5, 0.0, 0.03, seed=2600)
    side = 180
    with rv.Context() as ctx:
        r = ctx.alg1([(dev(p.a), dev(p.b), 720, side)])[0]
    assert r.status == rv.OK
    # a cell of side 2/n in the chart spans at most 2 * sqrt(3) * (2/n) on S^3 (conformal factor <= 2)
    assert quat_angle(r.q, p.q_true) <= 2 * (2 * np.sqrt(3) * 2 / side)


# ---- multiple rotations (Sec. 4.4): peaks by greedy suppression ----

def run_peaks(a, b, J, side, M, theta, min_count=0):
    import oracle
    acc = np.zeros(side ** 3, np.int32)
    with rv.Context() as ctx:
        r = ctx.alg1([(dev(a), dev(b), J, side, acc)], peaks=M, nms_angle=theta, min_count=min_count)[0]
    theta32 = float(np.float32(theta))  # the ABI carries the angle as float32
    o_idx, o_cnt, o_q, o_T = oracle.alg1_peaks(acc, side, M, theta32, min_count=min_count,
                                               kmax=rv.ALG1_PEAK_CANDIDATES)
    return r, acc, (o_idx, o_cnt, o_q, o_T)


def check_peaks(r, o):
    o_idx, o_cnt, o_q, o_T = o
    assert r.status == rv.OK
    assert r.peak_threshold == o_T
    assert [p[0] for p in r.peaks] == list(o_idx)
    assert [p[1] for p in r.peaks] == list(o_cnt)
    for (_, _, q), oq in zip(r.peaks, o_q):
        assert np.array_equal(q, oq)


@pytest.mark.parametrize("M,theta,min_count,side", [(1, 0.1, 0, 120), (6, 0.15, 0, 120), (64, 0.05, 0, 120),
                                                    (9, 0.3, 40, 120), (12, 0.0, 0, 120), (6, 0.15, 0, 90)])
def test_alg1_peaks_multi_motion_scene(M, theta, min_count, side):
    """At side 120 the argmax after the return-less vote reads only the ball
    region's words; at side 90 (not a multiple of 8) it reads every word."""
    mp = synth.make_multi_problem(4, 800, sigma=0.01, outlier_frac=0.5, seed=2700 + M)
    r, acc, o = run_peaks(mp.a, mp.b, 540, side, M, theta, min_count)
    check_peaks(r, o)
    if M == 1:
        assert r.peaks[0][0] == r.best_cell and r.peaks[0][1] == r.best_count


def test_alg1_peaks_threshold_above_one():
    """1e5 pairs at the paper's resolution: more than 16384 cells are voted, so the
    candidate threshold T rises above 1, exactly as the oracle computes it."""
    p = synth.make_problem(100000, 0.99, 0.01, 0.03, seed=2801)
    r, acc, o = run_peaks(p.a, p.b, 180, 360, 9, 0.1)
    assert o[3] > 1
    check_peaks(r, o)


def test_alg1_peaks_recover_nine_motions():
    """The paper's multiple-rotation experiment shape: 9 motions x 3000 pairs, noise
    0.01, J = 540: the 9 highest peaks are the 9 rotations."""
    from tests._util import quat_angle
    mp = synth.make_multi_problem(9, 3000, sigma=0.01, seed=2802)
    r, acc, o = run_peaks(mp.a, mp.b, 540, 360, 9, 0.1)
    check_peaks(r, o)
    assert len(r.peaks) == 9
    for qt in mp.q_true:
        assert min(quat_angle(q, qt) for _, _, q in r.peaks) < 0.05


def test_alg1_peaks_argument_errors():
    p = synth.make_problem(300, 0.5, 0.01, 0.03, seed=2803)
    with rv.Context() as ctx:
        for kw in (dict(peaks=65, nms_angle=0.1), dict(peaks=3, nms_angle=-1.0), dict(peaks=3, nms_angle=float("nan")),
                   dict(peaks=3, nms_angle=0.1, min_count=-2)):
            r = ctx.alg1([(dev(p.a), dev(p.b), 90, 32)], **kw)[0]
            assert r.status == rv.EINVAL


# ---- the 16-bit counters: wraps of a word's low half, carries, wraps of the word ----

def _pairs_by_cell(side, J, n_try=4000, seed=2900):
    """Random pairs and the cell of their last sample (the oracle's cell function)."""
    import oracle
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n_try, 3))
    b = rng.standard_normal((n_try, 3))
    a = (a / np.linalg.norm(a, axis=1, keepdims=True)).astype(np.float32)
    b = (b / np.linalg.norm(b, axis=1, keepdims=True)).astype(np.float32)
    cs = oracle.alg1_table(J)
    cells = []
    for i in range(n_try):
        ok, q1, q2 = oracle.alg1_basis(a[i], b[i])
        cells.append(oracle.alg1_cell(q1, q2, cs[-1, 0], cs[-1, 1], side) if ok else -1)
    return a, b, np.array(cells)


@pytest.mark.parametrize("n_lo,n_hi", [(140000, 70000), (65535, 0), (65536, 1), (0, 65536), (131072, 65535)])
def test_alg1_counter_wraps(n_lo, n_hi):
    """n_lo copies of a pair whose second sample (alpha = 0: q_b1) lands in an even
    cell 2w and n_hi of one landing in 2w + 1, plus random pairs: counts of 65536
    and more wrap the 16-bit halves; the int32 accumulator, the winner and the peaks
    equal the oracle's."""
    side, J = 8, 2
    a, b, cells = _pairs_by_cell(side, J)
    pick = None
    for i in np.nonzero((cells >= 0) & (cells % 2 == 0))[0]:
        j = np.nonzero(cells == cells[i] + 1)[0]
        if len(j):
            pick = (i, j[0])
            break
    assert pick is not None
    i, j = pick
    A = np.concatenate([np.repeat(a[i:i + 1], n_lo, 0), np.repeat(a[j:j + 1], n_hi, 0), a[:1000]])
    B = np.concatenate([np.repeat(b[i:i + 1], n_lo, 0), np.repeat(b[j:j + 1], n_hi, 0), b[:1000]])
    r, acc, o = run_both(A, B, J, side)
    check(r, acc, o)
    assert acc[cells[i]] >= n_lo and acc[cells[i] + 1] >= n_hi
    rp, accp, op = run_peaks(A, B, J, side, 4, 0.3)
    check_peaks(rp, op)
    assert np.array_equal(accp, acc) and rp.wrapped_words == r.wrapped_words and rp.vote_path == r.vote_path


def test_alg1_vote_path_follows_the_previous_problem():
    """One context, problems with and without counter wraps in turn: the
    return-less vote first (re-voting when it wrapped), the recording vote
    alone after a problem with wraps; every accumulator equals the oracle's."""
    import oracle
    side, J = 8, 2
    a, b, cells = _pairs_by_cell(side, J)
    i = int(np.nonzero(cells >= 0)[0][0])
    hot_a = np.concatenate([np.repeat(a[i:i + 1], 70000, 0), a[:500]])
    hot_b = np.concatenate([np.repeat(b[i:i + 1], 70000, 0), b[:500]])
    # 40000 random pairs: 80000 samples (enough to wrap a counter) over 512 cells, none near 65536
    rng = np.random.default_rng(2910)
    cold_a, cold_b = (rng.standard_normal((40000, 3)) for _ in range(2))
    cold_a = (cold_a / np.linalg.norm(cold_a, axis=1, keepdims=True)).astype(np.float32)
    cold_b = (cold_b / np.linalg.norm(cold_b, axis=1, keepdims=True)).astype(np.float32)
    seq = [(cold_a, cold_b, 0), (hot_a, hot_b, 1), (hot_a, hot_b, 2), (cold_a, cold_b, 2), (cold_a, cold_b, 0)]
    with rv.Context() as ctx:
        for A, B, path in seq:
            acc = np.zeros(side ** 3, np.int32)
            r = ctx.alg1([(dev(A), dev(B), J, side, acc)])[0]
            o = oracle.alg1(A, B, J, side)
            assert r.vote_path == path
            assert r.wrapped_words == wrapped_words(o[0])
            assert np.array_equal(acc, o[0])
            assert (r.best_cell, r.best_count, r.samples_cast) == (o[1], o[2], o[4])
            assert np.array_equal(r.q, o[3])


def test_alg1_zeroing_after_stray_counts_and_side_changes():
    """One context: a problem whose FP64-only pairs count far outside the ball
    (re-voted on path 1, leaving counts outside the region), then problems of
    the same and of other sides, which must start from a fully zeroed
    accumulator whenever the words outside the region are not known to be zero."""
    import oracle
    p = synth.make_problem(4000, 0.9, 0.01, 0.03, seed=2920)
    ea, eb = with_edges(p)
    seq = [(ea, eb, 64), (p.a, p.b, 64), (p.a, p.b, 64), (p.a, p.b, 48), (p.a, p.b, 64), (ea, eb, 48),
           (p.a, p.b, 48)]
    with rv.Context() as ctx:
        for k, (A, B, side) in enumerate(seq):
            acc = np.zeros(side ** 3, np.int32)
            r = ctx.alg1([(dev(A), dev(B), 180, side, acc)])[0]
            o = oracle.alg1(A, B, 180, side)
            assert np.array_equal(acc, o[0]), k
            assert (r.best_cell, r.best_count, r.samples_cast) == (o[1], o[2], o[4]), k
            assert np.array_equal(r.q, o[3]), k
            if k == 0:
                # the near-antipodal non-unit pairs count outside the region
                assert (o[0][box_distance(side) > 1.2] > 0).any() and r.vote_path == 1
