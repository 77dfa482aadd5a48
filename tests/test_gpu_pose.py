"""GPU parity of the rigid-pose front end (Sec. 4.5) through the C ABI against
the FP64 oracle.

- Kept pairs: bit-exact. Same pairs, same order, same float32 unit vectors:
  each length decision equals the IEEE double definition.
- Rotation: the rotation-vote parity bar on those identical inputs:
  - the same winning cell and the same count;
  - the same number of ambiguous tests;
  - 1e-4 rad.
- Translation: each side votes with its own rotation. Where the two rotations
  agree to 1e-12, the winning cell and its count agree exactly, up to a
  candidate within 1e-9 of a cell boundary; otherwise within one cell.
"""
import numpy as np
import pytest

from paper_2506_11547_gb300 import synth
from tests._util import f32, quat_angle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

from paper_2506_11547_gb300 import rot_vote as rv  # noqa: E402

MU, DELTA, GRID, LEVELS = 0.04, 0.03, 32, 2


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_both(x, y, mu=MU, lmin=0.0, device=True):
    import oracle
    oa, ob = oracle.pose_pairs(x, y, f32(mu), f32(lmin))
    cap = len(oa) + 8
    ga, gb = np.zeros((cap, 3), np.float32), np.zeros((cap, 3), np.float32)
    with rv.Context(grid_n=GRID, levels=LEVELS) as ctx:
        r = ctx.pose(dev(x) if device else x, dev(y) if device else y, mu, DELTA, min_length=lmin,
                     pairs_out=(ga, gb))
    o_rot, o_t, o_cell, o_cnt, o_K = oracle.pose(x, y, f32(mu), f32(DELTA), GRID, LEVELS, lmin=f32(lmin), nthreads=16)
    return r, (ga, gb), (oa, ob), (o_rot, o_t, o_cell, o_cnt, o_K)


def check(r, g_pairs, o_pairs, o):
    o_rot, o_t, o_cell, o_cnt, o_K = o
    assert r.status == rv.OK
    assert r.pairs_kept == o_K == len(o_pairs[0])
    K = r.pairs_kept
    assert np.array_equal(g_pairs[0][:K], o_pairs[0]) and np.array_equal(g_pairs[1][:K], o_pairs[1])
    assert r.rot.best_cell == o_rot.best_cell
    assert r.rot.best_count == o_rot.best_count
    assert r.rot.ambiguous == o_rot.ambiguous
    assert quat_angle(r.rot.q, o_rot.q) < 1e-4
    assert r.rot.tests == o_rot.tests
    if quat_angle(r.rot.q, o_rot.q) < 1e-12:
        assert r.t_cell == o_cell and abs(r.t_count - o_cnt) <= 1 and np.array_equal(r.t, o_t)
    else:
        assert np.max(np.abs(r.t - o_t)) <= 0.025 + 1e-12


def test_pose_small_with_duplicates_and_min_length():
    p = synth.make_pose_problem(400, 0.5, 0.01, seed=3001)
    x, y = p.x.copy(), p.y.copy()
    x[9], y[9] = x[4], y[4]  # duplicated correspondence: |m| = |n| = 0
    for lmin in (0.0, 0.3):
        r, g, op, o = run_both(x, y, lmin=lmin)
        check(r, g, op, o)
        assert r.pairs_tested == 400 * 399 // 2


def test_pose_host_inputs_equal_device_inputs():
    p = synth.make_pose_problem(300, 0.4, 0.01, seed=3002)
    with rv.Context(grid_n=GRID, levels=LEVELS) as ctx:
        rh = ctx.pose(p.x, p.y, MU, DELTA)
        rd = ctx.pose(dev(p.x), dev(p.y), MU, DELTA)
    assert rh.pairs_kept == rd.pairs_kept and np.array_equal(rh.rot.q, rd.rot.q) and np.array_equal(rh.t, rd.t)


@pytest.mark.parametrize("n,rho", [(2, 0.0), (3, 0.0), (257, 0.3), (1000, 0.8)])
def test_pose_sizes(n, rho):
    p = synth.make_pose_problem(n, rho, 0.01, seed=3100 + n)
    r, g, op, o = run_both(p.x, p.y)
    if o[4] < 2:
        assert r.status == rv.EDEGENERATE and r.pairs_kept == o[4]
        return
    check(r, g, op, o)


def test_pose_paper_protocol_n5000():
    """The paper's default rigid setting (Sec. 5.4.1): N = 5000, 90% outliers,
    noise 0.01: 12.5M pairs checked; the pose is recovered."""
    p = synth.make_pose_problem(5000, 0.9, 0.01, seed=3003)
    r, g, op, o = run_both(p.x, p.y)
    check(r, g, op, o)
    assert quat_angle(r.rot.q, p.q_true) < 0.01
    assert np.linalg.norm(r.t - p.t_true) < 0.05


def test_pose_argument_and_input_errors():
    p = synth.make_pose_problem(100, 0.3, 0.01, seed=3004)
    bad = p.x.copy()
    bad[5, 2] = np.nan
    big = p.x.copy()
    big[3, 0] = 1e20
    with rv.Context(grid_n=GRID, levels=LEVELS) as ctx:
        assert ctx.pose(dev(bad), dev(p.y), MU, DELTA).status == rv.EINVAL
        assert ctx.pose(dev(big), dev(p.y), MU, DELTA).status == rv.EINVAL
        assert ctx.pose(dev(p.x[:1]), dev(p.y[:1]), MU, DELTA).status == rv.EINVAL
        assert ctx.pose(dev(p.x), dev(p.y), 0.0, DELTA).status == rv.EINVAL
        assert ctx.pose(dev(p.x), dev(p.y), MU, DELTA, t_cells=2000).status == rv.EINVAL
        assert ctx.pose(dev(p.x), dev(p.y), MU, DELTA).status == rv.OK
