"""rot_vote_count_cells_static (the entry point that allocates no device
memory), called through the C ABI, against the counts of a context's solve
(rot_vote_solve in the FP32 form, level-0 trace) on the same inputs and
against the oracle's counts of the same cells.  All three count exactly, so
the counts must be identical, call after call: the cases run back to back on
the shared static scratch, larger problem after smaller and smaller after
larger, up to both size limits."""
import os

import numpy as np
import pytest

from paper_2506_11547_gb300 import synth
from tests._util import f32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

from paper_2506_11547_gb300 import rot_vote as rv  # noqa: E402


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _solve_level0(p, grid_n):
    with rv.Context(grid_n=grid_n, levels=0, precision="fp32", keep_trace=1) as ctx:
        r = ctx.solve([(_dev(p.a), _dev(p.b), p.delta)])[0]
        idx, cnt, _ = ctx.level_trace(0, 0)
    assert r.status in (rv.OK, rv.EDEGENERATE)  # identical pairs make the fit degenerate
    return idx, cnt


def _static_counts(p, grid_n, idx):
    counts = torch.full((len(idx),), -7, dtype=torch.int32, device="cuda")
    rc = rv.count_cells_static(_dev(p.a), _dev(p.b), p.delta, grid_n, _dev(idx), counts)
    torch.cuda.synchronize()
    return rc, counts.cpu().numpy()


def _at_threshold(n, grid_n, delta, seed):
    """n copies of one pair whose test against one cell of the grid_n level lies on that
    cell's threshold (q_c^T S q_c = tau_c up to float32 rounding): b is R(q_c) a turned by
    2 asin(sqrt(tau_c)) about an axis normal to it.  All n tests of that cell fall within the
    FP64 band, more than the entry point's FP64 queue holds, so the resolution pass must
    recount the cell.  The cell's centre and threshold come from the oracle."""
    import oracle
    rng = np.random.default_rng(seed)
    cells = oracle.level_cells(grid_n)
    idx = int(cells[len(cells) // 3])
    ix, iy, iz = idx % grid_n, (idx // grid_n) % grid_n, idx // (grid_n * grid_n)
    q, chord = oracle.cell_geom(grid_n, ix, iy, iz)
    tau = oracle.tau(f32(delta), chord)
    a = rng.standard_normal(3)
    a /= np.linalg.norm(a)
    ra = oracle.quat_to_R(q) @ a
    axis = np.cross(ra, rng.standard_normal(3))
    b = synth.rodrigues(axis, 2.0 * np.arcsin(np.sqrt(tau))) @ ra
    pr = synth.make_problem(n, rho=0.0, sigma=0.0, delta=delta, seed=seed)
    pr.a[:] = np.float32(a)
    pr.b[:] = np.float32(b / np.linalg.norm(b))
    return pr


def test_static_counts_equal_solve_counts_call_after_call():
    cases = [
        (synth.make_problem(5000, rho=0.9, sigma=0.01, delta=0.03, seed=901), 16, None),
        (synth.make_problem(rv.STATIC_MAX_PAIRS, rho=0.5, sigma=0.01, delta=0.05, seed=902), 16, None),
        (synth.make_problem(3001, rho=0.8, sigma=0.01, delta=0.02, seed=903), 32, rv.STATIC_MAX_CELLS),
        (synth.make_problem(129, rho=0.3, sigma=0.01, delta=0.04, seed=904), 8, None),
        (_at_threshold(rv.STATIC_MAX_PAIRS, 32, 0.05, seed=908), 32, rv.STATIC_MAX_CELLS),
    ]
    import oracle
    for p, g, keep in cases:
        idx, cnt = _solve_level0(p, g)
        if keep is not None:
            idx, cnt = idx[:keep], cnt[:keep]
        oc, _, _ = oracle.vote_cells(p.a, p.b, f32(p.delta), g, idx, nthreads=max(1, os.cpu_count() or 1))
        assert np.array_equal(cnt, oc)
        rc, got = _static_counts(p, g, idx)
        assert rc == rv.OK
        assert np.array_equal(got, cnt)
        rc, again = _static_counts(p, g, idx)  # the same call twice in a row
        assert rc == rv.OK
        assert np.array_equal(again, cnt)


def test_static_rejects_sizes_above_its_limits():
    p = synth.make_problem(rv.STATIC_MAX_PAIRS + 1, rho=0.5, sigma=0.01, delta=0.05, seed=905)
    idx = np.arange(4, dtype=np.int64)
    rc, _ = _static_counts(p, 16, idx)
    assert rc == rv.ETOOLARGE
    q = synth.make_problem(100, rho=0.5, sigma=0.01, delta=0.05, seed=906)
    rc, _ = _static_counts(q, 64, np.zeros(rv.STATIC_MAX_CELLS + 1, dtype=np.int64))
    assert rc == rv.ETOOLARGE


def test_static_rejects_a_cell_outside_the_level_table():
    p = synth.make_problem(500, rho=0.5, sigma=0.01, delta=0.05, seed=907)
    idx, cnt = _solve_level0(p, 8)
    bad = np.concatenate([idx[:5], np.array([0], dtype=np.int64)])  # cell (0,0,0): its box misses the ball
    rc, _ = _static_counts(p, 8, bad)
    assert rc == rv.EINVAL
    rc, got = _static_counts(p, 8, idx)  # and the next call is unaffected
    assert rc == rv.OK
    assert np.array_equal(got, cnt)
