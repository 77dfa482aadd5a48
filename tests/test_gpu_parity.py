"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Counts: every cell's count equals the oracle's, at every level (the tests
within 2e-6 of the threshold are decided by the FP64 evaluation, in the
oracle's order of operations).
Ranking: the kept cells equal the oracle's, in rank order.
Ambiguous tests (|v - tau| <= 1e-6 in FP64): the same total as the oracle's.
Rotation: within 1e-4 rad of the oracle's.
"""
import os

import numpy as np
import pytest

from paper_2506_11547_gb300 import synth
from tests._util import f32, quat_angle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

from paper_2506_11547_gb300 import rot_vote as rv  # noqa: E402

ROT_TOL = 1e-4
NTHREADS = max(1, os.cpu_count() or 1)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def check_counts(gpu_idx, gpu_cnt, lev):
    assert np.array_equal(gpu_idx, lev["idx"]), "level tables differ"
    bad = np.nonzero(gpu_cnt.astype(np.int64) != lev["count"].astype(np.int64))[0]
    assert len(bad) == 0, (f"{len(bad)} of {len(gpu_cnt)} cells differ, e.g. pos {bad[:5]}: "
                           f"gpu {gpu_cnt[bad[:5]]} oracle {lev['count'][bad[:5]]} amb {lev['amb'][bad[:5]]}")


def check_kept(gpu_kept, lev):
    assert np.array_equal(gpu_kept, lev["topk_idx"]), (gpu_kept, lev["topk_idx"])


def run_both(p, grid_n, levels, precision="fp32", top_k=16, rank_mode="excess", refit=8, device=True, shape=0,
             chart=0):
    import oracle
    a, b = (dev(p.a), dev(p.b)) if device else (p.a, p.b)
    with rv.Context(grid_n=grid_n, levels=levels, top_k=top_k, precision=precision, rank_mode=rank_mode,
                    refit_iters=refit if refit else -1, keep_trace=1, autotune=shape, chart=chart) as ctx:
        r = ctx.solve([(a, b, p.delta)])[0]
        tr = [ctx.level_trace(0, lev) for lev in range(levels + 1)]
    o = oracle.solve(p.a, p.b, f32(p.delta), grid_n=grid_n, levels=levels, top_k=top_k,
                     rank_mode=rv.RANK[rank_mode], refit_iters=refit, nthreads=NTHREADS, chart=chart)
    return r, tr, o


def assert_parity(p, r, tr, o, levels):
    for lev in range(levels + 1):
        idx, cnt, kept = tr[lev]
        check_counts(idx, cnt, o.levels[lev])
        check_kept(kept, o.levels[lev])
    assert r.status == o.status
    assert r.best_cell == o.best_cell
    assert r.best_count == o.best_count
    assert r.ambiguous == o.ambiguous, (r.ambiguous, o.ambiguous)
    assert r.resolved >= r.ambiguous
    assert quat_angle(r.q, o.q) < ROT_TOL
    assert r.tests == o.tests
    assert (r.inliers, r.refits) == (o.inliers, o.refits)
    assert r.q[0] >= 0


def test_small_workload_every_cell():
    p, g, L = synth.config_problem("small_n1e3_32")
    r, tr, o = run_both(p, g, L)
    assert_parity(p, r, tr, o, L)


def test_multilevel_every_level():
    p = synth.make_problem(3000, rho=0.9, sigma=0.01, delta=0.03, seed=77)
    r, tr, o = run_both(p, 16, 3)
    assert_parity(p, r, tr, o, 3)


FP32_SHAPES = [4, 8, 102, 104, 114, 124]  # scalar (cells per thread); packed f32x2 (100 + cells per thread, +10/+20 occupancy)


@pytest.mark.parametrize("shape", FP32_SHAPES)
def test_every_fp32_tile_shape(shape):
    p = synth.make_problem(3001, rho=0.9, sigma=0.01, delta=0.03, seed=78)
    r, tr, o = run_both(p, 16, 2, shape=shape)
    assert_parity(p, r, tr, o, 2)
    q = synth.make_problem(257, rho=0.5, sigma=0.01, delta=0.05, seed=79)  # ragged: padded pair tile
    r, tr, o = run_both(q, 8, 1, shape=shape)
    assert_parity(q, r, tr, o, 1)


def test_unknown_tile_shape_is_rejected():
    p = synth.make_problem(300, rho=0.5, sigma=0.01, delta=0.05, seed=80)
    with rv.Context(grid_n=8, levels=0, autotune=12) as ctx:  # 12 exists only for the tensor-core forms
        with pytest.raises(rv.RotVoteError) as e:
            ctx.solve([(dev(p.a), dev(p.b), p.delta)])
        assert e.value.code == rv.EINVAL


@pytest.mark.parametrize("n", [2, 3, 127, 128, 129, 257, 1000])
def test_ragged_sizes(n):
    p = synth.make_problem(n, rho=0.5, sigma=0.01, delta=0.05, seed=100 + n)
    r, tr, o = run_both(p, 8, 2)
    assert_parity(p, r, tr, o, 2)


@pytest.mark.parametrize("grid_n,levels,top_k,rank", [(2, 0, 1, "excess"), (4, 3, 1, "raw"), (8, 1, 64, "excess"),
                                                      (32, 2, 5, "raw")])
def test_grid_and_rank_options(grid_n, levels, top_k, rank):
    p = synth.make_problem(700, rho=0.8, sigma=0.02, delta=0.06, seed=grid_n * 10 + levels)
    r, tr, o = run_both(p, grid_n, levels, top_k=top_k, rank_mode=rank)
    assert_parity(p, r, tr, o, levels)


def test_no_refit_and_degenerate():
    p = synth.make_problem(500, rho=0.9, sigma=0.01, delta=0.03, seed=5)
    r, tr, o = run_both(p, 16, 1, refit=0)
    assert_parity(p, r, tr, o, 1)
    assert r.refits == 0
    # pure outliers and a tiny tolerance: the winner has < 2 voters -> degenerate
    q = synth.make_problem(50, rho=1.0, sigma=0.0, delta=1e-4, seed=6)
    r2, tr2, o2 = run_both(q, 4, 0)
    assert r2.status == o2.status
    if o2.status == rv.EDEGENERATE:
        assert quat_angle(r2.q, o2.q) < 1e-12


def test_host_inputs_equal_device_inputs():
    p = synth.make_problem(5000, rho=0.9, sigma=0.01, delta=0.03, seed=9)
    with rv.Context(grid_n=32, levels=2) as ctx:
        rh = ctx.solve([(p.a, p.b, p.delta)])[0]
        rd = ctx.solve([(dev(p.a), dev(p.b), p.delta)])[0]
    assert np.array_equal(rh.q, rd.q) and rh.best_count == rd.best_count and rh.inliers == rd.inliers


def test_batched_equals_alone_and_deterministic():
    probs = [synth.make_problem(n, rho=0.8, sigma=0.01, delta=d, seed=s)
             for n, d, s in ((50, 0.03, 1), (700, 0.02, 2), (4096, 0.05, 3), (129, 0.04, 4), (20000, 0.03, 5))]
    args = [(dev(p.a), dev(p.b), p.delta) for p in probs]
    with rv.Context(grid_n=32, levels=2) as ctx:
        batch = ctx.solve(args)
        batch2 = ctx.solve(args)
        alone = [ctx.solve([x])[0] for x in args]
    for rb, rb2, ra in zip(batch, batch2, alone):
        for x in (rb2, ra):
            assert np.array_equal(rb.q, x.q)
            assert (rb.best_count, rb.inliers, rb.best_cell, rb.tests, rb.rechecked) == \
                   (x.best_count, x.inliers, x.best_cell, x.tests, x.rechecked)


def test_large_problems_fitted_together_equal_alone():
    """Three problems above 32768 pairs, fitted together in whole-GPU passes
    (their slices in one flat list), and two small ones in the same call: each
    result equals the problem solved alone, bit for bit, and the large ones
    match the oracle (same winning cell, rotation within 1e-4 rad)."""
    import oracle
    probs = [synth.make_problem(n, rho=0.9, sigma=0.01, delta=0.03, seed=s)
             for n, s in ((40000, 21), (50, 22), (70000, 23), (5000, 24), (33000, 25))]
    args = [(dev(p.a), dev(p.b), p.delta) for p in probs]
    with rv.Context(grid_n=32, levels=2) as ctx:
        batch = ctx.solve(args)
        alone = [ctx.solve([x])[0] for x in args]
    for rb, ra in zip(batch, alone):
        assert np.array_equal(rb.q, ra.q)
        assert (rb.best_count, rb.inliers, rb.best_cell, rb.refits) == (ra.best_count, ra.inliers, ra.best_cell,
                                                                        ra.refits)
    for p, r in zip(probs, batch):
        if p.n <= 32768:
            continue
        o = oracle.solve(p.a, p.b, f32(p.delta), grid_n=32, levels=2, nthreads=NTHREADS, trace=False)
        assert r.status == o.status == 0
        assert r.best_cell == o.best_cell
        assert quat_angle(r.q, o.q) < ROT_TOL


def test_graph_replay_with_new_inputs():
    """The captured pipeline is replayed for a second solve of the same shape
    with different data; results must be those of the new data."""
    import oracle
    p1 = synth.make_problem(3000, rho=0.9, sigma=0.01, delta=0.03, seed=11)
    p2 = synth.make_problem(3000, rho=0.9, sigma=0.01, delta=0.04, seed=12)
    with rv.Context(grid_n=16, levels=2, use_graphs=1) as cg, rv.Context(grid_n=16, levels=2, use_graphs=-1) as cn:
        g1 = cg.solve([(dev(p1.a), dev(p1.b), p1.delta)])[0]
        g2 = cg.solve([(dev(p2.a), dev(p2.b), p2.delta)])[0]
        n2 = cn.solve([(dev(p2.a), dev(p2.b), p2.delta)])[0]
    o2 = oracle.solve(p2.a, p2.b, f32(p2.delta), grid_n=16, levels=2)
    assert np.array_equal(g2.q, n2.q) and g2.best_cell == n2.best_cell
    assert quat_angle(g2.q, o2.q) < ROT_TOL
    assert g1.best_cell != g2.best_cell or not np.array_equal(g1.q, g2.q)


def test_batches_reusing_the_plan_equal_fresh_solves():
    """A context keeps a batch's plan (layout, work items, tables) for the next
    batch of the same shapes and refreshes only the inputs and tolerances.  A
    sequence that repeats, changes and restores the shapes and switches the
    inputs between device and host memory must give, batch by batch, the results
    of a fresh context."""
    def batch(seed, sizes, deltas):
        return [synth.make_problem(n, rho=0.9, sigma=0.01, delta=d, seed=seed + k)
                for k, (n, d) in enumerate(zip(sizes, deltas))]
    s1, s2 = [300, 5000, 1200], [300, 700]
    seq = [(batch(40, s1, [0.03, 0.03, 0.03]), True), (batch(50, s1, [0.04, 0.02, 0.035]), True),
           (batch(60, s2, [0.03, 0.03]), True), (batch(70, s1, [0.03, 0.05, 0.03]), False),
           (batch(80, s1, [0.025, 0.03, 0.03]), True)]
    for prec in ("fp16x2", "fp32"):
        with rv.Context(grid_n=16, levels=2, precision=prec) as ctx:
            got = []
            for probs, on_dev in seq:
                args = [((dev(p.a), dev(p.b)) if on_dev else (p.a, p.b)) + (p.delta,) for p in probs]
                got.append(ctx.solve(args))
        for (probs, on_dev), res in zip(seq, got):
            with rv.Context(grid_n=16, levels=2, precision=prec) as fresh:
                ref = fresh.solve([(dev(p.a), dev(p.b), p.delta) for p in probs])
            for r, f in zip(res, ref):
                assert np.array_equal(r.q, f.q)
                assert (r.best_count, r.best_cell, r.inliers, r.tests, r.rechecked, r.ambiguous, r.status) == \
                       (f.best_count, f.best_cell, f.inliers, f.tests, f.rechecked, f.ambiguous, f.status)


def test_invalid_inputs_are_rejected():
    p = synth.make_problem(300, rho=0.5, sigma=0.01, delta=0.03, seed=13)
    bad_nan = p.a.copy()
    bad_nan[7, 1] = np.nan
    bad_norm = p.a.copy()
    bad_norm[3] *= 1.001
    with rv.Context(grid_n=8) as ctx:
        res = ctx.solve([(p.a[:1], p.b[:1], 0.03), (bad_nan, p.b, 0.03), (bad_norm, p.b, 0.03),
                         (p.a, p.b, 0.0), (p.a, p.b, 2.0), (p.a, p.b, 0.03)])
    assert [r.status for r in res[:5]] == [rv.EINVAL] * 5
    assert res[5].status == 0


def test_full_size_fp32_workload():
    """The 1e5-pair, 64^3 + 3-level workload at full size, in the launch
    configuration the benchmark times: the oracle's complete solve (threads
    over cells) against the GPU's every level."""
    p, g, L = synth.config_problem("fp32_n1e5_64L3")
    r, tr, o = run_both(p, g, L)
    assert_parity(p, r, tr, o, L)
    assert quat_angle(r.q, p.q_true) < 0.01


# ---- the stereographic chart of Sec. 4.3.1 (rot_vote_config.chart = 1) ----

@pytest.mark.parametrize("precision", ["fp32", "fp16x2", "bf16"])
def test_stereographic_chart_every_level(precision):
    p, g, L = synth.config_problem("small_n1e3_32")
    r, tr, o = run_both(p, g, L, precision=precision, chart=1)
    assert_parity(p, r, tr, o, L)
    q = synth.make_problem(3000, rho=0.9, sigma=0.01, delta=0.03, seed=81)
    r, tr, o = run_both(q, 16, 3, precision=precision, chart=1)
    assert_parity(q, r, tr, o, 3)


@pytest.mark.parametrize("n", [2, 129, 257])
def test_stereographic_chart_ragged(n):
    p = synth.make_problem(n, rho=0.5, sigma=0.01, delta=0.05, seed=300 + n)
    r, tr, o = run_both(p, 8, 2, chart=1)
    assert_parity(p, r, tr, o, 2)


def test_stereographic_chart_full_size_fp32_workload():
    """The 1e5-pair, 64^3 + 3-level workload in the stereographic chart, every level."""
    p, g, L = synth.config_problem("fp32_n1e5_64L3")
    r, tr, o = run_both(p, g, L, chart=1)
    assert_parity(p, r, tr, o, L)
    assert quat_angle(r.q, p.q_true) < 0.01


def test_stereographic_chart_batched_equals_alone():
    probs = [synth.make_problem(n, rho=0.8, sigma=0.01, delta=0.03, seed=s)
             for n, s in ((50, 21), (700, 22), (4096, 23))]
    args = [(dev(p.a), dev(p.b), p.delta) for p in probs]
    with rv.Context(grid_n=32, levels=2, chart="stereographic") as ctx:
        batch = ctx.solve(args)
        alone = [ctx.solve([x])[0] for x in args]
    for rb, ra in zip(batch, alone):
        assert np.array_equal(rb.q, ra.q) and (rb.best_cell, rb.best_count) == (ra.best_cell, ra.best_count)


# ---- extremes of the configuration space ----

def test_largest_coarse_grid_256():
    """256^3 coarse grid (about 8.8M cells meeting the ball) + 1 level, FP32 and FP16X2."""
    p = synth.make_problem(300, rho=0.8, sigma=0.01, delta=0.03, seed=401)
    for prec in ("fp32", "fp16x2"):
        r, tr, o = run_both(p, 256, 1, precision=prec)
        assert_parity(p, r, tr, o, 1)


def test_deep_refinement_side_512():
    """8^3 + 6 levels: the last level is a 512-per-axis grid."""
    p = synth.make_problem(2000, rho=0.7, sigma=0.005, delta=0.01, seed=402)
    r, tr, o = run_both(p, 8, 6)
    assert_parity(p, r, tr, o, 6)


@pytest.mark.parametrize("delta", [1e-4, 1.5])
def test_delta_extremes(delta):
    """delta = 1e-4 (few voters; the fit may be degenerate) and delta = 1.5 rad
    (every threshold saturates at 1: every cell votes for every pair)."""
    p = synth.make_problem(500, rho=0.5, sigma=0.0, delta=delta, seed=403)
    r, tr, o = run_both(p, 16, 1)
    assert_parity(p, r, tr, o, 1)
    if delta == 1.5:
        assert all(int(c.min()) == p.n for _, c, _ in tr[:1])


def test_batched_workload_4096_problems_sample_equals_oracle():
    """The benchmark's batched workload at full scale: 4096 independent problems
    (N log-uniform in [50, 2e4], outliers U[0.5, 0.95], noise U[0.001, 0.02],
    delta = 3 sigma; 32^3 + 2 levels) in one call, FP16 hi/lo form.  A seeded
    sample of 64 problems, including the smallest and the largest, must equal
    the oracle's solve: the winning cell and its count, the ambiguous tests, the
    tests, the inliers and the status; the rotation within 1e-4 rad."""
    import oracle
    probs = synth.batched_problems(4096)
    args = [(dev(p.a), dev(p.b), p.delta) for p in probs]
    with rv.Context(grid_n=32, levels=2, precision="fp16x2") as ctx:
        res = ctx.solve(args)
    ns = np.array([p.n for p in probs])
    rng = np.random.default_rng(4096)
    pick = set(rng.choice(len(probs), 62, replace=False).tolist()) | {int(ns.argmin()), int(ns.argmax())}
    for k in sorted(pick):
        p, r = probs[k], res[k]
        o = oracle.solve(p.a, p.b, f32(p.delta), grid_n=32, levels=2, nthreads=NTHREADS, trace=False)
        assert r.status == o.status, k
        assert (r.best_cell, r.best_count, r.ambiguous, r.tests, r.inliers) == \
               (o.best_cell, o.best_count, o.ambiguous, o.tests, o.inliers), k
        assert quat_angle(r.q, o.q) < ROT_TOL, k
