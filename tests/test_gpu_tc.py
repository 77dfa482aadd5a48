"""GPU parity of the tcgen05 tensor-core vote (FP16 / BF16, single and hi/lo
split operands) against the FP64 oracle, and against the FP32 CUDA-core form.

Every non-ambiguous decision of every mode is the FP64 decision, and every
test within 1e-6 of the threshold lies inside every mode's re-check band and
gets the same FP32 re-check; so all modes must give identical counts."""
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
from tests.test_gpu_parity import assert_parity, dev, run_both, ROT_TOL  # noqa: E402

PRECS = ["fp16x2", "bf16x2", "fp16", "bf16"]
NTHREADS = max(1, os.cpu_count() or 1)


@pytest.mark.parametrize("prec", PRECS)
def test_tc_small_workload_every_cell(prec):
    p, g, L = synth.config_problem("small_n1e3_32")
    r, tr, o = run_both(p, g, L, precision=prec)
    assert_parity(p, r, tr, o, L)


@pytest.mark.parametrize("prec", PRECS)
def test_tc_multilevel_every_level(prec):
    p = synth.make_problem(3000, rho=0.9, sigma=0.01, delta=0.03, seed=77)
    r, tr, o = run_both(p, 16, 3, precision=prec)
    assert_parity(p, r, tr, o, 3)


@pytest.mark.parametrize("prec", ["fp16x2", "bf16"])
@pytest.mark.parametrize("n", [2, 129, 1000, 4097])
def test_tc_ragged_sizes(prec, n):
    p = synth.make_problem(n, rho=0.5, sigma=0.01, delta=0.05, seed=300 + n)
    r, tr, o = run_both(p, 8, 2, precision=prec)
    assert_parity(p, r, tr, o, 2)


@pytest.mark.parametrize("prec", PRECS)
def test_tc_counts_identical_to_fp32_form(prec):
    p = synth.make_problem(20000, rho=0.95, sigma=0.01, delta=0.03, seed=21)
    out = {}
    for pr in ("fp32", prec):
        with rv.Context(grid_n=32, levels=2, precision=pr, keep_trace=1) as ctx:
            r = ctx.solve([(dev(p.a), dev(p.b), p.delta)])[0]
            out[pr] = (r, [ctx.level_trace(0, lev) for lev in range(3)])
    (r32, t32), (rtc, ttc) = out["fp32"], out[prec]
    for lev in range(3):
        assert np.array_equal(t32[lev][0], ttc[lev][0])
        assert np.array_equal(t32[lev][1], ttc[lev][1])
        assert np.array_equal(t32[lev][2], ttc[lev][2])
    assert np.array_equal(r32.q, rtc.q) and r32.inliers == rtc.inliers


TC_SHAPES = [2, 4, 12, 14, 102, 104, 112, 114]


@pytest.mark.parametrize("shape", TC_SHAPES)
def test_every_tc_tile_shape_counts_identical_to_fp32(shape):
    p = synth.make_problem(9000, rho=0.95, sigma=0.01, delta=0.03, seed=22)
    out = {}
    for pr, sh in (("fp32", 4), ("fp16x2", shape), ("bf16", shape)):
        with rv.Context(grid_n=16, levels=2, precision=pr, keep_trace=1, autotune=sh) as ctx:
            r = ctx.solve([(dev(p.a), dev(p.b), p.delta)])[0]
            out[pr] = (r, [ctx.level_trace(0, lev) for lev in range(3)])
    r32, t32 = out["fp32"]
    for pr in ("fp16x2", "bf16"):
        rr, tt = out[pr]
        for lev in range(3):
            assert np.array_equal(t32[lev][1], tt[lev][1])
            assert np.array_equal(t32[lev][2], tt[lev][2])
        assert np.array_equal(r32.q, rr.q)


@pytest.mark.parametrize("prec", ["fp16x2", "bf16x2"])
def test_tc_batched_equals_alone(prec):
    probs = [synth.make_problem(n, rho=0.8, sigma=0.01, delta=d, seed=s)
             for n, d, s in ((50, 0.03, 1), (700, 0.02, 2), (4096, 0.05, 3), (129, 0.04, 4), (20000, 0.03, 5))]
    args = [(dev(p.a), dev(p.b), p.delta) for p in probs]
    with rv.Context(grid_n=32, levels=2, precision=prec) as ctx:
        batch = ctx.solve(args)
        alone = [ctx.solve([x])[0] for x in args]
    for rb, ra in zip(batch, alone):
        assert np.array_equal(rb.q, ra.q)
        assert (rb.best_count, rb.inliers, rb.best_cell, rb.tests, rb.rechecked) == \
               (ra.best_count, ra.inliers, ra.best_cell, ra.tests, ra.rechecked)


@pytest.mark.parametrize("prec", ["fp16x2"])
def test_tc_full_size_paper_workload(prec):
    """1e6 pairs, 99% outliers, 128^3 + 3 levels, in the benchmark's launch
    configuration.  The oracle cannot vote all 1.1e12 tests, so it checks:
    sampled coarse cells and the kept ones (exact counts), the ranking
    property on the sample, every refinement level in full (counts and the
    kept ranking recomputed by the oracle on the GPU's child table), and the
    fit from the GPU's winner."""
    import oracle
    p, g, L = synth.config_problem("lowp_n1e6_128L3")
    delta = f32(p.delta)
    with rv.Context(grid_n=g, levels=L, precision=prec, keep_trace=1) as ctx:
        r = ctx.solve([(dev(p.a), dev(p.b), p.delta)])[0]
        tr = [ctx.level_trace(0, lev) for lev in range(L + 1)]
    assert r.status == 0
    idx0, cnt0, kept0 = tr[0]
    assert len(idx0) == 1136840
    rng = np.random.default_rng(5)
    sample = rng.choice(len(idx0), 256, replace=False)
    pos_kept = np.searchsorted(idx0, kept0)
    pos = np.concatenate([sample, pos_kept])
    oc, oa, ot = oracle.vote_cells(p.a, p.b, delta, g, idx0[pos], nthreads=NTHREADS)
    assert np.all(np.abs(cnt0[pos].astype(np.int64) - oc) <= oa)
    score = oc - p.n * ot
    ns = len(sample)
    assert score[ns:].min() >= score[:ns].max() - 1e-9  # kept cells outrank the sample
    for lev in range(1, L + 1):
        idx, cnt, kept = tr[lev]
        n_side = g << lev
        oc, oa, ot = oracle.vote_cells(p.a, p.b, delta, n_side, idx, nthreads=NTHREADS)
        assert np.all(np.abs(cnt.astype(np.int64) - oc) <= oa)
        opos, _ = oracle.rank(oc, ot, idx, p.n, 0, 16)
        assert np.array_equal(idx[opos], kept)
    assert r.best_cell == tr[L][2][0]
    of = oracle.fit_cell(p.a, p.b, delta, g << L, r.best_cell)
    assert of.status == r.status
    assert quat_angle(r.q, of.q) < ROT_TOL
    assert quat_angle(r.q, p.q_true) < 0.01
