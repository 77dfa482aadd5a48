"""GPU parity of the tcgen05 tensor-core vote (FP16 / BF16, single and hi/lo
split operands) against the FP64 oracle, and against the FP32 CUDA-core form.

Every decision of every mode is the FP64 decision: outside its rigorous band
the fast value decides, inside it the FP32 re-check, and within 2e-6 of the
threshold the FP64 evaluation; so all modes give the oracle's counts."""
import hashlib
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


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_scale_trace.npz")


@pytest.mark.parametrize("prec", ["fp16x2", "bf16x2", "fp16", "bf16", "fp32"])
def test_full_size_paper_workload_every_form(prec):
    """1e6 pairs, 99% outliers, 128^3 + 3 levels (1.14e12 tests), in the
    benchmark's launch configuration, in every precision form: every one of
    the 1,136,840 coarse counts, every refinement level's cells, counts and
    kept ranking, the total of ambiguous tests and the result, against the
    oracle's full trace of the same seeded inputs (tests/golden/
    paper_scale_trace.npz, written by make_paper_scale_trace.py there)."""
    import oracle
    gold = np.load(GOLDEN)
    p, g, L = synth.config_problem("lowp_n1e6_128L3")
    assert hashlib.sha256(p.a.tobytes() + p.b.tobytes()).hexdigest() == str(gold["input_sha256"]), \
        "the seeded generator no longer reproduces the stored workload"
    with rv.Context(grid_n=g, levels=L, precision=prec, keep_trace=1) as ctx:
        r = ctx.solve([(dev(p.a), dev(p.b), p.delta)])[0]
        tr = [ctx.level_trace(0, lev) for lev in range(L + 1)]
    assert r.status == int(gold["status"]) == 0
    idx0, cnt0, kept0 = tr[0]
    assert len(idx0) == 1136840
    assert np.array_equal(idx0, oracle.level_cells(g))
    bad = np.nonzero(cnt0 != gold["l0_count"])[0]
    assert len(bad) == 0, f"{len(bad)} coarse cells differ, e.g. {bad[:5]}"
    assert np.array_equal(kept0, gold["topk0"])
    for lev in range(1, L + 1):
        idx, cnt, kept = tr[lev]
        assert np.array_equal(idx, gold[f"l{lev}_idx"])
        assert np.array_equal(cnt, gold[f"l{lev}_count"])
        assert np.array_equal(kept, gold[f"topk{lev}"])
    assert r.ambiguous == int(gold["ambiguous"])
    assert r.tests == int(gold["tests"])
    assert (r.best_cell, r.best_count) == (int(gold["best_cell"]), int(gold["best_count"]))
    assert r.inliers == int(gold["inliers"])
    assert quat_angle(r.q, gold["q"]) < ROT_TOL
    assert quat_angle(r.q, p.q_true) < 0.01
