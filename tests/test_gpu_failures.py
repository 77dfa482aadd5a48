"""Failure detection without a GPU fault: faults are injected on the host (an
allocation that fails, a context destroyed with work in flight), and a device
wait is made to run out (the tensor-core producer never issues its copies, and
waits are bounded by 1 ms): the kernel reports through its error word, the call
returns ETIMEDOUT and the context stays usable.  Plus a determinism check."""
import numpy as np
import pytest

from paper_2506_11547_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

from paper_2506_11547_gb300 import rot_vote as rv  # noqa: E402


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _same(r, s):
    return (np.array_equal(r.q, s.q) and r.best_cell == s.best_cell and r.best_count == s.best_count
            and r.inliers == s.inliers and r.tests == s.tests and r.rechecked == s.rechecked)


def _problem():
    p = synth.make_problem(4000, rho=0.9, sigma=0.01, delta=0.03, seed=61)
    return p, (_dev(p.a), _dev(p.b), p.delta)


def test_injected_allocation_failure_leaves_a_clean_context(monkeypatch):
    p, x = _problem()
    with rv.Context(grid_n=16, levels=2) as ref:
        want = ref.solve([x])[0]
    monkeypatch.setenv("ROT_VOTE_TEST_FAIL_ALLOC", "1")  # the first workspace allocation fails
    with rv.Context(grid_n=16, levels=2) as ctx:
        with pytest.raises(rv.RotVoteError) as e:
            ctx.solve([x])
        assert e.value.code == rv.ENOMEM
        got = ctx.solve([x])[0]  # the next call allocates and runs normally
    assert got.status == rv.OK and _same(got, want)


@pytest.mark.parametrize("prec", ["fp16x2", "bf16"])
def test_device_wait_expiry_is_reported_and_the_context_recovers(monkeypatch, prec):
    p, x = _problem()
    with rv.Context(grid_n=16, levels=2, precision=prec, autotune=2) as ref:
        want = ref.solve([x])[0]
    monkeypatch.setenv("ROT_VOTE_TEST_STALL", "2")  # the next two solves' copies never arrive
    with rv.Context(grid_n=16, levels=2, precision=prec, autotune=2) as ctx:
        for _ in range(2):
            with pytest.raises(rv.RotVoteError) as e:
                ctx.solve([x])
            assert e.value.code == rv.ETIMEDOUT
        got = ctx.solve([x])[0]
        got2 = ctx.solve([x])[0]  # graph capture and replay after the failures
    torch.cuda.synchronize()  # the device is healthy
    assert _same(got, want) and _same(got2, want)


def test_destroy_with_work_in_flight():
    probs = [synth.make_problem(n, rho=0.9, sigma=0.01, delta=0.03, seed=70 + k)
             for k, n in enumerate((300, 5000, 20000, 800, 12000))]
    args = [(_dev(p.a), _dev(p.b), p.delta) for p in probs]
    ctx = rv.Context(grid_n=32, levels=2, precision="fp16x2")
    tickets = [ctx.submit(*x) for x in args * 4]
    assert all(t > 0 for t in tickets)
    ctx.close()  # waits for the in-flight waves, frees everything
    with rv.Context(grid_n=32, levels=2, precision="fp16x2") as ctx2:
        res = ctx2.solve(args)
    assert all(r.status == rv.OK for r in res)


@pytest.mark.parametrize("prec", ["fp32", "fp16x2"])
def test_ten_repeated_runs_are_bitwise_equal(prec):
    p, x = _problem()
    with rv.Context(grid_n=32, levels=2, precision=prec, keep_trace=1) as ctx:
        first = ctx.solve([x])[0]
        tr0 = [ctx.level_trace(0, lev) for lev in range(3)]
        for _ in range(9):
            r = ctx.solve([x])[0]
            assert _same(r, first) and r.ambiguous == first.ambiguous
            tr = [ctx.level_trace(0, lev) for lev in range(3)]
            for a, b in zip(tr0, tr):
                assert all(np.array_equal(u, v) for u, v in zip(a, b))


@pytest.mark.parametrize("cap", ["0", "16"])
def test_full_fp64_queue_recounts_exactly(cap, monkeypatch):
    """Host hook ROT_VOTE_TEST_AMB_CAP shrinks the FP64 resolution queue (0 or 16
    tests), so the tests near the threshold that it cannot take flag their cells
    and the resolution pass recounts those cells from all pairs.  Counts, kept
    cells, ambiguous totals and the rotation must still equal the oracle's, in
    the FP32 and the tensor-core forms."""
    from tests.test_gpu_parity import assert_parity, run_both
    monkeypatch.setenv("ROT_VOTE_TEST_AMB_CAP", cap)
    p = synth.make_problem(20000, rho=0.9, sigma=0.01, delta=0.03, seed=41)
    for prec in ("fp32", "fp16x2", "bf16"):
        r, tr, o = run_both(p, 16, 2, precision=prec)
        assert_parity(p, r, tr, o, 2)
        assert r.resolved > 0
