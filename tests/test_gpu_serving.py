"""Serving (rot_vote_submit / rot_vote_poll): continuous batching on several
overlapping waves.  Each result must be the same when the problem is solved
alone and when it runs in the mix; the queue bound answers EAGAIN; poll has
PENDING / ENOTFOUND semantics; invalid problems are rejected at submit."""
import time

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
            and r.inliers == s.inliers and r.tests == s.tests and r.rechecked == s.rechecked
            and r.status == s.status)


def _drain(ctx, tickets, timeout_s=120.0):
    out = {}
    t_end = time.time() + timeout_s
    while len(out) < len(tickets) and time.time() < t_end:
        for t in tickets:
            if t not in out:
                r = ctx.poll(t, timeout_us=2000)
                if r is not None:
                    out[t] = r
    assert len(out) == len(tickets), "serving did not finish in time"
    return out


@pytest.mark.parametrize("prec", ["fp16x2", "fp32"])
def test_serving_result_same_alone_and_in_the_mix(prec):
    rng = np.random.default_rng(11)
    ns = np.exp(rng.uniform(np.log(60), np.log(8000), size=40)).astype(int)
    probs = [synth.make_problem(int(n), rho=float(rng.uniform(0.5, 0.95)), sigma=0.01, delta=0.03,
                                seed=500 + k) for k, n in enumerate(ns)]
    args = [(_dev(p.a), _dev(p.b), p.delta) for p in probs]
    with rv.Context(grid_n=16, levels=2, precision=prec, max_inflight=8) as ctx:
        # burst: later problems are queued while earlier waves are on the device
        tickets = [ctx.submit(*x) for x in args]
        assert all(t > 0 for t in tickets)
        mixed = _drain(ctx, tickets)
    with rv.Context(grid_n=16, levels=2, precision=prec) as ctx:
        alone = [ctx.solve([x])[0] for x in args]
    for t, ra in zip(tickets, alone):
        rm = mixed[t]
        assert rm.latency_ms > 0
        assert _same(rm, ra)


def test_serving_queue_bound_and_poll_semantics():
    p = synth.make_problem(2000, rho=0.9, sigma=0.01, delta=0.03, seed=77)
    x = (_dev(p.a), _dev(p.b), p.delta)
    with rv.Context(grid_n=16, levels=1, precision="fp32", max_inflight=1) as ctx:
        tickets, refused = [], 0
        for _ in range(64):  # the admission queue holds max_inflight * 8 problems
            t = ctx.submit(*x)
            if t < 0:
                refused += 1
            else:
                tickets.append(t)
        assert refused > 0
        with pytest.raises(rv.RotVoteError) as e:
            ctx.poll(max(tickets) + 1000)
        assert e.value.code == rv.ENOTFOUND
        res = _drain(ctx, tickets)
        assert all(r.status == rv.OK for r in res.values())
        assert len({tuple(r.q) for r in res.values()}) == 1  # same problem, same answer
        with pytest.raises(rv.RotVoteError) as e:  # a collected ticket is released
            ctx.poll(tickets[0])
        assert e.value.code == rv.ENOTFOUND


def test_serving_rejects_invalid_problem_at_submit():
    p = synth.make_problem(100, rho=0.5, sigma=0.01, delta=0.03, seed=3)
    with rv.Context(grid_n=16, levels=0) as ctx:
        with pytest.raises(rv.RotVoteError) as e:
            ctx.submit(_dev(p.a[:1]), _dev(p.b[:1]), p.delta)  # n < 2
        assert e.value.code == rv.EINVAL
        with pytest.raises(rv.RotVoteError) as e:
            ctx.submit(_dev(p.a), _dev(p.b), 2.0)  # delta outside (0, pi/2)
        assert e.value.code == rv.EINVAL


def _serve_alone(budget, x, prec="fp16x2"):
    """Status of one problem served on a fresh context with the given device budget."""
    with rv.Context(grid_n=16, levels=2, precision=prec, device_mem_budget=budget, max_inflight=64) as ctx:
        t = ctx.submit(*x)
        return _drain(ctx, [t])[t].status


def test_serving_results_equal_the_oracle():
    """A burst of uneven problems through submit/poll: every result equals the
    oracle's solve of the same problem (winning cell and count, ambiguous
    tests, status; rotation within 1e-4 rad)."""
    import oracle
    from tests._util import f32, quat_angle
    rng = np.random.default_rng(12)
    ns = np.exp(rng.uniform(np.log(100), np.log(20000), size=24)).astype(int)
    probs = [synth.make_problem(int(n), rho=float(rng.uniform(0.8, 0.99)), sigma=0.01, delta=0.03, seed=700 + k)
             for k, n in enumerate(ns)]
    args = [(_dev(p.a), _dev(p.b), p.delta) for p in probs]
    with rv.Context(grid_n=16, levels=2, precision="fp16x2", max_inflight=6) as ctx:
        tickets = [ctx.submit(*x) for x in args]
        got = _drain(ctx, tickets)
    for p, t in zip(probs, tickets):
        r = got[t]
        o = oracle.solve(p.a, p.b, f32(p.delta), grid_n=16, levels=2, trace=False)
        assert r.status == o.status
        assert (r.best_cell, r.best_count, r.ambiguous, r.tests) == (o.best_cell, o.best_count, o.ambiguous, o.tests)
        assert quat_angle(r.q, o.q) < 1e-4


def test_serving_admits_a_large_problem_under_a_small_memory_budget():
    """Admission by device memory: the budget is just above what the large
    problem needs alone, so it cannot run while the waves of the small problems
    hold their workspaces.  Submitted between bursts of small problems, it must
    wait for memory (not fail), and every result must equal the problem solved
    alone."""
    big = synth.make_problem(60000, rho=0.95, sigma=0.01, delta=0.03, seed=801)
    xb = (_dev(big.a), _dev(big.b), big.delta)
    lo, hi = 1 << 20, 1 << 32  # smallest budget (to 4%) that serves the large problem alone
    assert _serve_alone(hi, xb) == rv.OK
    while hi > lo * 1.04:
        mid = (lo + hi) // 2
        if _serve_alone(mid, xb) == rv.OK:
            hi = mid
        else:
            lo = mid
    budget = int(hi * 1.1)
    small = [synth.make_problem(int(n), rho=0.9, sigma=0.01, delta=0.03, seed=820 + k)
             for k, n in enumerate([3000, 150, 8000, 900, 5000, 2500, 12000, 400] * 2)]
    xs = [(_dev(p.a), _dev(p.b), p.delta) for p in small]
    with rv.Context(grid_n=16, levels=2, precision="fp16x2", device_mem_budget=budget, max_inflight=3) as ctx:
        order = xs[:8] + [xb] + xs[8:]
        tickets = [ctx.submit(*x) for x in order]
        got = _drain(ctx, tickets)
        spans = ctx.serve_spans()
    with rv.Context(grid_n=16, levels=2, precision="fp16x2") as ctx:
        alone = [ctx.solve([x])[0] for x in order]
    for t, ra in zip(tickets, alone):
        assert got[t].status == rv.OK, got[t].status
        assert _same(got[t], ra)
    assert sum(s[3] for s in spans) == len(order)
    assert all(s[1] >= s[0] >= 0.0 for s in spans)


def test_serving_spans_show_overlapping_waves():
    """The batch spans of a stream: one per completed batch, with device start <=
    end.  Requests arrive two at a time while earlier batches run, so they are
    admitted onto other waves and are in flight at the same time (their spans
    intersect).  (A burst submitted at once is one batch on one wave.)"""
    rng = np.random.default_rng(13)
    ns = np.exp(rng.uniform(np.log(20000), np.log(60000), size=32)).astype(int)
    probs = [synth.make_problem(int(n), rho=0.9, sigma=0.01, delta=0.03, seed=900 + k) for k, n in enumerate(ns)]
    args = [(_dev(p.a), _dev(p.b), p.delta) for p in probs]
    with rv.Context(grid_n=32, levels=2, precision="fp32", max_inflight=64) as ctx:
        ctx.solve([args[0]])  # tuning and the coarse table before the stream
        tickets = []
        for k in range(0, len(args), 2):
            tickets += [ctx.submit(*x) for x in args[k:k + 2]]
            time.sleep(0.0005)
        _drain(ctx, tickets)
        spans = ctx.serve_spans()
    assert sum(s[3] for s in spans) == len(args)
    assert len({s[2] for s in spans}) > 1  # more than one wave ran batches
    ivs = sorted((s[0], s[1]) for s in spans)
    overlap = any(ivs[k + 1][0] < ivs[k][1] for k in range(len(ivs) - 1))
    assert overlap, ivs[:8]
