"""Per-kernel event timing (btc_plan_set_timing / btc_plan_timing), the
device-side item trace (btc_plan_set_trace) of the persistent launches and the
per-node phase stamps of the factorization (btc_plan_set_phase_trace).

The trace doubles as an on-device check of the interlaced schedule: every item
may start only after each of the items it depends on has finished (times from
the global nanosecond timer)."""
import numpy as np
import pytest

from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import dev, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


def _inputs(N, n, seed=0):
    D, B = gen.bt_random(N, n, delta=1.0, seed=seed)
    b = gen.rhs(N, n, 1, seed=seed)
    return dev(D, torch.float64), dev(B, torch.float64), dev(b, torch.float64)


def test_timing_classes_of_a_refined_call():
    N, n = 300, 32
    Dd, Bd, bd = _inputs(N, n)
    p = btc.btc_plan(N, n, btc.MIXED_F32)
    x = torch.zeros_like(bd)
    btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, 1)  # tuning run
    btc.btc_plan_set_timing(p, True)
    it, rel, _ = btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, 1)
    ms, cnt = btc.btc_plan_timing(p)
    assert cnt[btc.TIME_FACTOR_FORWARD] == 1 and cnt[btc.TIME_ROOT] == 1 and cnt[btc.TIME_SOLVE_TAIL] == 1
    assert cnt[btc.TIME_SOLVE] == it and cnt[btc.TIME_RESIDUAL] == it + 1
    assert cnt[btc.TIME_FACTOR] == 0
    for c in range(btc.TIMING_CLASSES):
        assert (ms[c] > 0) == (cnt[c] > 0), c
    ms2, cnt2 = btc.btc_plan_timing(p)  # read and reset
    assert sum(cnt2) == 0 and sum(ms2) == 0
    btc.btc_factor(p, Dd, Bd)
    ms3, cnt3 = btc.btc_plan_timing(p)
    assert cnt3[btc.TIME_FACTOR] == 1 and cnt3[btc.TIME_ROOT] == 1
    btc.btc_plan_set_timing(p, False)
    btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, 1)
    assert sum(btc.btc_plan_timing(p)[1]) == 0


@pytest.mark.parametrize("N,n", [(257, 16), (1024, 64)])
def test_trace_shows_every_interlaced_item_after_its_dependencies(N, n):
    Dd, Bd, bd = _inputs(N, n, seed=3)
    kind, node, level, deps, ntail = btc.btc_schedule_interlaced(N, True)
    cnt = len(kind)
    tf = torch.zeros(4 * cnt, dtype=torch.int64, device="cuda")
    ts = torch.zeros(4 * max(ntail, 1), dtype=torch.int64, device="cuda")
    p = btc.btc_plan(N, n, btc.MIXED_F32)
    btc.btc_plan_set_trace(p, tf, ts)
    x = bd.clone()
    btc.btc_factor_solve(p, Dd, Bd, x, 1)
    assert btc.btc_info(p)[0] == btc.OK
    F = tf.view(-1, 4).cpu().numpy()
    claim, ready, done, sm = F[:, 0], F[:, 1], F[:, 2], F[:, 3]
    assert np.all(done > 0), "every item of the interlaced launch ran"
    assert np.all(claim <= ready) and np.all(ready <= done)
    assert np.all((sm >= 0) & (sm < 1024))
    for t in range(cnt):
        for d in deps[t]:
            if d == -1:
                continue
            q = int(d) if d >= 0 else -int(d) - 2
            # every entry starts after its dependencies started; a forward entry's "ready" stamp
            # follows the completion of its complete-dependencies; a factor entry's "ready" stamp
            # follows only its dependencies' factor blocks (it waits for the rest inside), and it
            # completes after them
            assert ready[t] >= ready[q], (t, q)
            if d >= 0:
                if kind[t] == 1:
                    assert ready[t] >= done[q], (t, q)
                else:
                    assert done[t] >= done[q], (t, q)
    S = ts.view(-1, 4).cpu().numpy()
    assert np.all(S[:ntail, 2] > 0), "every item of the solve tail ran"
    # tracing does not change the result
    q = btc.btc_plan(N, n, btc.MIXED_F32)
    y = bd.clone()
    btc.btc_factor_solve(q, Dd, Bd, y, 1)
    assert torch.equal(x, y)


@pytest.mark.parametrize("dt,variant", [(btc.MIXED_F32, btc.VARIANT_HYBRID), (btc.F64, btc.VARIANT_HYBRID),
                                        (btc.MIXED_F32, btc.VARIANT_RIGHT_LOOKING)], ids=["mixed", "f64", "mixed-rl"])
def test_phase_stamps_are_ordered_and_leave_results_unchanged(dt, variant):
    N, n = 300, 32
    Dd, Bd, bd = _inputs(N, n, seed=7)
    ph = torch.zeros(8 * N, dtype=torch.int64, device="cuda")
    out = []
    for stamps in (ph, None):
        p = btc.btc_plan(N, n, dt)
        btc.btc_plan_set_variant(p, variant)
        btc.btc_plan_set_phase_trace(p, stamps)
        x = bd.clone()
        if variant == btc.VARIANT_HYBRID:
            btc.btc_factor_solve(p, Dd, Bd, x, 1)
        else:
            btc.btc_factor(p, Dd, Bd)
            btc.btc_solve(p, x, 1)
        assert btc.btc_info(p)[0] == btc.OK
        out.append(x)
    if variant == btc.VARIANT_HYBRID:
        assert torch.equal(out[0], out[1]), "stamping does not change the result"
    else:  # the right-looking updates are floating-point atomics in no fixed order
        assert torch.allclose(out[0], out[1], rtol=1e-4, atol=1e-6)
    P = ph.view(N, 8).cpu().numpy()
    stamped = P[:, 5] > 0
    expect = np.ones(N, dtype=bool)
    if dt == btc.MIXED_F32:  # the top separator is factored by the separate root kernel
        expect[(1 << (N.bit_length() - 1)) - 1] = False
    assert np.array_equal(stamped, expect)
    assert np.all(np.diff(P[stamped, :6], axis=1) >= 0), "phases in order"
    assert np.all(P[stamped, 6] < 1024)
    # a node's operands are in place only after the nodes of the previous level that write them have
    # finished: node e at level l (stride s = 2^(l-1)) depends on e - s/2 and e + s/2 (its deferred
    # products may start earlier, from their factor blocks)
    lev = np.array([((i + 1) & -(i + 1)).bit_length() for i in range(N)])
    for e in np.where(stamped & (lev > 1))[0]:
        h = 1 << (lev[e] - 2)
        for q in (e - h, e + h):
            if 0 <= q < N and stamped[q]:
                assert P[e, 1] >= P[q, 5], (int(e), int(q))
                assert P[e, 0] >= P[q, 0], (int(e), int(q))
