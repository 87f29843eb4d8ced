"""The one-CTA solve of small plans (FP32 factor, padded n <= 16, one
right-hand side, no dependency wave of the solve wider than 64 items) against
the persistent dataflow kernel; FP64 and n_p = 32 plans stay on the dataflow
kernel and run the same cases.

Both run the same per-item arithmetic (Alg. 7's pull-form forward step and the
backward step, with the same split of the products and the same triangular
solve), so the results must be bitwise equal. The dataflow kernel is forced by
a solve trace buffer (tracing is a dataflow-kernel feature); the level
schedule's per-level kernels are a second bitwise reference. Covered: the
separate solve, the tail after the interlaced factorization (mixed and FP64),
the refined solve, the partition order, and the wave limit (a plan just above
it stays on the dataflow kernel and still agrees)."""
import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import dev, need_gpu, tdtype, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


def _plan(N, n, dt, trace=False, order=None):
    p = btc.btc_plan(N, n, dt)
    if order is not None:
        btc.btc_plan_set_order(p, btc.ORDER_PARTITION, order)
    if trace:
        buf = torch.zeros(4 * (4 * N + 64), dtype=torch.int64, device="cuda")  # above any solve's item count
        btc.btc_plan_set_trace(p, None, buf)
        p._keep = buf
    return p


SIZES = [(1, 8), (2, 16), (3, 32), (17, 12), (64, 16), (100, 24), (128, 32), (129, 8)]


@pytest.mark.parametrize("dt", [btc.F64, btc.F32, btc.MIXED_F32], ids=["f64", "f32", "mixed"])
@pytest.mark.parametrize("N,n", SIZES)
def test_small_solve_is_bitwise_equal_to_the_dataflow_solve(N, n, dt):
    D, B = gen.bt_random(N, n, delta=0.1, seed=3 * N + n)
    b = gen.rhs(N, n, 1, seed=N)
    Dd, Bd = dev(D, tdtype(dt)), dev(B if B.size else np.zeros((1, n, n)), tdtype(dt))
    xs = []
    for trace, sched in ((False, btc.SCHED_FLOW), (True, btc.SCHED_FLOW), (False, btc.SCHED_LEVELS)):
        p = _plan(N, n, dt, trace)
        btc.btc_plan_set_schedule(p, sched)
        btc.btc_factor(p, Dd, Bd)
        assert btc.btc_info(p)[0] == btc.OK
        x = dev(b, tdtype(dt))
        for _ in range(2):  # a second call reuses the wave lists
            x.copy_(dev(b, tdtype(dt)))
            btc.btc_solve(p, x, 1)
        xs.append(x.cpu().numpy())
    np.testing.assert_array_equal(xs[0], xs[1])
    np.testing.assert_array_equal(xs[0], xs[2])
    tol = 1e-12 if dt == btc.F64 else 1e-5
    assert oracle.relres(D, B, xs[0].astype(np.float64), b) <= tol


@pytest.mark.parametrize("dt", [btc.F64, btc.MIXED_F32], ids=["f64", "mixed"])
@pytest.mark.parametrize("N,n", [(5, 8), (64, 16), (127, 32)])
def test_small_solve_tail_after_the_interlaced_factor(N, n, dt):
    D, B = gen.bt_random(N, n, delta=0.1, seed=N + 1)
    b = gen.rhs(N, n, 1, seed=N + 2)
    Dd, Bd = dev(D, tdtype(dt)), dev(B, tdtype(dt))
    out = []
    for trace in (False, True):
        p = _plan(N, n, dt, trace)
        x = dev(b, tdtype(dt))
        btc.btc_factor_solve(p, Dd, Bd, x, 1)
        assert btc.btc_info(p)[0] == btc.OK
        out.append(x.cpu().numpy())
    np.testing.assert_array_equal(out[0], out[1])


@pytest.mark.parametrize("N,n", [(64, 16), (128, 8)])
def test_small_solve_inside_the_refined_solve(N, n):
    D, B = gen.bt_random(N, n, delta=1e-2, seed=N)
    b = gen.rhs(N, n, 1, seed=N + 4)
    Dd, Bd, bd = dev(D, torch.float64), dev(B, torch.float64), dev(b, torch.float64)
    res = []
    for trace in (False, True):
        p = _plan(N, n, btc.MIXED_F32, trace)
        x = torch.zeros_like(bd)
        for _ in range(3):  # the second and third calls replay the captured graph
            x.zero_()
            it, rel, rc = btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, 1, tol=1e-12, maxit=30)
            assert rc == btc.OK and rel <= 1e-12
        res.append((it, x.cpu().numpy()))
    assert res[0][0] == res[1][0]
    np.testing.assert_array_equal(res[0][1], res[1][1])
    assert oracle.relres(D, B, res[0][1], b) <= 1e-12


def test_small_solve_with_the_partition_order():
    N, n, c = 60, 16, 3
    D, B = gen.bt_random(N, n, delta=1.0, seed=9)
    b = gen.rhs(N, n, 1, seed=10)
    Dd, Bd = dev(D, torch.float64), dev(B, torch.float64)
    out = []
    for trace in (False, True):
        p = _plan(N, n, btc.F64, trace, order=c)
        btc.btc_factor(p, Dd, Bd)
        x = dev(b, torch.float64)
        btc.btc_solve(p, x, 1)
        out.append(x.cpu().numpy())
    np.testing.assert_array_equal(out[0], out[1])
    assert oracle.relres(D, B, out[0], b) <= 1e-12
