"""The persistent dataflow schedule against the level-by-level schedule.

Both schedules run the same per-node arithmetic, so the factor blocks and the
solutions must be bitwise equal; repeated calls exercise the reset of the
completion flags between launches."""
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


def _factor_and_solve(D, B, b, dt, mode, reps=1):
    N, n = D.shape[0], D.shape[1]
    p = btc.btc_plan(N, n, dt)
    btc.btc_plan_set_schedule(p, mode)
    Dd, Bd = dev(D, tdtype(dt)), dev(B if B.size else np.zeros((1, n, n)), tdtype(dt))
    for _ in range(reps):
        btc.btc_factor(p, Dd, Bd)
        x = dev(b, tdtype(dt))
        btc.btc_solve(p, x, b.shape[1])
    rc, blk, col = btc.btc_info(p)
    assert rc == btc.OK
    return btc.btc_get_factor(p), x.cpu().numpy()


@pytest.mark.parametrize("dt", [btc.F64, btc.F32, btc.MIXED_F32], ids=["f64", "f32", "mixed"])
@pytest.mark.parametrize("N,n,m", [(1, 8, 1), (2, 16, 1), (7, 12, 2), (64, 16, 1), (129, 32, 3), (300, 64, 1),
                                   (1024, 8, 1)])
def test_flow_schedule_is_bitwise_equal_to_level_schedule(N, n, m, dt):
    D, B = gen.bt_random(N, n, delta=0.1, seed=N + n)
    b = gen.rhs(N, n, m, seed=N)
    (Dl, Ul, Pl), xl = _factor_and_solve(D, B, b, dt, btc.SCHED_LEVELS)
    (Df, Uf, Pf), xf = _factor_and_solve(D, B, b, dt, btc.SCHED_FLOW, reps=3)
    np.testing.assert_array_equal(Dl, Df)
    np.testing.assert_array_equal(Ul, Uf)
    np.testing.assert_array_equal(xl, xf)
    tol = 1e-12 if dt == btc.F64 else 1e-5
    assert oracle.relres(D, B, xf.astype(np.float64), b) <= tol


def test_flow_refined_solve_full_size():
    N, n = 1024, 64
    D, B = gen.bt_random(N, n, delta=1e-2, seed=77)
    b = gen.rhs(N, n, 1, seed=77)
    p = btc.btc_plan(N, n, btc.MIXED_F32)
    btc.btc_plan_set_schedule(p, btc.SCHED_FLOW)
    Dd, Bd, bd = dev(D, torch.float64), dev(B, torch.float64), dev(b, torch.float64)
    for _ in range(3):
        btc.btc_factor(p, Dd, Bd)
        xd = torch.zeros_like(bd)
        it, rel, rc = btc.btc_solve_refined(p, bd, xd, 1, tol=1e-10, maxit=30)
        assert rc == btc.OK and rel <= 1e-10
    assert oracle.relres(D, B, xd.cpu().numpy(), b) <= 1e-10
