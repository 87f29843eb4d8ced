"""The interlaced factorization + forward substitution (btc_factor_solve,
btc_factor_solve_refined) against the separate calls.

A forward item performs the same arithmetic whether it runs inside the
factorization's persistent launch or in the solve's, so the factor blocks and
the solutions must be bitwise equal to btc_factor followed by btc_solve (or
btc_solve_refined); the refined results are also checked against the oracle's
solution. Repeated calls exercise the reset of the completion flags."""
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


def _inputs(N, n, m, seed, delta=1.0):
    D, B = gen.bt_random(N, n, delta=delta, seed=seed)
    b = gen.rhs(N, n, m, seed=seed)
    return D, B, b


def _dev_inputs(D, B, dt):
    n = D.shape[1]
    return dev(D, tdtype(dt)), dev(B if B.size else np.zeros((1, n, n)), tdtype(dt))


@pytest.mark.parametrize("dt", [btc.F64, btc.F32, btc.MIXED_F32], ids=["f64", "f32", "mixed"])
@pytest.mark.parametrize("N,n,m", [(1, 8, 1), (2, 16, 1), (3, 8, 2), (7, 12, 2), (64, 16, 1), (129, 32, 3),
                                   (300, 64, 1), (257, 48, 5), (1024, 8, 1)])
def test_factor_solve_is_bitwise_equal_to_separate_calls(N, n, m, dt):
    D, B, b = _inputs(N, n, m, seed=N + n + m)
    Dd, Bd = _dev_inputs(D, B, dt)
    p1 = btc.btc_plan(N, n, dt)
    btc.btc_factor(p1, Dd, Bd)
    x1 = dev(b, tdtype(dt))
    btc.btc_solve(p1, x1, m)
    p2 = btc.btc_plan(N, n, dt)
    for _ in range(2):
        x2 = dev(b, tdtype(dt))
        btc.btc_factor_solve(p2, Dd, Bd, x2, m)
    for p in (p1, p2):
        rc, _, _ = btc.btc_info(p)
        assert rc == btc.OK
    assert torch.equal(x1, x2)
    f1, f2 = btc.btc_get_factor(p1), btc.btc_get_factor(p2)
    assert np.array_equal(f1[0], f2[0]) and np.array_equal(f1[1], f2[1])
    # the factor left by the interlaced call serves later solves
    x3 = dev(b, tdtype(dt))
    btc.btc_solve(p2, x3, m)
    assert torch.equal(x1, x3)


@pytest.mark.parametrize("dt", [btc.F64, btc.MIXED_F32], ids=["f64", "mixed"])
@pytest.mark.parametrize("N,n,m,delta", [(1, 16, 1, 1.0), (5, 8, 1, 1.0), (100, 24, 2, 1e-2), (513, 64, 1, 1.0),
                                         (200, 96, 1, 1e-4)])
def test_factor_solve_refined_matches_separate_calls_and_oracle(N, n, m, delta, dt):
    D, B, b = _inputs(N, n, m, seed=3 * N + n, delta=delta)
    Dd, Bd = _dev_inputs(D, B, dt)
    bd = dev(b, torch.float64)
    p1 = btc.btc_plan(N, n, dt)
    btc.btc_factor(p1, Dd, Bd)
    x1 = torch.zeros_like(bd)
    it1, rel1, _ = btc.btc_solve_refined(p1, bd, x1, m, tol=1e-12)
    p2 = btc.btc_plan(N, n, dt)
    x2 = torch.zeros_like(bd)
    it2, rel2, _ = btc.btc_factor_solve_refined(p2, Dd, Bd, bd, x2, m, tol=1e-12)
    assert torch.equal(x1, x2) and it1 == it2 and rel1 == rel2
    assert rel2 <= 1e-12
    xo = oracle.solve(D, B, b)
    assert np.abs(x2.cpu().numpy() - xo).max() <= 1e-8 * max(1.0, np.abs(xo).max())


def test_fallback_paths_give_the_same_results():
    """Level schedule, right-looking variant and more columns than one pass fall back to separate calls."""
    N, n = 77, 16
    D, B, _ = _inputs(N, n, 1, seed=11)
    dt = btc.MIXED_F32
    Dd, Bd = _dev_inputs(D, B, dt)
    ref = btc.btc_plan(N, n, dt)
    mmax = 17  # above the 16 columns of one pass
    b = gen.rhs(N, n, mmax, seed=5)
    btc.btc_factor(ref, Dd, Bd)
    xr = dev(b, torch.float64)
    btc.btc_solve(ref, xr, mmax)
    for setup in (lambda p: btc.btc_plan_set_schedule(p, btc.SCHED_LEVELS),
                  lambda p: None):
        p = btc.btc_plan(N, n, dt)
        setup(p)
        x = dev(b, torch.float64)
        btc.btc_factor_solve(p, Dd, Bd, x, mmax)
        assert torch.equal(x, xr)
    p = btc.btc_plan(N, n, dt)
    btc.btc_plan_set_variant(p, btc.VARIANT_RIGHT_LOOKING)
    x = dev(b[:, :1], torch.float64)
    btc.btc_factor_solve(p, Dd, Bd, x, 1)
    xo = oracle.solve(D, B, b[:, :1])
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-3 * np.abs(xo).max()


def test_factor_solve_reports_a_failed_pivot():
    N, n = 33, 8
    D, B, b = _inputs(N, n, 1, seed=2)
    D[17] = -np.eye(n)  # node 18 (1-based) is not positive definite
    Dd, Bd = _dev_inputs(D, B, btc.MIXED_F32)
    p = btc.btc_plan(N, n, btc.MIXED_F32)
    x = torch.zeros(N * n, 1, dtype=torch.float64, device="cuda")
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_factor_solve_refined(p, Dd, Bd, dev(b, torch.float64), x, 1)
    assert ei.value.code == btc.ERR_NOT_SPD
