"""The fully right-looking variant (Alg. 6: packing pass, immediate atomic
updates of both neighbours) against the oracle and against Alg. 5. Floating-
point atomics make the summation order of the two updates of a block
run-dependent, so the comparisons use the tolerances, not bitwise equality."""
import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import compare_factor_with_oracle, dev, need_gpu, tdtype, torch

pytestmark = pytest.mark.gpu

FACT_TOL = {btc.F64: 1e-11, btc.F32: 5e-5, btc.MIXED_F32: 5e-5}
REC_TOL = {btc.F64: 1e-12, btc.F32: 1e-5, btc.MIXED_F32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


@pytest.mark.parametrize("sched", [btc.SCHED_LEVELS, btc.SCHED_FLOW], ids=["levels", "flow"])
@pytest.mark.parametrize("dt", [btc.F64, btc.F32, btc.MIXED_F32], ids=["f64", "f32", "mixed"])
@pytest.mark.parametrize("N,n", [(1, 8), (2, 5), (7, 16), (33, 24), (100, 64), (257, 12), (30, 96)])
def test_right_looking_factor_matches_oracle(N, n, dt, sched):
    D, B = gen.bt_random(N, n, delta=0.5, seed=N * 7 + n)
    t = tdtype(dt)
    p = btc.btc_plan(N, n, dt)
    btc.btc_plan_set_variant(p, btc.VARIANT_RIGHT_LOOKING)
    btc.btc_plan_set_schedule(p, sched)
    Dd, Bd = dev(D, t), dev(B if B.size else np.zeros((1, n, n)), t)
    btc.btc_factor(p, Dd, Bd)
    assert btc.btc_info(p)[0] == btc.OK
    err, rec = compare_factor_with_oracle(p, D, B, FACT_TOL[dt])
    assert err <= FACT_TOL[dt] and rec <= REC_TOL[dt], (err, rec)
    b = gen.rhs(N, n, 1, seed=N)
    if dt == btc.F32:
        x = dev(b, t)
        btc.btc_solve(p, x, 1)
        assert oracle.relres(D, B, x.cpu().numpy().astype(np.float64), b) <= 1e-5
    else:
        bd = dev(b, torch.float64)
        xd = torch.zeros_like(bd)
        it, rel, rc = btc.btc_solve_refined(p, bd, xd, 1, tol=1e-10, maxit=30)
        assert rc == btc.OK and oracle.relres(D, B, xd.cpu().numpy(), b) <= 1e-10


def test_right_looking_and_hybrid_agree_on_the_benchmark_size():
    N, n = 1024, 64
    D, B = gen.bt_random(N, n, delta=1.0, seed=3)
    b = gen.rhs(N, n, 1, seed=3)
    xs = []
    for variant in (btc.VARIANT_HYBRID, btc.VARIANT_RIGHT_LOOKING):
        p = btc.btc_plan(N, n, btc.F64)
        btc.btc_plan_set_variant(p, variant)
        btc.btc_factor(p, dev(D, torch.float64), dev(B, torch.float64))
        x = dev(b, torch.float64)
        btc.btc_solve(p, x, 1)
        xs.append(x.cpu().numpy())
    assert np.abs(xs[0] - xs[1]).max() <= 1e-12 * np.abs(xs[0]).max()
