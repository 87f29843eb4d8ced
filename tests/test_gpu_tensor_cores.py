"""The tensor-core factorizations (BTC_MIXED_TF32 and BTC_MIXED_BF16, padded
block size 128): tcgen05 products for the deferred syrk, the immediate syrk and
the fill gemm, with TF32 (kind::tf32) or BF16 (kind::f16) operands and FP32
accumulation.

Checked against the oracle's P_inf-order block Cholesky at the operand
format's accuracy (TF32 keeps 10 mantissa bits, unit roundoff 2^-11; BF16 keeps
7, unit roundoff 2^-8, so its bound is 8 times TF32's), through the
FP64-refined solve at the FP64 bar, across schedules (the MMA order is fixed,
so every schedule gives bitwise the same factor), against the FP32 FMA path,
and in batches."""
import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import compare_factor_with_oracle, dev, need_gpu, torch

pytestmark = pytest.mark.gpu

TC = [btc.MIXED_TF32, btc.MIXED_BF16]
TC_IDS = ["tf32", "bf16"]
FACT_TOL = {btc.MIXED_TF32: 5e-3, btc.MIXED_BF16: 4e-2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


def _dev(D, B):
    n = D.shape[1]
    return dev(D, torch.float64), dev(B if B.size else np.zeros((1, n, n)), torch.float64)


@pytest.mark.parametrize("dt", TC, ids=TC_IDS)
@pytest.mark.parametrize("N,n", [(1, 128), (2, 120), (5, 128), (37, 100), (64, 128)])
def test_tc_factor_matches_oracle(N, n, dt):
    D, B = gen.bt_random(N, n, delta=1.0, seed=N + n)
    Dd, Bd = _dev(D, B)
    p = btc.btc_plan(N, n, dt)
    assert btc.btc_plan_query(p)["np"] == 128
    btc.btc_factor(p, Dd, Bd)
    rc, _, _ = btc.btc_info(p)
    assert rc == btc.OK
    err, rec = compare_factor_with_oracle(p, D, B, None)
    # short operands in the products, FP32 elsewhere
    assert err <= FACT_TOL[dt], err
    assert rec <= FACT_TOL[dt], rec


@pytest.mark.parametrize("dt", TC, ids=TC_IDS)
@pytest.mark.parametrize("N,n,m,delta", [(3, 128, 1, 1.0), (129, 128, 2, 1.0), (300, 110, 1, 1e-2),
                                         (1000, 128, 1, 1.0)])
def test_tc_refined_solution_reaches_fp64_accuracy(N, n, m, delta, dt):
    D, B = gen.bt_random(N, n, delta=delta, seed=2 * N + n)
    b = gen.rhs(N, n, m, seed=N)
    Dd, Bd = _dev(D, B)
    bd = dev(b, torch.float64)
    p = btc.btc_plan(N, n, dt)
    x = torch.zeros_like(bd)
    it, rel, _ = btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, m, tol=1e-12, maxit=60)
    assert rel <= 1e-12
    if N <= 300:
        xo = oracle.solve(D, B, b)
        assert np.abs(x.cpu().numpy() - xo).max() <= 1e-8 * max(1.0, np.abs(xo).max())
    # the FP32 FMA path needs no more steps than the tensor-core path
    q = btc.btc_plan(N, n, btc.MIXED_F32)
    x32 = torch.zeros_like(bd)
    it32, rel32, _ = btc.btc_factor_solve_refined(q, Dd, Bd, bd, x32, m, tol=1e-12, maxit=40)
    assert it32 <= it


@pytest.mark.parametrize("dt", TC, ids=TC_IDS)
def test_tc_schedules_are_bitwise_equal(dt):
    N, n = 77, 128
    D, B = gen.bt_random(N, n, delta=1.0, seed=9)
    b = gen.rhs(N, n, 1, seed=9)
    Dd, Bd = _dev(D, B)
    out = []
    for mode, fused in ((btc.SCHED_LEVELS, False), (btc.SCHED_FLOW, False), (btc.SCHED_FLOW, True)):
        p = btc.btc_plan(N, n, dt)
        btc.btc_plan_set_schedule(p, mode)
        x = dev(b, torch.float64)
        if fused:
            btc.btc_factor_solve(p, Dd, Bd, x, 1)
        else:
            btc.btc_factor(p, Dd, Bd)
            btc.btc_solve(p, x, 1)
        assert btc.btc_info(p)[0] == btc.OK
        out.append((btc.btc_get_factor(p), x.cpu().numpy()))
    for f, x in out[1:]:
        assert np.array_equal(f[0], out[0][0][0]) and np.array_equal(f[1], out[0][0][1])
        assert np.array_equal(x, out[0][1])


@pytest.mark.parametrize("dt", TC, ids=TC_IDS)
def test_tc_below_128_is_the_fp32_path(dt):
    N, n = 50, 64
    D, B = gen.bt_random(N, n, delta=1.0, seed=4)
    b = gen.rhs(N, n, 1, seed=4)
    Dd, Bd = _dev(D, B)
    xs = []
    for dt in (dt, btc.MIXED_F32):
        p = btc.btc_plan(N, n, dt)
        x = dev(b, torch.float64)
        btc.btc_factor_solve(p, Dd, Bd, x, 1)
        xs.append(x)
    assert torch.equal(xs[0], xs[1])


@pytest.mark.parametrize("dt", TC, ids=TC_IDS)
def test_tc_batch_matches_single_plans(dt):
    specs = [(40, 128), (9, 16), (130, 100), (1, 128), (64, 64)]
    Ds, Bs, bs = [], [], []
    for k, (N, n) in enumerate(specs):
        D, B = gen.bt_random(N, n, delta=1e-2, seed=50 + k)
        Ds.append(dev(D, torch.float64))
        Bs.append(dev(B if B.size else np.zeros((1, n, n)), torch.float64))
        bs.append(dev(gen.rhs(N, n, 1, seed=k), torch.float64))
    bt = btc.btc_batch_plan([N for N, _ in specs], [n for _, n in specs], dt)
    btc.btc_batch_factor(bt, Ds, Bs)
    xs = [torch.zeros_like(b) for b in bs]
    btc.btc_batch_solve(bt, bs, xs)
    for k, (N, n) in enumerate(specs):
        p = btc.btc_plan(N, n, dt)
        btc.btc_factor(p, Ds[k], Bs[k])
        x = bs[k].clone()
        btc.btc_solve(p, x, 1)
        assert torch.equal(x, xs[k]), k


def test_bf16_and_tf32_factors_differ_at_their_own_precision():
    """The BF16 products are not silently TF32 (or FP32): its factor is further from the oracle than the
    TF32 factor, which is further than the FP32 FMA factor, each within its own bound."""
    N, n = 31, 128
    D, B = gen.bt_random(N, n, delta=1.0, seed=77)
    Dd, Bd = _dev(D, B)
    errs = {}
    for dt in (btc.MIXED_F32, btc.MIXED_TF32, btc.MIXED_BF16):
        p = btc.btc_plan(N, n, dt)
        btc.btc_factor(p, Dd, Bd)
        errs[dt] = compare_factor_with_oracle(p, D, B, None)[0]
    assert errs[btc.MIXED_F32] < errs[btc.MIXED_TF32] < errs[btc.MIXED_BF16] <= FACT_TOL[btc.MIXED_BF16], errs
