"""Blocked 256 x 256 nodes (padded block size 256, BTC_MIXED_TF32 and BTC_MIXED_BF16):
every node of Alg. 5 runs as tile tasks on 128 x 128 tiles in one persistent
launch (deferred products, blocked Cholesky, column strips of the two
triangular solves, next-diagonal and fill products; products on tcgen05).

Parity: every factor block against the oracle's P_inf-order block Cholesky at
the operand format's tolerance (the same bounds as the 128 x 128 tensor-core
path: TF32 5e-3, BF16 8 times that), the reconstruction identity on the GPU's
own blocks, the FP64-refined solution at the FP64 bar against the oracle, at
sizes with one, two and several levels, ragged n (129, 200) and N = 1 (the
top separator alone). At N = 1024 the refined residual is recomputed by the
oracle on the host. Edge cases: a non-SPD input reports its failing block and
column (columns past 128 come from the second diagonal tile)."""
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
@pytest.mark.parametrize("N,n", [(1, 256), (2, 256), (3, 200), (6, 256), (13, 129), (17, 256)])
def test_blocked_factor_matches_oracle(N, n, dt):
    D, B = gen.bt_random(N, n, delta=1.0, seed=3 * N + n)
    Dd, Bd = _dev(D, B)
    p = btc.btc_plan(N, n, dt)
    assert btc.btc_plan_query(p)["np"] == 256
    btc.btc_factor(p, Dd, Bd)
    rc, blk, col = btc.btc_info(p)
    assert rc == btc.OK and blk == -1
    err, rec = compare_factor_with_oracle(p, D, B, None)
    assert err <= FACT_TOL[dt], err
    assert rec <= FACT_TOL[dt], rec


@pytest.mark.parametrize("dt", TC, ids=TC_IDS)
@pytest.mark.parametrize("N,n,m,delta", [(1, 256, 1, 1.0), (5, 256, 2, 1e-3), (33, 256, 1, 1.0), (40, 160, 1, 1e-6)])
def test_blocked_refined_solution_reaches_fp64_accuracy(N, n, m, delta, dt):
    D, B = gen.bt_random(N, n, delta=delta, seed=N + 5 * n)
    b = gen.rhs(N, n, m, seed=N + 1)
    Dd, Bd = _dev(D, B)
    bd = dev(b, torch.float64)
    p = btc.btc_plan(N, n, dt)
    x = torch.zeros_like(bd)
    for _ in range(2):  # a second call reuses the plan
        x.zero_()
        it, rel, rc = btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, m, tol=1e-12, maxit=60)
        assert rc == btc.OK and rel <= 1e-12
    xh = x.cpu().numpy()
    assert oracle.relres(D, B, xh, b) <= 1e-12
    xo = oracle.solve(D, B, b)
    assert np.abs(xh - xo).max() <= 1e-8 * max(1.0, np.abs(xo).max())


@pytest.mark.parametrize("dt", TC, ids=TC_IDS)
def test_blocked_full_size_refined_residual(dt):
    N, n = 1024, 256
    D, B = gen.bt_random_torch(N, n, delta=1e-3, seed=11)
    g = torch.Generator(device="cuda")
    g.manual_seed(12)
    b = torch.randn((N * n, 1), generator=g, device="cuda", dtype=torch.float64)
    x = torch.zeros_like(b)
    p = btc.btc_plan(N, n, dt)
    it, rel, rc = btc.btc_factor_solve_refined(p, D, B, b, x, 1, tol=1e-10, maxit=60)
    assert rc == btc.OK and rel <= 1e-10
    # recomputed independently by the oracle on the host
    assert oracle.relres(D.cpu().numpy(), B.cpu().numpy(), x.cpu().numpy(), b.cpu().numpy()) <= 1e-10
    p.free()


@pytest.mark.parametrize("dt", TC, ids=TC_IDS)
def test_blocked_tc_products_are_the_operand_precision(dt):
    """The blocked path's factor error against the oracle tracks its operand format: BF16 is further
    from the oracle than TF32 (both within bound), as for the 128 x 128 kernels."""
    N, n = 9, 256
    D, B = gen.bt_random(N, n, delta=1.0, seed=90)
    Dd, Bd = _dev(D, B)
    errs = {}
    for d in TC:
        p = btc.btc_plan(N, n, d)
        btc.btc_factor(p, Dd, Bd)
        errs[d] = compare_factor_with_oracle(p, D, B, None)[0]
    assert errs[btc.MIXED_TF32] < errs[btc.MIXED_BF16] <= FACT_TOL[btc.MIXED_BF16], errs


@pytest.mark.parametrize("col", [5, 200])
def test_blocked_non_spd_reports_block_and_column(col):
    N, n = 6, 256
    D, B = gen.bt_random(N, n, delta=1.0, seed=4)
    D[2, col, col] = -50.0  # node 2 (eliminated at level 1)
    Dd, Bd = _dev(D, B)
    p = btc.btc_plan(N, n, btc.MIXED_TF32)
    btc.btc_factor(p, Dd, Bd)
    rc, blk, c = btc.btc_info(p)
    assert rc == btc.ERR_NOT_SPD and blk == 2 and c == col


def test_blocked_sizes_are_tensor_core_dtypes_only():
    assert btc.btc_describe(10, 256, btc.MIXED_BF16)["np"] == 256
    for dt in (btc.F64, btc.F32, btc.MIXED_F32):
        with pytest.raises(btc.BtcError) as ei:
            btc.btc_describe(10, 200, dt)
        assert ei.value.code == btc.ERR_UNSUPPORTED
    with pytest.raises(btc.BtcError):
        btc.btc_batch_plan([4, 5], [256, 16], btc.MIXED_TF32)
