"""The top-separator Cholesky of the mixed paths in its two precisions (btc_plan_set_root_precision):
FP64 (default) and double-FP32. Both factor the FP32 Schur complement and round the factor back to
FP32, so the top block agrees to FP32 rounding, every other block is untouched, and the refined
solutions agree."""
import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import dev, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


def _run(p, Dd, Bd, bd, m):
    x = torch.zeros_like(bd)
    it, rel, _ = btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, m, tol=1e-11, maxit=40)
    return x.cpu().numpy(), it, rel, btc.btc_get_factor(p)


@pytest.mark.parametrize("dt,N,n,m,delta", [(btc.MIXED_F32, 1, 16, 1, 1.0), (btc.MIXED_F32, 2, 8, 1, 1.0),
                                            (btc.MIXED_F32, 300, 32, 2, 1e-4), (btc.MIXED_F32, 1024, 64, 1, 1.0),
                                            (btc.MIXED_TF32, 129, 128, 1, 1e-2)])
def test_root_precisions_agree(dt, N, n, m, delta):
    D, B = gen.bt_random(N, n, delta=delta, seed=N + n)
    b = gen.rhs(N, n, m, seed=N)
    Dd, Bd = dev(D, torch.float64), dev(B if B.size else np.zeros((1, n, n)), torch.float64)
    bd = dev(b, torch.float64)
    out = {}
    for prec in (btc.ROOT_DOUBLE_FP32, btc.ROOT_FP64):
        p = btc.btc_plan(N, n, dt)
        btc.btc_plan_set_root_precision(p, prec)
        out[prec] = _run(p, Dd, Bd, bd, m)
    (xa, ita, rela, fa), (xb, itb, relb, fb) = out[btc.ROOT_DOUBLE_FP32], out[btc.ROOT_FP64]
    top = (1 << (N.bit_length() - 1)) - 1
    others = [i for i in range(N) if i != top]
    assert np.array_equal(fa[0][others], fb[0][others]) and np.array_equal(fa[1], fb[1])
    ta, tb = fa[0][top].astype(np.float64), fb[0][top].astype(np.float64)
    assert np.abs(ta - tb).max() <= 2.0 ** -22 * np.abs(tb).max()
    assert rela <= 1e-11 and relb <= 1e-11 and ita == itb
    assert np.abs(xa - xb).max() <= 1e-9 * np.abs(xb).max()
    if N <= 300:
        assert oracle.relres(D, B, xb, b) <= 1e-11


def test_switching_precision_recaptures_the_graph():
    N, n, m = 200, 16, 1
    D, B = gen.bt_random(N, n, delta=1e-2, seed=3)
    b = gen.rhs(N, n, m, seed=3)
    Dd, Bd, bd = dev(D, torch.float64), dev(B, torch.float64), dev(b, torch.float64)
    p = btc.btc_plan(N, n, btc.MIXED_F32)
    btc.btc_plan_set_root_precision(p, btc.ROOT_DOUBLE_FP32)
    for _ in range(3):  # tuning, capture, replay
        _run(p, Dd, Bd, bd, m)
    btc.btc_plan_set_root_precision(p, btc.ROOT_FP64)
    q = btc.btc_plan(N, n, btc.MIXED_F32)
    btc.btc_plan_set_root_precision(q, btc.ROOT_FP64)
    btc.btc_plan_set_graphs(q, False)
    ref = _run(q, Dd, Bd, bd, m)
    for _ in range(2):
        got = _run(p, Dd, Bd, bd, m)
        assert np.array_equal(got[0], ref[0]) and got[1:3] == ref[1:3]
        assert np.array_equal(got[3][0], ref[3][0])
    with pytest.raises(btc.BtcError):
        btc.btc_plan_set_root_precision(p, 2)
