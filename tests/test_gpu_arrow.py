"""Bordered ("arrow") systems Psi_a = [[Psi, C^T], [C, A]] (btc_arrow_*): the block-tridiagonal part
factored by the plan (FP64 or a mixed dtype), the border eliminated last with its Schur complement in
FP64. Checked against the oracle's plain definition (Gaussian elimination on the assembled matrix,
itself pinned to LAPACK) element by element, and by the oracle's residual of the bordered system at
larger sizes; edge cases: N = 1, one border row, zero border (decoupled), a border that makes the
matrix indefinite (reported), repeated solves."""
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


def _dev_all(D, B, C, A):
    n = D.shape[1]
    return (dev(D, torch.float64), dev(B if B.size else np.zeros((1, n, n)), torch.float64), dev(C, torch.float64),
            dev(A, torch.float64))


@pytest.mark.parametrize("dt", [btc.F64, btc.MIXED_F32, btc.MIXED_BF16], ids=["f64", "mixed", "bf16"])
@pytest.mark.parametrize("N,n,m", [(1, 4, 1), (2, 3, 2), (9, 8, 5), (17, 16, 8), (33, 12, 16), (20, 64, 33)])
def test_arrow_solution_matches_oracle(N, n, m, dt):
    D, B, C, A = gen.arrow(N, n, m, delta=0.5, seed=N * 7 + m)
    b = np.random.default_rng(N + m).standard_normal(N * n + m)
    a = btc.btc_arrow_plan(N, n, m, dt)
    Dd, Bd, Cd, Ad = _dev_all(D, B, C, A)
    btc.btc_arrow_factor(a, Dd, Bd, Cd, Ad)
    bd = dev(b, torch.float64)
    for _ in range(2):  # repeated solves reuse the factors
        x = torch.zeros_like(bd)
        it, rel, rc = btc.btc_arrow_solve(a, bd, x, tol=1e-12, maxit=10)
        assert rc == btc.OK and rel <= 1e-12
    xh = x.cpu().numpy()
    assert oracle.arrow_relres(D, B, C, A, xh, b) <= 1e-12
    if N * n + m <= 1400:
        xo = oracle.arrow_solve(D, B, C, A, b)
        assert np.abs(xh - xo).max() <= 1e-9 * max(1.0, np.abs(xo).max())


def test_arrow_large_residual_by_oracle():
    N, n, m = 1024, 32, 24
    D, B, C, A = gen.arrow(N, n, m, delta=1e-2, seed=5)
    b = np.random.default_rng(5).standard_normal(N * n + m)
    a = btc.btc_arrow_plan(N, n, m, btc.MIXED_F32)
    mats = _dev_all(D, B, C, A)  # kept alive: the plan reads them again in every solve
    btc.btc_arrow_factor(a, *mats)
    bd = dev(b, torch.float64)
    x = torch.zeros_like(bd)
    it, rel, rc = btc.btc_arrow_solve(a, bd, x, tol=1e-10)
    assert rc == btc.OK and rel <= 1e-10
    assert oracle.arrow_relres(D, B, C, A, x.cpu().numpy(), b) <= 1e-10


def test_arrow_zero_border_decouples():
    N, n, m = 12, 8, 4
    D, B, C, A = gen.arrow(N, n, m, seed=2)
    C = np.zeros_like(C)
    b = np.random.default_rng(2).standard_normal(N * n + m)
    a = btc.btc_arrow_plan(N, n, m, btc.F64)
    mats = _dev_all(D, B, C, A)
    btc.btc_arrow_factor(a, *mats)
    bd = dev(b, torch.float64)
    x = torch.zeros_like(bd)
    btc.btc_arrow_solve(a, bd, x, tol=1e-13)
    xh = x.cpu().numpy()
    np.testing.assert_allclose(xh[:N * n], oracle.solve(D, B, b[:N * n]), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(xh[N * n:], np.linalg.solve(A, b[N * n:]), rtol=1e-10, atol=1e-12)


def test_arrow_indefinite_border_is_reported():
    N, n, m = 10, 4, 3
    D, B, C, A = gen.arrow(N, n, m, seed=3)
    A = A - 1e3 * np.eye(m)  # the Schur complement loses positive definiteness
    a = btc.btc_arrow_plan(N, n, m, btc.MIXED_F32)
    mats = _dev_all(D, B, C, A)
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_arrow_factor(a, *mats)
    assert ei.value.code == btc.ERR_NOT_SPD and "column 0" in str(ei.value)
    x = torch.zeros(N * n + m, dtype=torch.float64, device="cuda")
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_arrow_solve(a, x, x)
    assert ei.value.code == btc.ERR_NOT_FACTORED


def test_arrow_arguments():
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_arrow_plan(10, 8, 65, btc.F64)
    assert ei.value.code == btc.ERR_UNSUPPORTED
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_arrow_plan(10, 8, 4, btc.F32)
    assert ei.value.code == btc.ERR_ARG
