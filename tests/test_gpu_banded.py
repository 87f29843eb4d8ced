"""Block-banded systems (lower block bandwidth w; the conclusion's extension
of the method to wider bands) through btc_banded_*.

The band is grouped on the device into a block-tridiagonal matrix of w-row
super-rows; the grouped blocks must equal the oracle's grouping bit for bit
(pure data movement), and the refined solution must reach the FP64 bar against
the oracle (dense Cholesky of the assembled band at small sizes, the banded
residual at any size). Sizes: w = 1 (block tridiagonal), 2, 3, 4; ragged
groupings (Nb not a multiple of w, padded with identity); every dtype family;
a non-SPD band reports its block row; and the inner plan's partition order."""
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


@pytest.mark.parametrize("dt", [btc.F64, btc.MIXED_F32, btc.MIXED_TF32], ids=["f64", "mixed", "tf32"])
@pytest.mark.parametrize("Nb,b,w,m", [(1, 8, 2, 1), (7, 8, 1, 1), (12, 16, 2, 2), (13, 16, 3, 1), (30, 8, 4, 1),
                                       (64, 32, 2, 1), (50, 24, 4, 3)])
def test_banded_refined_solution_matches_oracle(Nb, b, w, m, dt):
    if dt == btc.F64 and w * b > 96:
        pytest.skip("FP64 blocks up to 96")
    if dt == btc.MIXED_TF32 and w * b < 16:
        pytest.skip("tensor-core sets start at n = 16")
    A = gen.banded(Nb, b, w, delta=1e-2, seed=Nb + w)
    rhs = gen.rhs(Nb, b, m, seed=Nb)
    Ad, bd = dev(A, torch.float64), dev(rhs, torch.float64)
    band = btc.btc_banded_plan(Nb, b, w, dt)
    x = torch.zeros_like(bd)
    for _ in range(2):
        x.zero_()
        it, rel, rc = btc.btc_banded_factor_solve_refined(band, Ad, bd, x, m, tol=1e-12, maxit=40)
        assert rc == btc.OK and rel <= 1e-12
    xh = x.cpu().numpy()
    assert oracle.band_relres(A, xh, rhs) <= 1e-12
    if Nb * b <= 1600:
        xo = oracle.band_solve(A, rhs)
        assert np.abs(xh - xo).max() <= 1e-9 * max(1.0, np.abs(xo).max())
    # a second solve with the stored factor
    x2 = torch.zeros_like(bd)
    it2, rel2, _ = btc.btc_banded_solve_refined(band, bd, x2, m, tol=1e-12, maxit=40)
    assert rel2 <= 1e-12 and oracle.band_relres(A, x2.cpu().numpy(), rhs) <= 1e-12


@pytest.mark.parametrize("Nb,b,w", [(5, 4, 2), (9, 3, 3), (16, 8, 4), (11, 16, 1)])
def test_banded_grouping_equals_the_oracle_grouping(Nb, b, w):
    A = gen.banded(Nb, b, w, seed=7)
    Ad = dev(A, torch.float64)
    band = btc.btc_banded_plan(Nb, b, w, btc.F64)
    btc.btc_banded_factor(band, Ad)
    Dg, Bg = btc.btc_banded_grouped(band)
    Dr, Br = oracle.band_group(A, w)
    assert np.array_equal(Dg, Dr) and np.array_equal(Bg, Br)


def test_banded_full_size_residual():
    Nb, b, w = 2048, 32, 2  # grouped: N = 1024 super-rows of n = 64
    A = gen.banded(Nb, b, w, delta=1e-2, seed=1)
    rhs = gen.rhs(Nb, b, 1, seed=2)
    Ad, bd = dev(A, torch.float64), dev(rhs, torch.float64)
    band = btc.btc_banded_plan(Nb, b, w, btc.MIXED_F32)
    x = torch.zeros_like(bd)
    it, rel, rc = btc.btc_banded_factor_solve_refined(band, Ad, bd, x, 1, tol=1e-10, maxit=30)
    assert rc == btc.OK and rel <= 1e-10
    assert oracle.band_relres(A, x.cpu().numpy(), rhs) <= 1e-10


def test_banded_with_the_partition_order():
    Nb, b, w = 90, 16, 3
    A = gen.banded(Nb, b, w, delta=1e-2, seed=4)
    rhs = gen.rhs(Nb, b, 1, seed=5)
    Ad, bd = dev(A, torch.float64), dev(rhs, torch.float64)
    band = btc.btc_banded_plan(Nb, b, w, btc.MIXED_F32)
    btc.btc_plan_set_order(band.inner, btc.ORDER_PARTITION, 3)
    x = torch.zeros_like(bd)
    it, rel, rc = btc.btc_banded_factor_solve_refined(band, Ad, bd, x, 1, tol=1e-12, maxit=40)
    assert rc == btc.OK and oracle.band_relres(A, x.cpu().numpy(), rhs) <= 1e-12


def test_banded_non_spd_names_the_block_row():
    Nb, b, w = 20, 8, 2
    A = gen.banded(Nb, b, w, seed=6)
    A[0, 13, 3, 3] = -100.0  # block row 13 (super-row 6, second block row in it)
    band = btc.btc_banded_plan(Nb, b, w, btc.F64)
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_banded_factor_solve_refined(band, dev(A, torch.float64), dev(gen.rhs(Nb, b, 1), torch.float64),
                                            torch.zeros((Nb * b, 1), dtype=torch.float64, device="cuda"), 1)
    assert ei.value.code == btc.ERR_NOT_SPD


def test_banded_rejections():
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_banded_plan(10, 64, 3, btc.MIXED_F32)  # n = 192 above 128
    assert ei.value.code == btc.ERR_UNSUPPORTED
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_banded_plan(10, 8, 0, btc.F64)
    assert ei.value.code == btc.ERR_ARG
