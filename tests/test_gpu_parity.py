"""GPU parity of the nested-dissection factor + solve against the FP64 oracle.

Tolerances (from the accuracy targets of the method's plain and mixed paths):
  * FP64 factor: relative residual and relative reconstruction error <= 1e-12;
  * plain FP32: both <= 1e-5;
  * mixed FP32 + FP64 refinement: relative residual <= 1e-10 after refinement.
Element-wise factor parity uses max |L_gpu - L_oracle| / max |L_oracle| with
1e-11 (FP64) and 5e-5 (FP32), on inputs with delta = 1 (well conditioned).
"""
import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import compare_factor_with_oracle, dev, factor_on_gpu, need_gpu, tdtype, torch

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 16), (2, 3), (3, 8), (5, 12), (7, 16), (16, 5), (20, 24), (33, 32), (64, 16), (100, 48),
          (129, 64), (257, 8), (9, 96), (40, 80), (3, 65)]
FACT_TOL = {btc.F64: 1e-11, btc.F32: 5e-5, btc.MIXED_F32: 5e-5}
REC_TOL = {btc.F64: 1e-12, btc.F32: 1e-5, btc.MIXED_F32: 1e-5}
RES_TOL = {btc.F64: 1e-12, btc.F32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


@pytest.mark.parametrize("dt", [btc.F64, btc.F32, btc.MIXED_F32], ids=["f64", "f32", "mixed"])
@pytest.mark.parametrize("N,n", SHAPES)
def test_factor_blocks_match_oracle(N, n, dt):
    D, B = gen.bt_random(N, n, delta=1.0, seed=N * 100 + n)
    p, Dd, Bd = factor_on_gpu(D, B, dt)
    rc, blk, col = btc.btc_info(p)
    assert rc == btc.OK and blk == -1
    err, rec = compare_factor_with_oracle(p, D, B, FACT_TOL[dt])
    assert err <= FACT_TOL[dt], err
    assert rec <= REC_TOL[dt], rec


@pytest.mark.parametrize("dt", [btc.F64, btc.F32], ids=["f64", "f32"])
@pytest.mark.parametrize("N,n,m", [(1, 4, 1), (3, 8, 2), (64, 16, 1), (100, 12, 3), (129, 64, 1), (65, 33, 16),
                                   (40, 7, 17), (33, 96, 3), (20, 72, 1)])
def test_solve_residual_and_solution(N, n, m, dt):
    D, B = gen.bt_random(N, n, delta=1.0, seed=7 + N + n)
    b = gen.rhs(N, n, m, seed=N)
    p, Dd, Bd = factor_on_gpu(D, B, dt)
    x = dev(b, tdtype(dt))
    btc.btc_solve(p, x, m)
    xh = x.cpu().numpy().astype(np.float64)
    rel = oracle.relres(D, B, xh, b)
    assert rel <= RES_TOL[dt], rel
    xo = oracle.solve(D, B, b)
    fwd = np.abs(xh - xo).max() / np.abs(xo).max()
    assert fwd <= (1e-11 if dt == btc.F64 else 1e-4), fwd


@pytest.mark.parametrize("delta", [1.0, 1e-2, 1e-4])
@pytest.mark.parametrize("dt", [btc.F64, btc.MIXED_F32], ids=["f64", "mixed"])
def test_refined_solve_reaches_1e10(dt, delta):
    N, n, m = 96, 32, 2
    D, B = gen.bt_random(N, n, delta=delta, seed=11)
    b = gen.rhs(N, n, m, seed=12)
    p, Dd, Bd = factor_on_gpu(D, B, dt)
    bd = dev(b, torch.float64)
    xd = torch.zeros_like(bd)
    it, rel, rc = btc.btc_solve_refined(p, bd, xd, m, tol=1e-10, maxit=30)
    assert rc == btc.OK and rel <= 1e-10
    xh = xd.cpu().numpy()
    assert oracle.relres(D, B, xh, b) <= 1e-10  # independently re-evaluated on the host
    if dt == btc.F64:
        assert it <= 1


def test_mpc_variant_mixed():
    N, n = 200, 16
    D, B = gen.mpc(N, n, seed=3)
    b = gen.rhs(N, n, 1, seed=4)
    p, Dd, Bd = factor_on_gpu(D, B, btc.MIXED_F32)
    bd = dev(b, torch.float64)
    xd = torch.zeros_like(bd)
    it, rel, rc = btc.btc_solve_refined(p, bd, xd, 1, tol=1e-10, maxit=30)
    assert rel <= 1e-10
    xo = oracle.solve(D, B, b)
    assert np.abs(xd.cpu().numpy() - xo).max() / np.abs(xo).max() < 1e-8


def test_repeated_solves_reuse_the_factor():
    N, n = 50, 16
    D, B = gen.bt_random(N, n, seed=5)
    p, Dd, Bd = factor_on_gpu(D, B, btc.F64)
    for s in range(3):
        b = gen.rhs(N, n, 1, seed=100 + s)
        x = dev(b, torch.float64)
        btc.btc_solve(p, x, 1)
        assert oracle.relres(D, B, x.cpu().numpy(), b) <= 1e-12


def test_refactor_with_new_values_in_same_plan():
    N, n = 37, 24
    p = btc.btc_plan(N, n, btc.F64)
    for seed in (1, 2):
        D, B = gen.bt_random(N, n, seed=seed)
        Dd, Bd = dev(D, torch.float64), dev(B, torch.float64)
        btc.btc_factor(p, Dd, Bd)
        err, rec = compare_factor_with_oracle(p, D, B, 1e-11)
        assert err <= 1e-11 and rec <= 1e-12


def test_upper_triangle_of_D_is_ignored():
    N, n = 9, 12
    D, B = gen.bt_random(N, n, seed=6)
    Dg = D.copy()
    for i in range(N):
        Dg[i][np.triu_indices(n, 1)] = np.nan
    p, Dd, Bd = factor_on_gpu(Dg, B, btc.F64)
    err, rec = compare_factor_with_oracle(p, D, B, 1e-11)
    assert err <= 1e-11


@pytest.mark.parametrize("bad_node", [0, 5, 8])
def test_not_spd_is_reported(bad_node):
    N, n = 9, 8  # P_inf: level 1 = 1,3,5,7,9; level 2 = 2,6; level 3 = 4; level 4 = 8 (1-based)
    D, B = gen.bt_random(N, n, seed=7)
    D[bad_node] = -np.eye(n) * 50.0
    p, Dd, Bd = factor_on_gpu(D, B, btc.F64)
    rc, blk, col = btc.btc_info(p)
    assert rc == btc.ERR_NOT_SPD
    # the reported (node, column) is the smallest failing one; the planted node's own
    # first pivot is -50 - ... < 0, so it always fails at column 0
    assert blk <= bad_node
    assert col >= 0
    if bad_node == 0:
        assert (blk, col) == (0, 0)
    x = dev(gen.rhs(N, n, 1), torch.float64)
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_solve_refined(p, x, torch.zeros_like(x), 1)
    assert ei.value.code == btc.ERR_NOT_SPD


def test_nan_input_is_reported():
    N, n = 6, 8
    D, B = gen.bt_random(N, n, seed=8)
    D[2, 3, 3] = np.nan
    p, Dd, Bd = factor_on_gpu(D, B, btc.F32)
    rc, blk, col = btc.btc_info(p)
    assert rc == btc.ERR_NOT_SPD and blk <= 2


def test_solve_before_factor_is_rejected():
    p = btc.btc_plan(4, 4, btc.F64)
    x = torch.zeros(16, 1, dtype=torch.float64, device="cuda")
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_solve(p, x, 1)
    assert ei.value.code == btc.ERR_NOT_FACTORED


def test_device_residual_matches_oracle():
    N, n, m = 40, 24, 3
    D, B = gen.bt_random(N, n, seed=9)
    x = gen.rhs(N, n, m, seed=1)
    b = gen.rhs(N, n, m, seed=2)
    r, a, xn = btc.btc_residual(N, n, m, dev(D, torch.float64), dev(B, torch.float64), dev(x, torch.float64),
                                dev(b, torch.float64))
    ro, ao, xo = oracle.resid(D, B, x, b)
    assert abs(r - ro) <= 1e-13 * ro and abs(a - ao) <= 1e-14 * ao and xn == xo


@pytest.mark.parametrize("dt", [btc.F64, btc.MIXED_F32, btc.F32], ids=["f64", "mixed", "f32"])
def test_host_buffer_entry_point(dt):
    N, n, m = 70, 16, 2
    D, B = gen.bt_random(N, n, seed=10)
    b = gen.rhs(N, n, m, seed=10)
    p = btc.btc_plan(N, n, dt)
    if dt == btc.F32:
        Dh, Bh, bh = D.astype(np.float32), B.astype(np.float32), b.astype(np.float32)
    else:
        Dh, Bh, bh = D, B, b
    x = np.zeros_like(bh)
    it, rel, rc = btc.btc_factor_solve_host(p, Dh, Bh, bh, x, m)
    assert oracle.relres(D, B, x.astype(np.float64), b) <= (1e-5 if dt == btc.F32 else 1e-10)


def test_full_size_c2_against_oracle():
    """N = 1024, n = 64 (the benchmark workload) in FP64: every factor block against the
    oracle's full P_inf-order factor, and the solution against the sequential oracle."""
    N, n = 1024, 64
    D, B = gen.bt_random(N, n, delta=1.0, seed=2024)
    b = gen.rhs(N, n, 1, seed=2024)
    p, Dd, Bd = factor_on_gpu(D, B, btc.F64)
    err, rec = compare_factor_with_oracle(p, D, B, 1e-11)
    assert err <= 1e-11 and rec <= 1e-12
    x = dev(b, torch.float64)
    btc.btc_solve(p, x, 1)
    assert oracle.relres(D, B, x.cpu().numpy(), b) <= 1e-12


@pytest.mark.parametrize("N", [257, 1024])
def test_refinement_on_ill_conditioned_block_laplacian(N):
    """D_i = 2I + small SPD perturbation, B_i = -I: kappa ~ 4 (N+1)^2 / pi^2 (4e5 at N=1024)."""
    n = 16
    rng = np.random.default_rng(N)
    M = rng.standard_normal((N, n, n)) * 0.05
    D = 2.0 * np.eye(n)[None] + M @ np.swapaxes(M, 1, 2) / n
    B = np.tile(-np.eye(n), (N - 1, 1, 1))
    b = gen.rhs(N, n, 1, seed=N)
    for dt in (btc.F64, btc.MIXED_F32):
        p, Dd, Bd = factor_on_gpu(D, B, dt)
        bd = dev(b, torch.float64)
        xd = torch.zeros_like(bd)
        it, rel, rc = btc.btc_solve_refined(p, bd, xd, 1, tol=1e-10, maxit=50)
        assert rc == btc.OK and rel <= 1e-10
        assert oracle.relres(D, B, xd.cpu().numpy(), b) <= 1e-10


@pytest.mark.parametrize("dt", [btc.F32, btc.MIXED_F32], ids=["f32", "mixed"])
@pytest.mark.parametrize("N,n", [(1, 128), (5, 128), (37, 100), (130, 128)])
def test_block_size_128(N, n, dt):
    D, B = gen.bt_random(N, n, delta=1.0, seed=N + n)
    p, Dd, Bd = factor_on_gpu(D, B, dt)
    assert btc.btc_info(p)[0] == btc.OK
    err, rec = compare_factor_with_oracle(p, D, B, FACT_TOL[dt])
    assert err <= FACT_TOL[dt] and rec <= REC_TOL[dt], (err, rec)
    b = gen.rhs(N, n, 2, seed=N)
    if dt == btc.MIXED_F32:
        bd = dev(b, torch.float64)
        xd = torch.zeros_like(bd)
        it, rel, rc = btc.btc_solve_refined(p, bd, xd, 2, tol=1e-10, maxit=30)
        assert rc == btc.OK and oracle.relres(D, B, xd.cpu().numpy(), b) <= 1e-10
    else:
        x = dev(b, torch.float32)
        btc.btc_solve(p, x, 2)
        assert oracle.relres(D, B, x.cpu().numpy().astype(np.float64), b) <= 1e-5


def test_f64_plans_stop_at_96():
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_plan(4, 128, btc.F64)
    assert ei.value.code == btc.ERR_UNSUPPORTED
