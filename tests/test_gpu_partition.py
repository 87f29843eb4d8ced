"""The partition elimination order Psi_p (Sec. 4.1, Alg. 4; chunk sizes by
Proposition 1) on the GPU, through btc_plan_set_order.

Parity: every factor block against the oracle's block Cholesky in the same
order (FP64 plans at 1e-12 relative to max|L|, FP32 operands at 1e-5), the
solution against the oracle's, and the FP64-refined solutions of the mixed
paths (FP32, TF32, BF16 factors with the FP64 top separator) at the FP64 bar.
Sizes: a single chunk (the natural order of Alg. 1), two to eight chunks,
ragged chunk splits, N = 1 and 2, both schedules (per-level launches and the
persistent kernel), the host-buffer entry point, and switching a plan back to
the nested-dissection order. Edge cases: a non-SPD block reports its block and
column; too many chunks, the right-looking variant and blocked 256 plans are
rejected."""
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


def _dev(D, B, dt):
    n = D.shape[1]
    return dev(D, tdtype(dt)), dev(B if B.size else np.zeros((1, n, n)), tdtype(dt))


def _compare(p, D, B, chunks):
    """(max abs error of every factor block relative to max|L|, reconstruction error)."""
    Dh, U, pairs = btc.btc_get_factor(p)
    order, Ld, opairs, Loff = oracle.partition_factor(D, B, chunks)
    scale = max(np.abs(Ld).max(), np.abs(Loff).max() if Loff.size else 0.0)
    err = np.abs(Dh.astype(np.float64) - Ld).max() / scale
    ref = {(int(r), int(c)): blk for (r, c), blk in zip(opairs, Loff)}
    assert len(ref) == len(pairs)
    gp, gb = [], []
    for (e, o), u in zip(pairs, U):
        blk = ref[(int(o), int(e))]
        err = max(err, np.abs(u.astype(np.float64).T - blk).max() / scale)
        gp.append((int(o), int(e)))
        gb.append(u.astype(np.float64).T)
    rec = oracle.bs_reconstruct(D, B, order, Dh.astype(np.float64), np.array(gp, dtype=np.int32).reshape(-1, 2),
                                np.array(gb).reshape(-1, D.shape[1], D.shape[1]))
    return err, rec


SIZES = [(1, 16, 1), (2, 16, 1), (9, 32, 1), (9, 32, 2), (37, 24, 3), (64, 64, 4), (100, 16, 8), (31, 128, 2)]


@pytest.mark.parametrize("sched", [btc.SCHED_LEVELS, btc.SCHED_FLOW], ids=["levels", "flow"])
@pytest.mark.parametrize("N,n,c", SIZES)
def test_partition_factor_f64_matches_oracle(N, n, c, sched):
    if n > 96:
        pytest.skip("FP64 kernels up to n = 96")
    D, B = gen.bt_random(N, n, delta=1.0, seed=N + 3 * c)
    Dd, Bd = _dev(D, B, btc.F64)
    p = btc.btc_plan(N, n, btc.F64)
    btc.btc_plan_set_order(p, btc.ORDER_PARTITION, c)
    btc.btc_plan_set_schedule(p, sched)
    btc.btc_factor(p, Dd, Bd)
    rc, blk, col = btc.btc_info(p)
    assert rc == btc.OK and blk == -1
    err, rec = _compare(p, D, B, c)
    assert err <= 1e-12 and rec <= 1e-13, (err, rec)
    # the solve (persistent pull-form items) against the oracle
    b = gen.rhs(N, n, 3, seed=N)
    x = dev(b, torch.float64)
    btc.btc_solve(p, x, 3)
    xo = oracle.solve(D, B, b)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-10 * max(1.0, np.abs(xo).max())


@pytest.mark.parametrize("N,n,c", [(9, 32, 2), (37, 24, 3), (64, 64, 4), (31, 128, 2)])
def test_partition_factor_f32_matches_oracle(N, n, c):
    D, B = gen.bt_random(N, n, delta=1.0, seed=N + 5 * c)
    Dd, Bd = _dev(D, B, btc.F32)
    p = btc.btc_plan(N, n, btc.F32)
    btc.btc_plan_set_order(p, btc.ORDER_PARTITION, c)
    btc.btc_factor(p, Dd, Bd)
    assert btc.btc_info(p)[0] == btc.OK
    err, rec = _compare(p, D, B, c)
    assert err <= 1e-5 and rec <= 1e-5, (err, rec)


MIXED = [btc.MIXED_F32, btc.MIXED_TF32, btc.MIXED_BF16]


@pytest.mark.parametrize("dt", MIXED, ids=["f32", "tf32", "bf16"])
@pytest.mark.parametrize("N,n,c,m", [(1, 16, 1, 1), (2, 8, 1, 1), (50, 64, 1, 1), (129, 64, 3, 2), (257, 32, 6, 1),
                                     (40, 128, 2, 1)])
def test_partition_refined_solution_reaches_fp64(N, n, c, m, dt):
    if dt != btc.MIXED_F32 and n < 16:
        pytest.skip("tensor-core sets start at n = 16")
    D, B = gen.bt_random(N, n, delta=1e-2, seed=2 * N + c)
    b = gen.rhs(N, n, m, seed=N + 9)
    Dd, Bd = _dev(D, B, btc.F64)
    bd = dev(b, torch.float64)
    p = btc.btc_plan(N, n, dt)
    btc.btc_plan_set_order(p, btc.ORDER_PARTITION, c)
    x = torch.zeros_like(bd)
    for _ in range(2):  # the second call reuses the plan (and its tuned configuration)
        x.zero_()
        it, rel, rc = btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, m, tol=1e-12, maxit=60)
        assert rc == btc.OK and rel <= 1e-12
    xh = x.cpu().numpy()
    assert oracle.relres(D, B, xh, b) <= 1e-12
    xo = oracle.solve(D, B, b)
    assert np.abs(xh - xo).max() <= 1e-8 * max(1.0, np.abs(xo).max())


@pytest.mark.parametrize("pinned", [False, True], ids=["pageable", "pinned"])
def test_partition_host_entry_point(pinned):
    """Host buffers in, host solution out; only the lower triangles of D are read (the upper ones are NaN)."""
    N, n, c = 65, 32, 3
    D, B = gen.bt_random(N, n, delta=1e-2, seed=5)
    b = gen.rhs(N, n, 1, seed=6)
    Dg = D.copy()
    for i in range(N):
        Dg[i][np.triu_indices(n, 1)] = np.nan
    p = btc.btc_plan(N, n, btc.MIXED_F32)
    btc.btc_plan_set_order(p, btc.ORDER_PARTITION, c)
    if pinned:
        Dh, Bh, bh = (torch.from_numpy(a).pin_memory() for a in (Dg, B, b))
        xh = torch.zeros((N * n, 1), dtype=torch.float64).pin_memory()
    else:
        Dh, Bh, bh, xh = Dg, B, b, np.zeros_like(b)
    it, rel, rc = btc.btc_factor_solve_host(p, Dh, Bh, bh, xh, 1, 1e-11, 60)
    x = xh.numpy() if pinned else xh
    assert rc == btc.OK and rel <= 1e-11
    assert oracle.relres(D, B, x, b) <= 1e-11


def test_switching_back_to_nd_restores_the_nd_factor():
    from gpu_helpers import compare_factor_with_oracle
    N, n = 33, 32
    D, B = gen.bt_random(N, n, delta=1.0, seed=8)
    Dd, Bd = _dev(D, B, btc.F64)
    p = btc.btc_plan(N, n, btc.F64)
    nd_blocks = btc.btc_plan_query(p)["offdiag_blocks"]
    btc.btc_plan_set_order(p, btc.ORDER_PARTITION, 3)
    btc.btc_factor(p, Dd, Bd)
    assert _compare(p, D, B, 3)[0] <= 1e-12
    btc.btc_plan_set_order(p, btc.ORDER_ND, 0)
    assert btc.btc_plan_query(p)["offdiag_blocks"] == nd_blocks
    btc.btc_factor(p, Dd, Bd)
    err, rec = compare_factor_with_oracle(p, D, B, None)
    assert err <= 1e-12 and rec <= 1e-13


@pytest.mark.parametrize("bad", [0, 7, 20])
def test_partition_non_spd_reports_block_and_column(bad):
    N, n, c = 21, 16, 3
    D, B = gen.bt_random(N, n, delta=1.0, seed=4)
    D[bad, 5, 5] = -80.0
    Dd, Bd = _dev(D, B, btc.F64)
    p = btc.btc_plan(N, n, btc.F64)
    btc.btc_plan_set_order(p, btc.ORDER_PARTITION, c)
    btc.btc_factor(p, Dd, Bd)
    rc, blk, col = btc.btc_info(p)
    assert rc == btc.ERR_NOT_SPD
    # the smallest failing node is reported; node `bad` fails, and node 0 (the first of chunk 1) sees D_0
    # itself, so it fails exactly at column 5
    assert 0 <= blk <= bad and col >= 0
    if bad == 0:
        assert (blk, col) == (0, 5)
    with pytest.raises(oracle.NotSPD):
        oracle.partition_factor(D, B, c)


def test_partition_rejections_on_a_plan():
    p = btc.btc_plan(5, 16, btc.F64)
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_plan_set_order(p, btc.ORDER_PARTITION, 4)
    assert ei.value.code == btc.ERR_ARG
    btc.btc_plan_set_order(p, btc.ORDER_PARTITION, 2)
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_plan_set_variant(p, btc.VARIANT_RIGHT_LOOKING)
    assert ei.value.code == btc.ERR_UNSUPPORTED
    q = btc.btc_plan(5, 256, btc.MIXED_TF32)
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_plan_set_order(q, btc.ORDER_PARTITION, 2)
    assert ei.value.code == btc.ERR_UNSUPPORTED
