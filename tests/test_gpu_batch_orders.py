"""Batches with an elimination order per instance (nested dissection, or the
partition permutation of Sec. 4.1 with c chunks) and the dispatch model that
chooses them.

Parity: every instance's solution bitwise equal to a single plan set to the
same order (same per-node arithmetic; the batched packing pass converts the
inputs exactly as the single plan's does), the FP64-refined solutions against
the oracle, the captured graph against the plain launches, and a dispatched
batch of the benchmark's size mix against the oracle's residual."""
import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import dev, need_gpu, tdtype, torch

pytestmark = pytest.mark.gpu

SIZES = [(1, 8), (2, 3), (5, 12), (17, 16), (33, 24), (64, 33), (100, 48), (129, 64), (40, 8), (7, 64), (200, 16),
         (3, 48), (90, 5), (30, 96), (11, 70)]
CHUNKS = [1, 1, 2, 0, 3, 4, 0, 8, 1, 2, 16, 1, 5, 2, 0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


def _inputs(seed=0, delta=0.1):
    Ds, Bs, bs = [], [], []
    for k, (N, n) in enumerate(SIZES):
        D, B = gen.bt_random(N, n, delta=delta, seed=seed + 31 * k)
        Ds.append(D)
        Bs.append(B if B.size else np.zeros((1, n, n)))
        bs.append(gen.rhs(N, n, 1, seed=seed + k))
    return Ds, Bs, bs


@pytest.mark.parametrize("dt", [btc.F64, btc.F32, btc.MIXED_F32], ids=["f64", "f32", "mixed"])
def test_batch_orders_equal_single_plans(dt):
    Ds, Bs, bs = _inputs()
    t = tdtype(dt)
    Dd = [dev(D, t) for D in Ds]
    Bd = [dev(B, t) for B in Bs]
    bd = [dev(b, t) for b in bs]
    xd = [torch.zeros_like(b) for b in bd]
    batch = btc.btc_batch_plan([N for N, _ in SIZES], [n for _, n in SIZES], dt, chunks=CHUNKS)
    assert list(btc.btc_batch_orders(batch)) == CHUNKS
    btc.btc_batch_factor(batch, Dd, Bd)
    assert btc.btc_batch_info(batch)[0] == btc.OK
    btc.btc_batch_solve(batch, bd, xd)
    for k, (N, n) in enumerate(SIZES):
        p = btc.btc_plan(N, n, dt)
        if CHUNKS[k]:
            btc.btc_plan_set_order(p, btc.ORDER_PARTITION, CHUNKS[k])
        btc.btc_factor(p, Dd[k], Bd[k])
        x1 = bd[k].clone()
        btc.btc_solve(p, x1, 1)
        np.testing.assert_array_equal(xd[k].cpu().numpy(), x1.cpu().numpy())
        tol = 1e-12 if dt == btc.F64 else 1e-5
        assert oracle.relres(Ds[k], Bs[k][:max(N - 1, 0)], xd[k].cpu().numpy().astype(np.float64), bs[k]) <= tol


@pytest.mark.parametrize("graphs", [False, True], ids=["plain", "graph"])
def test_batch_orders_refined_reach_fp64(graphs):
    dt = btc.MIXED_F32
    Ds, Bs, bs = _inputs(seed=5, delta=1e-2)
    Dd = [dev(D, torch.float64) for D in Ds]
    Bd = [dev(B, torch.float64) for B in Bs]
    bd = [dev(b, torch.float64) for b in bs]
    batch = btc.btc_batch_plan([N for N, _ in SIZES], [n for _, n in SIZES], dt, chunks=CHUNKS)
    btc.btc_batch_set_graphs(batch, graphs)
    for _ in range(2):
        xd = [torch.zeros_like(b) for b in bd]
        it, worst, rc = btc.btc_batch_factor_solve_refined(batch, Dd, Bd, bd, xd, tol=1e-12, maxit=40)
        assert rc == btc.OK and worst <= 1e-12
        for k, (N, n) in enumerate(SIZES):
            assert oracle.relres(Ds[k], Bs[k][:max(N - 1, 0)], xd[k].cpu().numpy(), bs[k]) <= 1e-12


def test_dispatched_wide_batch_reaches_fp64():
    # many identical short systems: the model takes the partition order
    specs = [(64, 32)] * 1500 + [(40, 16)] * 500
    Ns, ns = [N for N, _ in specs], [n for _, n in specs]
    chunks = btc.btc_dispatch_orders(Ns, ns, btc.MIXED_F32)
    assert (chunks > 0).any()
    Ds, Bs, bs = [], [], []
    for k, (N, n) in enumerate(specs):
        D, B = gen.bt_random_torch(N, n, delta=1e-2, seed=k)
        Ds.append(D)
        Bs.append(B if N > 1 else torch.zeros((1, n, n), dtype=torch.float64, device="cuda"))
        bs.append(torch.randn((N * n, 1), dtype=torch.float64, device="cuda"))
    batch = btc.btc_batch_plan(Ns, ns, btc.MIXED_F32, chunks=chunks)
    xd = [torch.zeros_like(b) for b in bs]
    it, worst, rc = btc.btc_batch_factor_solve_refined(batch, Ds, Bs, bs, xd, tol=1e-10, maxit=30)
    assert rc == btc.OK and worst <= 1e-10
    for k in range(0, len(specs), 97):  # recomputed by the oracle on the host
        N = Ns[k]
        assert oracle.relres(Ds[k].cpu().numpy(), Bs[k].cpu().numpy()[:max(N - 1, 0)], xd[k].cpu().numpy(),
                             bs[k].cpu().numpy()) <= 1e-10


def test_batch_orders_reject_too_many_chunks():
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_batch_plan([5, 9], [8, 8], btc.MIXED_F32, chunks=[0, 9])
    assert ei.value.code == btc.ERR_ARG
