"""Failure detection without a GPU fault.

* Bounded waits: btc_plan_inject_stall makes one factor item of the persistent
  launches wait for a completion flag that no item ever sets, with a poll
  limit of a few thousand polls. The wait must run out, the launch must drain,
  and btc_info, the refined solve and the graph-resident refined factor + solve
  must report BTC_ERR_TIMEOUT within a second; after restoring the plan the
  same plan (same CUDA context) must factor and solve correctly again.
* NaN in the right-hand side: the FP64 residual norms propagate NaN, so a
  refined solve never reports convergence on a NaN residual (single plan,
  graph path, batch), and the residual entry points return a NaN norm.
"""
import time

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


def _case(N, n, seed, m=1):
    D, B = gen.bt_random(N, n, delta=1e-2, seed=seed)
    b = gen.rhs(N, n, m, seed=seed + 1)
    return D, B, b, dev(D, torch.float64), dev(B, torch.float64), dev(b, torch.float64)


@pytest.mark.parametrize("dt,item", [(btc.MIXED_F32, 40), (btc.F64, 63), (btc.MIXED_F32, 0)],
                         ids=["mixed-level2", "f64-root", "mixed-level1"])
def test_stalled_wait_runs_out_and_reports_timeout(dt, item):
    N, n = 64, 16
    D, B, b, Dd, Bd, bd = _case(N, n, seed=5)
    p = btc.btc_plan(N, n, dt)
    btc.btc_plan_set_autotune(p, False)
    btc.btc_plan_inject_stall(p, item, 4096)
    t0 = time.perf_counter()
    btc.btc_factor(p, Dd, Bd)
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_info(p)
    assert ei.value.code == btc.ERR_TIMEOUT
    x = torch.zeros_like(bd)
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_solve_refined(p, bd, x, 1, tol=1e-10, maxit=5)
    assert ei.value.code == btc.ERR_TIMEOUT
    # the interlaced factor + forward launch inside the captured refinement graph
    for _ in range(2):
        with pytest.raises(btc.BtcError) as ei:
            btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, 1, tol=1e-10, maxit=5)
        assert ei.value.code == btc.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    # restored: the same plan and context work again
    btc.btc_plan_inject_stall(p, -1, 0)
    x.zero_()
    it, rel, rc = btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, 1, tol=1e-10, maxit=30)
    assert rc == btc.OK and btc.btc_info(p)[0] == btc.OK
    assert oracle.relres(D, B, x.cpu().numpy(), b) <= 1e-10
    p.free()


def test_stall_hook_rejects_bad_items():
    p = btc.btc_plan(8, 8, btc.MIXED_F32)
    with pytest.raises(btc.BtcError):
        btc.btc_plan_inject_stall(p, 7, 4096)  # the mixed path's top separator has no wait
    with pytest.raises(btc.BtcError):
        btc.btc_plan_inject_stall(p, 2, 10)  # limit below 64
    btc.btc_plan_inject_stall(p, -1, 0)


@pytest.mark.parametrize("graphs", [False, True], ids=["plain", "graph"])
def test_nan_in_rhs_is_never_reported_converged(graphs):
    N, n = 100, 24
    D, B, b, Dd, Bd, bd = _case(N, n, seed=9)
    bd[37 * n + 5, 0] = float("nan")
    p = btc.btc_plan(N, n, btc.MIXED_F32)
    btc.btc_plan_set_graphs(p, graphs)
    x = torch.zeros_like(bd)
    for _ in range(3):  # tuning, capture, replay
        it, rel, rc = btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, 1, tol=1e-10, maxit=5,
                                                   allow_not_converged=True)
        assert rc == btc.ERR_NOT_CONVERGED and rel != rel
    it, rel, rc = btc.btc_solve_refined(p, bd, x, 1, tol=1e-10, maxit=5, allow_not_converged=True)
    assert rc == btc.ERR_NOT_CONVERGED and rel != rel
    # a NaN in one column of several right-hand sides
    b2 = dev(gen.rhs(N, n, 3, seed=3), torch.float64)
    b2[11, 2] = float("nan")
    x2 = torch.zeros_like(b2)
    it, rel, rc = btc.btc_solve_refined(p, b2, x2, 3, tol=1e-10, maxit=5, allow_not_converged=True)
    assert rc == btc.ERR_NOT_CONVERGED and rel != rel


def test_nan_in_batch_rhs_is_never_reported_converged():
    specs = [(40, 8), (70, 16), (33, 32)]
    Ds, Bs, bs, xs = [], [], [], []
    for k, (N, n) in enumerate(specs):
        D, B, b, Dd, Bd, bd = _case(N, n, seed=20 + k)
        Ds.append(Dd)
        Bs.append(Bd)
        bs.append(bd[:, 0].contiguous())
        xs.append(torch.zeros_like(bs[-1]))
    bs[1][17] = float("nan")
    batch = btc.btc_batch_plan([N for N, _ in specs], [n for _, n in specs], btc.MIXED_F32)
    btc.btc_batch_factor(batch, Ds, Bs)
    it, rel, rc = btc.btc_batch_solve_refined(batch, bs, xs, tol=1e-10, maxit=5)
    assert rc == btc.ERR_NOT_CONVERGED and rel != rel
    batch.free()


@pytest.mark.parametrize("where", ["b", "x", "B"])
def test_residual_entry_points_return_nan_norms(where):
    N, n = 50, 12
    D, B, b, Dd, Bd, bd = _case(N, n, seed=31)
    x = dev(gen.rhs(N, n, 1, seed=32), torch.float64)
    target = {"b": bd, "x": x, "B": Bd}[where]
    target.view(-1)[77] = float("nan")
    r1 = btc.btc_residual(N, n, 1, Dd, Bd, x, bd)
    r2 = btc.btc_residual_noalloc(N, n, 1, Dd, Bd, x, bd)
    for r in (r1, r2):
        assert r[0] != r[0], r  # ||b - Psi x||
        if where == "x":
            assert r[2] != r[2], r  # ||x||
        if where == "B":
            assert r[1] != r[1], r  # ||Psi||
