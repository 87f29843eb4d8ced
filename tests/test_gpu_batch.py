"""Batched plans: many uneven instances in one persistent launch per block-size
group, against single-instance plans (bitwise, same per-node arithmetic) and
against the FP64 oracle; the per-group autotuner (every configuration gives the
same factor) and the captured factor + refined-solve graph (bitwise equal to the
plain launches, replayed with new inputs)."""
import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import dev, need_gpu, tdtype, torch

pytestmark = pytest.mark.gpu

SIZES = [(1, 8), (2, 3), (5, 12), (17, 16), (33, 24), (64, 33), (100, 48), (129, 64), (40, 8), (7, 64), (200, 16),
         (3, 48), (90, 5), (30, 96), (11, 70)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


def _inputs(dt, seed=0, delta=0.1):
    Ds, Bs, bs = [], [], []
    for k, (N, n) in enumerate(SIZES):
        D, B = gen.bt_random(N, n, delta=delta, seed=seed + 31 * k)
        Ds.append(D)
        Bs.append(B if B.size else np.zeros((1, n, n)))
        bs.append(gen.rhs(N, n, 1, seed=seed + k))
    return Ds, Bs, bs


@pytest.mark.parametrize("dt", [btc.F64, btc.F32, btc.MIXED_F32], ids=["f64", "f32", "mixed"])
def test_batch_solve_equals_single_plans(dt):
    Ds, Bs, bs = _inputs(dt)
    t = tdtype(dt)
    Dd = [dev(D, t) for D in Ds]
    Bd = [dev(B, t) for B in Bs]
    bd = [dev(b, t) for b in bs]
    xd = [torch.zeros_like(b) for b in bd]
    batch = btc.btc_batch_plan([N for N, _ in SIZES], [n for _, n in SIZES], dt)
    q = btc.btc_batch_query(batch)
    assert q["groups"] == len({btc.btc_describe(N, n)["np"] for N, n in SIZES})
    btc.btc_batch_factor(batch, Dd, Bd)
    assert btc.btc_batch_info(batch)[0] == btc.OK
    btc.btc_batch_solve(batch, bd, xd)
    for k, (N, n) in enumerate(SIZES):
        p = btc.btc_plan(N, n, dt)
        btc.btc_factor(p, Dd[k], Bd[k])
        x1 = bd[k].clone()
        btc.btc_solve(p, x1, 1)
        np.testing.assert_array_equal(xd[k].cpu().numpy(), x1.cpu().numpy())
        tol = 1e-12 if dt == btc.F64 else 1e-5
        assert oracle.relres(Ds[k], Bs[k][:max(N - 1, 0)], xd[k].cpu().numpy().astype(np.float64), bs[k]) <= tol


@pytest.mark.parametrize("dt", [btc.F64, btc.MIXED_F32], ids=["f64", "mixed"])
def test_batch_refined_reaches_1e10(dt):
    Ds, Bs, bs = _inputs(dt, seed=5, delta=1e-2)
    Dd = [dev(D, torch.float64) for D in Ds]
    Bd = [dev(B, torch.float64) for B in Bs]
    bd = [dev(b, torch.float64) for b in bs]
    xd = [torch.zeros_like(b) for b in bd]
    batch = btc.btc_batch_plan([N for N, _ in SIZES], [n for _, n in SIZES], dt)
    for rep in range(2):  # second pass reuses the plan (flags reset, norms recomputed)
        btc.btc_batch_factor(batch, Dd, Bd)
        it, rel, rc = btc.btc_batch_solve_refined(batch, bd, xd, tol=1e-10, maxit=30)
        assert rc == btc.OK and rel <= 1e-10
    for k, (N, n) in enumerate(SIZES):
        x = xd[k].cpu().numpy()
        assert oracle.relres(Ds[k], Bs[k][:max(N - 1, 0)], x, bs[k]) <= 1e-10
        xo = oracle.solve(Ds[k], Bs[k][:max(N - 1, 0)], bs[k])
        assert np.abs(x - xo).max() <= 1e-8 * np.abs(xo).max()


def test_batch_reports_the_failing_instance():
    Ds, Bs, bs = _inputs(btc.F64, seed=9)
    Ds[6] = Ds[6].copy()
    Ds[6][0] = -np.eye(Ds[6].shape[1])
    batch = btc.btc_batch_plan([N for N, _ in SIZES], [n for _, n in SIZES], btc.F64)
    btc.btc_batch_factor(batch, [dev(D, torch.float64) for D in Ds], [dev(B, torch.float64) for B in Bs])
    rc, k, blk, col = btc.btc_batch_info(batch)
    assert rc == btc.ERR_NOT_SPD and k == 6 and blk == 0 and col == 0


def _dev_inputs(Ds, Bs, bs):
    return ([dev(D, torch.float64) for D in Ds], [dev(B, torch.float64) for B in Bs],
            [dev(b, torch.float64) for b in bs])


@pytest.mark.parametrize("dt", [btc.F64, btc.MIXED_F32], ids=["f64", "mixed"])
def test_batch_tuned_configuration_gives_the_same_factor(dt):
    Ds, Bs, bs = _inputs(dt, seed=13)
    Dd, Bd, bd = _dev_inputs(Ds, Bs, bs)
    out = []
    for tune in (False, True):
        batch = btc.btc_batch_plan([N for N, _ in SIZES], [n for _, n in SIZES], dt)
        btc.btc_batch_set_autotune(batch, tune)
        btc.btc_batch_factor(batch, Dd, Bd)
        xd = [torch.zeros_like(b) for b in bd]
        btc.btc_batch_solve(batch, bd, xd)
        out.append([x.cpu().numpy() for x in xd])
        groups = btc.btc_batch_query(batch)["groups"]
        nps = []
        for g in range(groups):
            np_, cap, ctas, tuned, ms = btc.btc_batch_tuning(batch, g)
            assert tuned == tune and cap >= 1 and ctas >= 1 and (ms > 0) == tune
            nps.append(np_)
        assert sorted(nps) == sorted({btc.btc_describe(N, n)["np"] for N, n in SIZES})
        batch.free()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dt", [btc.F64, btc.MIXED_F32], ids=["f64", "mixed"])
def test_batch_graph_equals_plain_launches_and_replays_new_inputs(dt):
    sets = [_inputs(dt, seed=s, delta=1e-2) for s in (21, 22)]
    plain = []
    for Ds, Bs, bs in sets:  # reference: plain launches
        Dd, Bd, bd = _dev_inputs(Ds, Bs, bs)
        batch = btc.btc_batch_plan([N for N, _ in SIZES], [n for _, n in SIZES], dt)
        btc.btc_batch_set_graphs(batch, False)
        xd = [torch.zeros_like(b) for b in bd]
        it, rel, rc = btc.btc_batch_factor_solve_refined(batch, Dd, Bd, bd, xd, tol=1e-10, maxit=30)
        assert rc == btc.OK and rel <= 1e-10
        plain.append(([x.cpu().numpy() for x in xd], it, rel))
        batch.free()
    batch = btc.btc_batch_plan([N for N, _ in SIZES], [n for _, n in SIZES], dt)
    for rep in range(4):  # tuning pass, capture, replay, replay with the other inputs
        Ds, Bs, bs = sets[rep % 2] if rep >= 2 else sets[0]
        Dd, Bd, bd = _dev_inputs(Ds, Bs, bs)
        xd = [torch.zeros_like(b) for b in bd]
        it, rel, rc = btc.btc_batch_factor_solve_refined(batch, Dd, Bd, bd, xd, tol=1e-10, maxit=30)
        ref = plain[rep % 2] if rep >= 2 else plain[0]
        assert rc == btc.OK and it == ref[1] and rel == ref[2], (rep, it, rel, ref[1:])
        for a, b in zip(xd, ref[0]):
            np.testing.assert_array_equal(a.cpu().numpy(), b)
        for k, (N, n) in enumerate(SIZES):
            assert oracle.relres(Ds[k], Bs[k][:max(N - 1, 0)], xd[k].cpu().numpy(), bs[k]) <= 1e-10
    batch.free()
