"""Request server: continuous batching over worker slots with HBM-footprint
admission and a factor cache. Each result must be the same alone and in a mix
of concurrent requests (bitwise: same kernels, same plan shape, deterministic
schedule), and match the FP64 oracle to the refinement tolerance."""
import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import dev, need_gpu, torch

pytestmark = pytest.mark.gpu

PROBLEMS = [(60, 12), (333, 24), (101, 48), (70, 96), (500, 12), (257, 48), (64, 24), (129, 96)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


def _pool():
    pool = []
    for k, (N, n) in enumerate(PROBLEMS):
        D, B = gen.mpc(N, n, seed=40 + k)
        b = gen.rhs(N, n, 1, seed=80 + k)[:, 0]
        pool.append(dict(N=N, n=n, Dh=D, Bh=B, bh=b, D=dev(D, torch.float64), B=dev(B, torch.float64),
                         b=dev(b, torch.float64)))
    return pool


@pytest.mark.parametrize("dt", [btc.MIXED_F32, btc.F64], ids=["mixed", "f64"])
def test_results_same_alone_and_in_the_mix(dt):
    pool = _pool()
    # alone: one slot, one request at a time
    alone = []
    srv = btc.btc_server_start(dt, slots=1, hbm_budget_bytes=4 << 30, cache_factors=False)
    for p in pool:
        x = torch.zeros_like(p["b"])
        t = btc.btc_server_submit(srv, p["N"], p["n"], p["D"], p["B"], p["b"], x)
        r = btc.btc_server_poll(srv, t)
        assert r["status"] == btc.OK and r["relres"] <= 1e-10
        alone.append(x.cpu().numpy())
    srv.stop()
    # in the mix: 4 slots, every problem submitted 3 times at once, interleaved
    srv = btc.btc_server_start(dt, slots=4, hbm_budget_bytes=4 << 30, cache_factors=False)
    xs, tickets = [], []
    for rep in range(3):
        for k, p in enumerate(pool):
            x = torch.zeros_like(p["b"])
            xs.append((k, x))
            tickets.append(btc.btc_server_submit(srv, p["N"], p["n"], p["D"], p["B"], p["b"], x))
    for t in tickets:
        assert btc.btc_server_poll(srv, t)["status"] == btc.OK
    st = btc.btc_server_stats(srv)
    assert st["completed"] == len(tickets) and st["failed"] == 0 and st["p99_us"] >= st["p50_us"] > 0
    srv.stop()
    for k, x in xs:
        np.testing.assert_array_equal(x.cpu().numpy(), alone[k])
    for k, p in enumerate(pool):
        assert oracle.relres(p["Dh"], p["Bh"], alone[k], p["bh"]) <= 1e-10


def test_resolve_uses_the_cached_factor_and_eviction_recomputes():
    pool = _pool()
    srv = btc.btc_server_start(btc.MIXED_F32, slots=2, hbm_budget_bytes=4 << 30, cache_factors=True)
    p = pool[1]
    x0 = torch.zeros_like(p["b"])
    t0 = btc.btc_server_submit(srv, p["N"], p["n"], p["D"], p["B"], p["b"], x0)
    assert btc.btc_server_poll(srv, t0)["status"] == btc.OK
    b2 = dev(gen.rhs(p["N"], p["n"], 1, seed=999)[:, 0], torch.float64)
    x2 = torch.zeros_like(b2)
    t2 = btc.btc_server_submit(srv, p["N"], p["n"], p["D"], p["B"], b2, x2, factor_id=t0)
    r2 = btc.btc_server_poll(srv, t2)
    assert r2["status"] == btc.OK
    st = btc.btc_server_stats(srv)
    assert st["cache_hits"] == 1
    assert oracle.relres(p["Dh"], p["Bh"], x2.cpu().numpy(), b2.cpu().numpy()) <= 1e-10
    srv.stop()
    # a budget that holds one plan: the cached factor is evicted by the next request,
    # and the re-solve falls back to a fresh factorization (a cache miss)
    one = btc.btc_server_footprint(btc.MIXED_F32, pool[1]["N"], pool[1]["n"])
    other = btc.btc_server_footprint(btc.MIXED_F32, pool[4]["N"], pool[4]["n"])
    srv = btc.btc_server_start(btc.MIXED_F32, slots=1, hbm_budget_bytes=max(one, other) + 1024, cache_factors=True)
    t0 = btc.btc_server_submit(srv, p["N"], p["n"], p["D"], p["B"], p["b"], torch.zeros_like(p["b"]))
    q = pool[4]
    t1 = btc.btc_server_submit(srv, q["N"], q["n"], q["D"], q["B"], q["b"], torch.zeros_like(q["b"]))
    x3 = torch.zeros_like(b2)
    t3 = btc.btc_server_submit(srv, p["N"], p["n"], p["D"], p["B"], b2, x3, factor_id=t0)
    for t in (t0, t1, t3):
        assert btc.btc_server_poll(srv, t)["status"] == btc.OK
    st = btc.btc_server_stats(srv)
    assert st["evictions"] >= 1 and st["cache_misses"] == 1 and st["device_bytes"] <= max(one, other) + 1024
    np.testing.assert_array_equal(x3.cpu().numpy(), x2.cpu().numpy())
    srv.stop()


@pytest.mark.parametrize("dt", [btc.MIXED_F32, btc.F64], ids=["mixed", "f64"])
def test_concurrent_resolves_of_one_cached_factor(dt):
    """Many re-solves of the same cached factor submitted at once to a multi-slot server: they share
    that factor's plan, so the server must run them one at a time; each x must equal the x of the same
    re-solve run alone (bitwise) and meet the tolerance against the oracle."""
    pool = _pool()
    p = pool[5]
    rhs = [dev(gen.rhs(p["N"], p["n"], 1, seed=500 + k)[:, 0], torch.float64) for k in range(12)]
    # alone: each re-solve on its own after the factor request
    srv = btc.btc_server_start(dt, slots=1, hbm_budget_bytes=4 << 30, cache_factors=True)
    t0 = btc.btc_server_submit(srv, p["N"], p["n"], p["D"], p["B"], p["b"], torch.zeros_like(p["b"]))
    assert btc.btc_server_poll(srv, t0)["status"] == btc.OK
    alone = []
    for b in rhs:
        x = torch.zeros_like(b)
        t = btc.btc_server_submit(srv, p["N"], p["n"], p["D"], p["B"], b, x, factor_id=t0)
        assert btc.btc_server_poll(srv, t)["status"] == btc.OK
        alone.append(x.cpu().numpy())
    srv.stop()
    # together: 6 slots, all re-solves of one factor submitted back to back, with other requests between
    srv = btc.btc_server_start(dt, slots=6, hbm_budget_bytes=4 << 30, cache_factors=True)
    t0 = btc.btc_server_submit(srv, p["N"], p["n"], p["D"], p["B"], p["b"], torch.zeros_like(p["b"]))
    assert btc.btc_server_poll(srv, t0)["status"] == btc.OK
    xs, tickets, others = [], [], []
    for k, b in enumerate(rhs):
        x = torch.zeros_like(b)
        xs.append(x)
        tickets.append(btc.btc_server_submit(srv, p["N"], p["n"], p["D"], p["B"], b, x, factor_id=t0))
        if k % 4 == 0:
            q = pool[k % len(pool)]
            others.append(btc.btc_server_submit(srv, q["N"], q["n"], q["D"], q["B"], q["b"],
                                                torch.zeros_like(q["b"])))
    for t in tickets + others:
        assert btc.btc_server_poll(srv, t)["status"] == btc.OK
    st = btc.btc_server_stats(srv)
    assert st["cache_hits"] == len(rhs) and st["failed"] == 0
    srv.stop()
    for k, x in enumerate(xs):
        xh = x.cpu().numpy()
        np.testing.assert_array_equal(xh, alone[k])
        assert oracle.relres(p["Dh"], p["Bh"], xh, rhs[k].cpu().numpy()) <= 1e-10


def test_oversized_request_is_rejected():
    srv = btc.btc_server_start(btc.MIXED_F32, slots=1, hbm_budget_bytes=1 << 20, cache_factors=False)
    D = torch.zeros((1000, 48, 48), dtype=torch.float64, device="cuda")
    b = torch.zeros(1000 * 48, dtype=torch.float64, device="cuda")
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_server_submit(srv, 1000, 48, D, D, b, b)
    assert ei.value.code == btc.ERR_OOM
    srv.stop()


def test_bucketed_plans_serve_smaller_systems_and_prewarm():
    """A plan of a size bucket serves every N up to the bucket, padded: the result equals the result of the
    same request on an exact-size plan to the refinement tolerance, and meets it against the oracle; a
    prewarmed server builds no plan on the request path (its device bytes do not grow)."""
    srv = btc.btc_server_start(btc.MIXED_F32, slots=3, hbm_budget_bytes=8 << 30, cache_factors=True)
    btc.btc_server_prewarm(srv, 24, 400, copies=2)
    before = btc.btc_server_stats(srv)["device_bytes"]
    assert before > 0
    cases = []
    for k, N in enumerate((17, 63, 100, 101, 333, 400)):
        D, B = gen.mpc(N, 24, seed=300 + k)
        b = gen.rhs(N, 24, 1, seed=400 + k)[:, 0]
        cases.append((N, D, B, b))
    outs = []
    for N, D, B, b in cases:
        x = torch.zeros(N * 24, dtype=torch.float64, device="cuda")
        t = btc.btc_server_submit(srv, N, 24, dev(D, torch.float64), dev(B, torch.float64), dev(b, torch.float64), x)
        r = btc.btc_server_poll(srv, t)
        assert r["status"] == btc.OK and r["relres"] <= 1e-10
        outs.append((t, x))
    st = btc.btc_server_stats(srv)
    assert st["device_bytes"] <= before + 1
    # re-solves of the padded cached factors
    for (N, D, B, b), (t, x) in zip(cases, outs):
        xh = x.cpu().numpy()
        assert oracle.relres(D, B, xh, b) <= 1e-10
        b2 = gen.rhs(N, 24, 1, seed=N)[:, 0]
        x2 = torch.zeros_like(x)
        t2 = btc.btc_server_submit(srv, N, 24, dev(D, torch.float64), dev(B, torch.float64), dev(b2, torch.float64),
                                   x2, factor_id=t)
        assert btc.btc_server_poll(srv, t2)["status"] == btc.OK
        assert oracle.relres(D, B, x2.cpu().numpy(), b2) <= 1e-10
    srv.stop()
