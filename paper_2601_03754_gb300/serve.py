"""Open-loop load generator for the request server (btc_server_*).

A pool of distinct systems (MPC-like reduced KKT Hessians, n uniform over
{12, 24, 48, 96}, N log-uniform in [50, 5000]) is drawn once on the device;
requests arrive as a Poisson stream (gen.request_stream), 30% of them re-solve
the cached factor of an earlier request with a new right-hand side. Each
request is submitted at its arrival time; latency (completion - submission)
and throughput come from the server's own statistics.
"""
from __future__ import annotations

import time

from . import btc, gen


def make_pool(count=24, seed=0, sizes=(12, 24, 48, 96), nmin=50, nmax=5000, device="cuda"):
    import math

    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    pool = []
    for k in range(count):
        n = int(rng.choice(np.asarray(sizes)))
        N = int(np.clip(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))), nmin, nmax))
        D, B = gen.mpc_torch(N, n, seed=seed * 1000 + k, device=device)
        if B.numel() == 0:
            B = torch.zeros((1, n, n), dtype=torch.float64, device=device)
        pool.append(dict(N=N, n=n, D=D, B=B))
    return pool


def run_stream(server, pool, rate, count, seed=0, tol=1e-10, maxit=30):
    """Submit `count` requests at Poisson arrival times with mean `rate` per second.
    Returns (results, wall seconds, solutions, pool index of each request, right-hand sides, seconds
    from the first to the last submission)."""
    import torch
    reqs = gen.request_stream(rate, count, seed=seed)
    rhs, xs, tickets, which = [], [], [], []
    factor_ticket = {}
    for k, r in enumerate(reqs):
        p = pool[k % len(pool)] if r["resolve_of"] < 0 else pool[which[r["resolve_of"]]]
        which.append(k % len(pool) if r["resolve_of"] < 0 else which[r["resolve_of"]])
        g = torch.Generator(device="cuda")
        g.manual_seed(seed * 100003 + k)
        rhs.append(torch.randn((p["N"] * p["n"],), generator=g, device="cuda", dtype=torch.float64))
        xs.append(torch.zeros_like(rhs[-1]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, r in enumerate(reqs):
        now = time.perf_counter() - t0
        if r["t"] > now:
            time.sleep(r["t"] - now)
        p = pool[which[k]]
        fid = factor_ticket.get(r["resolve_of"], -1) if r["resolve_of"] >= 0 else -1
        t = btc.btc_server_submit(server, p["N"], p["n"], p["D"], p["B"], rhs[k], xs[k], factor_id=fid, tol=tol,
                                  maxit=maxit)
        tickets.append(t)
        if r["resolve_of"] < 0:
            factor_ticket[k] = t
    submit_span = time.perf_counter() - t0
    results = [btc.btc_server_poll(server, t, wait=True) for t in tickets]
    wall = time.perf_counter() - t0
    return results, wall, xs, which, rhs, submit_span


def check_results(pool, xs, which, rhs):
    """Relative residual ||b - Psi x|| / (||Psi|| ||x||) of every returned x, recomputed by the library's
    FP64 residual (btc_residual) on the request's own b, independently of what the server reported."""
    worst = 0.0
    for k, x in enumerate(xs):
        p = pool[which[k]]
        r, a, xn = btc.btc_residual(p["N"], p["n"], 1, p["D"], p["B"], x, rhs[k])
        rel = r / (a * xn) if a * xn > 0 else float("inf")
        if rel != rel:
            rel = float("inf")
        worst = max(worst, rel)
    return {"checked": len(xs), "max_relres_recomputed": worst}
