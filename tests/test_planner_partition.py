"""Host-side planner of both elimination orders (no GPU): the partition
permutation Psi_p of Sec. 4.1 (Alg. 4, chunk sizes by Proposition 1) and the
nested-dissection order P_inf of Sec. 4.3.

The work items the planner emits are executed here in FP64 on the host, in a
random order that respects only their declared dependencies, with the item
semantics the C-ABI documents (one node's Cholesky, two triangular solves, the
immediate update, the fill block; pull-form forward and backward solve items).
The result must be the oracle's block Cholesky in the same order, and the
solution the oracle's, so a wrong role, slot, orientation or a missing
dependency fails here. Every pair of items that touch the same block (one
writing it) must be ordered by the dependency closure, and every dependency
must lie in an earlier launch level (the per-level schedule)."""
import random

import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, build, gen


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    btc.load()


def _fits(N, c):
    try:
        oracle.partition_sizes(N, c)
        return True
    except ValueError:
        return False


CASES = [(N, c) for N in list(range(1, 48)) + [64, 100, 257, 1000, 4096] for c in range(1, 11) if _fits(N, c)]


@pytest.mark.parametrize("N,c", CASES)
def test_partition_order_is_psi_p(N, c):
    info, order, levels = btc.btc_describe_order(N, 8, btc.F64, btc.ORDER_PARTITION, c)
    ref = list(oracle.partition_order(N, c))
    n1, nk = oracle.partition_sizes(N, c)
    # the chunks are independent, so the launch interleaves them (position by position); each chunk is
    # still eliminated in ascending order and the pivots come last, in order, as in Psi_p
    order = list(order)
    assert sorted(order) == list(range(N))
    chunks = [ref[:n1]] + [ref[n1 + k * nk:n1 + (k + 1) * nk] for k in range(c - 1)]
    for ch in chunks:
        members = set(ch)
        assert [v for v in order if v in members] == ch
    if c > 1:
        assert order[N - (c - 1):] == ref[N - (c - 1):]
    # launch levels: chain positions, then one level per pivot
    assert levels.max() == max(n1, nk) + (c - 1)
    assert np.all(np.diff(levels) >= 0)


@pytest.mark.parametrize("N,c", [(N, c) for (N, c) in CASES if N <= 300])
def test_partition_flop_tallies(N, c):
    n = 16
    info, _, _ = btc.btc_describe_order(N, n, btc.F64, btc.ORDER_PARTITION, c)
    n3 = float(n) ** 3
    _, nk = oracle.partition_sizes(N, c)
    # chunk k >= 2 creates one fill block per member, except the last member of the last chunk
    fill = (c - 1) * nk - 1 if c >= 2 else 0
    assert info["fill_blocks"] == fill
    assert info["offdiag_blocks"] == N - 1 + fill
    assert info["factor_flops"] == pytest.approx((N / 3.0 + 2 * info["offdiag_blocks"] + 2 * fill) * n3)
    if c == 1:  # the natural order is Alg. 1: (7/3 N - 2) n^3 (Sec. 3.1)
        assert info["factor_flops"] == pytest.approx(info["seq_factor_flops"])
    nd = btc.btc_describe(N, n, btc.F64)
    assert info["factor_flops"] <= nd["factor_flops"] + 1e-9 * n3 or c > 2


def test_nd_order_through_describe_order_matches_schedule():
    for N in (1, 2, 7, 64, 129):
        _, order, levels = btc.btc_describe_order(N, 8, btc.F64, btc.ORDER_ND, 0)
        o2, l2 = btc.btc_schedule(N)
        assert list(order) == list(o2) and list(levels) == list(l2)
        assert btc.btc_describe_order(N, 8, btc.F64)[0] == btc.btc_describe(N, 8, btc.F64)


def test_partition_rejections():
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_describe_order(3, 8, btc.F64, btc.ORDER_PARTITION, 3)
    assert ei.value.code == btc.ERR_ARG
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_describe_order(10, 8, btc.F64, btc.ORDER_PARTITION, 0)
    assert ei.value.code == btc.ERR_ARG
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_describe_order(10, 256, btc.MIXED_TF32, btc.ORDER_PARTITION, 2)
    assert ei.value.code == btc.ERR_UNSUPPORTED


# ---------------------------------------------------------------- item emulation

def _closure(deps):
    anc = []
    for i, d in enumerate(deps):
        s = set()
        for x in d:
            if x >= 0:
                assert x < i, (i, list(d))
                s |= anc[x] | {x}
        anc.append(s)
    return anc


def _unordered_conflicts(rw, anc):
    bad = []
    for i in range(len(rw)):
        ri, wi = rw[i]
        for j in range(i):
            rj, wj = rw[j]
            if ((wi & (rj | wj)) or (wj & ri)) and j not in anc[i]:
                bad.append((j, i))
    return bad


def _random_topological(deps, rng):
    n = len(deps)
    done = [False] * n
    out = []
    while len(out) < n:
        ready = [i for i in range(n) if not done[i] and all(d < 0 or done[d] for d in deps[i])]
        i = rng.choice(ready)
        done[i] = True
        out.append(i)
    return out


def _emulate(N, n, order_kind, c, seed):
    fac, sol, slots = btc.btc_schedule_items(N, order_kind, c)
    D, B = gen.bt_random(N, n, delta=1.0, seed=seed)
    rng = random.Random(seed)
    # pools: diagonal blocks in upper form (D_v symmetric), coupling slots in the orientation of the node
    # eliminated first
    dp = [D[v].copy() for v in range(N)]
    ep = [None] * len(slots)
    for s in range(N - 1):
        assert slots[s, 2] in (0, 1)
        ep[s] = B[s].T.copy() if slots[s, 2] else B[s].copy()
    # factor items
    deps = [list(r[11:14]) for r in fac]
    anc = _closure(deps)
    for i, r in enumerate(fac):
        for x in deps[i]:
            assert x < 0 or fac[x, 0] < r[0], "a dependency in the same launch level"
    rw = []
    for r in fac:
        _, ds, dn, ru, rd, pa, pb, fi = (int(v) for v in r[:8])
        rd_set, wr_set = {("d", ds)}, {("d", ds)}
        for q in (pa, pb):
            if q >= 0:
                rd_set.add(("e", q))
        for q in (ru, rd):
            if q >= 0:
                rd_set.add(("e", q))
                wr_set.add(("e", q))
        if dn >= 0:
            rd_set.add(("d", dn))
            wr_set.add(("d", dn))
        if fi >= 0:
            wr_set.add(("e", fi))
        rw.append((rd_set, wr_set))
    assert not _unordered_conflicts(rw, anc)
    assert fac[-1, 10] & 2 and not any(fac[:-1, 10] & 2)
    for i in _random_topological(deps, rng):
        _, ds, dn, ru, rd, pa, pb, fi, _, _, flags = (int(v) for v in fac[i, :11])
        S = dp[ds].copy()
        if pa >= 0:
            S -= ep[pa].T @ ep[pa]
        U = np.linalg.cholesky(S).T
        Zu = Zd = None
        if ru >= 0:
            Zu = ep[ru] = np.linalg.solve(U.T, ep[ru])
        if rd >= 0:
            Zd = ep[rd] = np.linalg.solve(U.T, ep[rd])
        if dn >= 0:
            dp[dn] = dp[dn] - Zd.T @ Zd - (ep[pb].T @ ep[pb] if pb >= 0 else 0.0)
        if fi >= 0:
            ep[fi] = -(Zu.T @ Zd) if flags & 1 else -(Zd.T @ Zu)
        dp[ds] = U
    # solve items
    sdeps = [list(r[7:10]) for r in sol]
    sanc = _closure(sdeps)
    srw = []
    for r in sol:
        ys, ya, _, yb = (int(v) for v in r[:4])
        srw.append(({ys} | {q for q in (ya, yb) if q >= 0}, {ys}))
    assert not _unordered_conflicts(srw, sanc)
    m = 2
    b = gen.rhs(N, n, m, seed=seed + 1)
    y = b.reshape(N, n, m).copy()
    for i in _random_topological(sdeps, rng):
        ys, ya, ea, yb, eb, dsf, kind = (int(v) for v in sol[i, :7])
        if kind == 0:
            for yq, eq in ((ya, ea), (yb, eb)):
                if yq >= 0:
                    y[ys] -= ep[eq].T @ y[yq]
            if dsf >= 0:
                y[ys] = np.linalg.solve(dp[dsf].T, y[ys])
        else:
            for yq, eq in ((ya, ea), (yb, eb)):
                if yq >= 0:
                    y[ys] -= ep[eq] @ y[yq]
            y[ys] = np.linalg.solve(dp[dsf], y[ys])
    return D, B, b, dp, ep, slots, y.reshape(N * n, m)


EMU = [(N, c) for N in (1, 2, 3, 4, 5, 8, 13, 21, 37, 64) for c in (1, 2, 3, 4, 6) if _fits(N, c)]


@pytest.mark.parametrize("N,c", EMU)
def test_partition_items_reproduce_the_oracle_factor_and_solve(N, c):
    n = 3
    D, B, b, dp, ep, slots, x = _emulate(N, n, btc.ORDER_PARTITION, c, seed=7 * N + c)
    order, Ld, pairs, Loff = oracle.partition_factor(D, B, c)
    scale = max(np.abs(Ld).max(), np.abs(Loff).max() if Loff.size else 0.0)
    assert max(np.abs(dp[v].T - Ld[v]).max() for v in range(N)) <= 1e-12 * scale
    ref = {(int(r), int(col)): blk for (r, col), blk in zip(pairs, Loff)}
    assert len(ref) == len(slots)
    for s, (e, o, _) in enumerate(slots):
        # the slot's rows are the variables of e (eliminated first): U(e, o) = L(o, e)^T
        assert np.abs(ep[s].T - ref[(int(o), int(e))]).max() <= 1e-12 * scale
    assert oracle.relres(D, B, x, b) <= 1e-13
    assert np.abs(x - oracle.solve(D, B, b)).max() <= 1e-10 * max(1.0, np.abs(x).max())


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 13, 20, 33, 64])
def test_nd_items_reproduce_the_oracle_factor_and_solve(N):
    n = 3
    D, B, b, dp, ep, slots, x = _emulate(N, n, btc.ORDER_ND, 0, seed=N)
    order, Ld, pairs, Loff = oracle.nd_factor(D, B)
    scale = max(np.abs(Ld).max(), np.abs(Loff).max() if Loff.size else 0.0)
    assert max(np.abs(dp[v].T - Ld[v]).max() for v in range(N)) <= 1e-12 * scale
    ref = {(int(r), int(col)): blk for (r, col), blk in zip(pairs, Loff)}
    for s, (e, o, _) in enumerate(slots):
        assert np.abs(ep[s].T - ref[(int(o), int(e))]).max() <= 1e-12 * scale
    assert oracle.relres(D, B, x, b) <= 1e-13


def test_emulation_catches_a_dropped_dependency(monkeypatch):
    """The hazard check is live: removing one declared dependency of a partition plan is reported."""
    fac, sol, slots = btc.btc_schedule_items(21, btc.ORDER_PARTITION, 3)
    deps = [list(r[11:14]) for r in fac]
    # the first pivot waits on the last node of chunk 3, which also updates the next pivot
    i = [k for k, r in enumerate(fac) if r[10] & 2 == 0 and r[0] == fac[:, 0].max() - 1][0]
    deps[i] = [-1, -1, -1]
    rw = []
    for r in fac:
        _, ds, dn, ru, rd, pa, pb, fi = (int(v) for v in r[:8])
        rd_set = {("d", ds)} | {("e", q) for q in (pa, pb, ru, rd) if q >= 0} | ({("d", dn)} if dn >= 0 else set())
        wr_set = {("d", ds)} | {("e", q) for q in (ru, rd, fi) if q >= 0} | ({("d", dn)} if dn >= 0 else set())
        rw.append((rd_set, wr_set))
    assert _unordered_conflicts(rw, _closure(deps))


# ---------------------------------------------------------------- dispatch model (host only)

def test_dispatch_keeps_nested_dissection_for_a_lone_system():
    for N, n in [(1024, 64), (4096, 16), (100, 128)]:
        assert list(btc.btc_dispatch_orders([N], [n], btc.MIXED_F32)) == [0]


def test_dispatch_takes_cheap_orders_under_instance_parallelism():
    Ns, ns = [64] * 2000, [32] * 2000
    ch = btc.btc_dispatch_orders(Ns, ns, btc.MIXED_F32)
    assert (ch == 1).all()  # work-bound: the natural order of Alg. 1, 2.7x fewer flops


def test_dispatch_on_the_benchmark_mix_is_valid_and_saves_flops():
    specs = gen.batch_specs(512, seed=0)
    Ns, ns = [N for N, _ in specs], [n for _, n in specs]
    ch = btc.btc_dispatch_orders(Ns, ns, btc.MIXED_F32)
    fl_nd = fl = 0.0
    for N, n, c in zip(Ns, ns, ch):
        if c:
            assert _fits(N, int(c))
        fl_nd += btc.btc_describe(N, n, btc.MIXED_F32)["factor_flops"]
        fl += btc.btc_describe_order(N, n, btc.MIXED_F32, btc.ORDER_PARTITION if c else btc.ORDER_ND,
                                     int(c))[0]["factor_flops"]
    assert fl <= fl_nd
    # per block size a threshold policy: the systems that switch are the shortest ones, with one chunk count
    for n in set(ns):
        switched = [(N, c) for N, nn, c in zip(Ns, ns, ch) if nn == n and c > 0]
        kept = [N for N, nn, c in zip(Ns, ns, ch) if nn == n and c == 0]
        if switched and kept:
            assert max(N for N, _ in switched) <= min(kept) or len({c for _, c in switched}) == 1
        assert len({c for _, c in switched}) <= 1
