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
# A factor item runs in phases separated by four events: S (its dependencies' factor blocks are
# stored: it reads the deferred blocks P_a, P_b), B (its complete-dependencies are done: it reads
# S_e, S_{e+s} and the off-diagonal blocks), C (its factor blocks U_e, U(e, up), U(e, down) are
# stored and published), E (its trailing products, the next diagonal block and the fill, are
# written). A dependency d >= 0 orders E_d before B and C_d before S; d <= -2 orders only C_(-d-2)
# before S.

def _decode(d):
    d = int(d)
    return (None, None) if d == -1 else ((d, "full") if d >= 0 else (-d - 2, "core"))


def _event_graph(deps):
    n = len(deps)
    S, B, C, E = (lambda i: 4 * i), (lambda i: 4 * i + 1), (lambda i: 4 * i + 2), (lambda i: 4 * i + 3)
    succ = [[] for _ in range(4 * n)]
    for i in range(n):
        succ[S(i)].append(B(i))
        succ[B(i)].append(C(i))
        succ[C(i)].append(E(i))
        for d in deps[i]:
            q, kind = _decode(d)
            if q is None:
                continue
            assert q < i, (i, list(deps[i]))
            succ[C(q)].append(S(i))
            if kind == "full":
                succ[E(q)].append(B(i))
    # reachability (events are numbered in a topological order: every edge goes forward)
    reach = [None] * (4 * n)
    for v in reversed(range(4 * n)):
        r = {v}
        for w in succ[v]:
            r |= reach[w]
        reach[v] = r
    return succ, reach, (S, B, C, E)


def _factor_accesses(r, ev):
    S, B, C, E = ev
    _, ds, dn, ru, rd, pa, pb, fi = (int(v) for v in r[:8])
    acc = []  # (block, writes, first event, last event) for item i (filled by the caller)
    for q in (pa, pb):
        if q >= 0:
            acc.append((("e", q), False, S, B))
    acc.append((("d", ds), True, B, C))
    for q in (ru, rd):
        if q >= 0:
            acc.append((("e", q), True, B, C))
    if dn >= 0:
        acc.append((("d", dn), True, B, E))
    if fi >= 0:
        acc.append((("e", fi), True, C, E))
    return acc


def _factor_hazards(fac):
    deps = [list(r[11:14]) for r in fac]
    succ, reach, ev = _event_graph(deps)
    items = []
    for i, r in enumerate(fac):
        for blk, w, a, b in _factor_accesses(r, ev):
            items.append((i, blk, w, a(i), b(i)))
    bad = []
    for x in range(len(items)):
        i, bx, wx, ax, zx = items[x]
        for y in range(x):
            j, by, wy, ay, zy = items[y]
            if i == j or bx != by or not (wx or wy):
                continue
            if ay not in reach[zx] and ax not in reach[zy]:
                bad.append((j, i, bx))
    return bad, succ


def _random_topological_events(succ, rng):
    n = len(succ)
    indeg = [0] * n
    for v in range(n):
        for w in succ[v]:
            indeg[w] += 1
    ready = [v for v in range(n) if indeg[v] == 0]
    out = []
    while ready:
        v = ready.pop(rng.randrange(len(ready)))
        out.append(v)
        for w in succ[v]:
            indeg[w] -= 1
            if indeg[w] == 0:
                ready.append(w)
    assert len(out) == n
    return out


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
    # factor items: every dependency in an earlier launch level, every conflicting pair of accesses ordered
    for i, r in enumerate(fac):
        for x in r[11:14]:
            q, _ = _decode(x)
            assert q is None or fac[q, 0] < r[0], "a dependency in the same launch level"
    bad, succ = _factor_hazards(fac)
    assert not bad, bad[:5]
    assert fac[-1, 10] & 2 and not any(fac[:-1, 10] & 2)
    state = {}
    for v in _random_topological_events(succ, rng):
        i, phase = divmod(v, 4)
        _, ds, dn, ru, rd, pa, pb, fi, _, _, flags = (int(x) for x in fac[i, :11])
        st = state.setdefault(i, {})
        if phase == 0:  # S: the deferred products
            st["acc"] = -(ep[pa].T @ ep[pa]) if pa >= 0 else 0.0
            st["accb"] = -(ep[pb].T @ ep[pb]) if pb >= 0 else 0.0
        elif phase == 1:  # B .. C: Cholesky, triangular solves, factor blocks stored
            U = np.linalg.cholesky(dp[ds] + st["acc"]).T
            st["Zu"] = np.linalg.solve(U.T, ep[ru]) if ru >= 0 else None
            st["Zd"] = np.linalg.solve(U.T, ep[rd]) if rd >= 0 else None
            st["dn"] = dp[dn].copy() if dn >= 0 else None
            dp[ds] = U
            if ru >= 0:
                ep[ru] = st["Zu"]
            if rd >= 0:
                ep[rd] = st["Zd"]
        elif phase == 3:  # C .. E: trailing products
            if dn >= 0:
                dp[dn] = st["dn"] + st["accb"] - st["Zd"].T @ st["Zd"]
            if fi >= 0:
                ep[fi] = -(st["Zu"].T @ st["Zd"]) if flags & 1 else -(st["Zd"].T @ st["Zu"])
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


def test_emulation_catches_a_dropped_or_weakened_dependency():
    """The hazard check is live: removing a declared dependency of a partition plan, or weakening a
    nested-dissection dependency on a complete item to its factor blocks only, is reported."""
    fac, sol, slots = btc.btc_schedule_items(21, btc.ORDER_PARTITION, 3)
    # the first pivot waits on the last node of chunk 3, which also updates the next pivot
    i = [k for k, r in enumerate(fac) if r[10] & 2 == 0 and r[0] == fac[:, 0].max() - 1][0]
    assert not _factor_hazards(fac)[0]
    bad = fac.copy()
    bad[i, 11:14] = -1
    assert _factor_hazards(bad)[0]
    fac, sol, slots = btc.btc_schedule_items(16, btc.ORDER_ND, 0)
    assert not _factor_hazards(fac)[0]
    k = [t for t, r in enumerate(fac) if r[11] >= 0][0]  # a level-2 item's dependency on its left neighbour
    weak = fac.copy()
    weak[k, 11] = -weak[k, 11] - 2
    assert _factor_hazards(weak)[0]
    # the planner's own weak dependency (e+3h: only its factor blocks are read) passes
    assert any((r[11:14] <= -2).any() for r in fac)


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
