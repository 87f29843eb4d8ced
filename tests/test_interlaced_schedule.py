"""Host-side checks of the interlaced factorization + forward substitution
schedule (btc_schedule_interlaced), no GPU needed.

The forward substitution of Alg. 7 at level l for node j (a multiple of
s = 2^(l-1)) reads y_{j-h} and y_{j+h} (h = s/2, finished at level l-1), the
coupling blocks U(j-h, j), U(j+h, j) (written when nodes j-h, j+h are
eliminated at level l-1, Alg. 5) and, if j is eliminated at level l, its own
factor U_j. The interlaced launch must make every forward item wait, directly
or transitively, for each of those producers, and every factor item for the
level-(l-1) eliminations that update its blocks (e-h, e+h, and e+3h whose
coupling block is the deferred update of S_{e+s}). These sets are derived here
from the elimination order alone (node e is eliminated at level
1 + trailing zeros of e) and checked against the dependency closure of the
exported schedule.
"""
import numpy as np
import pytest

from paper_2601_03754_gb300 import btc


def elim_level(e):
    return (e & -e).bit_length()


def closure(deps):
    """(entries complete before t starts, entries whose factor blocks are stored before t starts). A
    dependency d >= 0 waits for entry d to complete; d <= -2 only for the factor blocks of entry -d-2."""
    full, core = [], []
    for t in range(len(deps)):
        f, c = set(), set()
        for d in deps[t]:
            if d == -1:
                continue
            q = int(d) if d >= 0 else -int(d) - 2
            assert q < t, "a dependency must be an earlier entry"
            f |= full[q]
            c |= core[q]
            (f if d >= 0 else c).add(q)
        full.append(f)
        core.append(c | f)
    return full, core


@pytest.mark.parametrize("N", [1, 2, 3, 7, 8, 13, 64, 100, 257])
@pytest.mark.parametrize("root_separate", [False, True])
def test_interlaced_schedule_dependencies(N, root_separate):
    kind, node, level, deps, tail = btc.btc_schedule_interlaced(N, root_separate)
    L = N.bit_length()  # floor(log2 N) + 1 levels
    root = 1 << (L - 1)
    entry = {}
    for t, (k, j, l) in enumerate(zip(kind, node, level)):
        key = (int(k), int(j), int(l))
        assert key not in entry, f"duplicate entry {key}"
        entry[key] = t
    # factor entries: every node at its elimination level (the root is separate on the mixed path)
    want_fac = {(0, e, elim_level(e)) for e in range(1, N + 1) if not (root_separate and e == root)}
    assert {k for k in entry if k[0] == 0} == want_fac
    # forward entries: (j, l) for j a multiple of s with work to do
    want_fwd = set()
    for l in range(1, L + 1):
        s = 1 << (l - 1)
        for j in range(s, N + 1, s):
            if l == 1 and j % 2 == 0:
                continue  # a level-1 survivor receives nothing
            if root_separate and l == L:
                continue  # the top separator's forward item runs in the tail
            want_fwd.add((1, j, l))
    assert {k for k in entry if k[0] == 1} == want_fwd
    full, core = closure(deps)
    for (k, j, l), t in entry.items():
        s, h = 1 << (l - 1), (1 << (l - 1)) // 2
        need_full, need_core = [], []
        if k == 0 and l > 1:
            # e-h and e+h update S_e and write the fill blocks it reads; of e+3h only the deferred block
            # (a factor block) is read
            need_full = [(0, c, l - 1) for c in (j - h, j + h) if 1 <= c <= N]
            need_core = [(0, c, l - 1) for c in (j + 3 * h,) if 1 <= c <= N]
        if k == 1:
            if elim_level(j) == l:
                need_core.append((0, j, l))
            if l > 1:
                for c in (j - h, j + h):
                    if 1 <= c <= N:
                        need_core.append((0, c, l - 1))
                        need_full.append((1, c, l - 1))
                need_full += [(1, j, lp) for lp in range(1, l) if (1, j, lp) in entry]
        for q in need_full:
            assert entry[q] in full[t], f"{(k, j, l)} does not wait for {q} to complete"
        for q in need_core:
            assert entry[q] in core[t], f"{(k, j, l)} does not wait for the factor blocks of {q}"
    assert tail == N + (1 if root_separate else 0)


def test_interlaced_schedule_orders_levels():
    """Factor items of level l precede the forward items of level l, which precede level l+1."""
    kind, node, level, deps, _ = btc.btc_schedule_interlaced(1024, True)
    key = level * 2 + kind
    assert np.all(np.diff(key) >= 0)
