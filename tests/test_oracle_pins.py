"""Pins for the FP64 CPU oracle (no GPU).

Each check compares the oracle with something other than itself:
  * LAPACK (numpy.linalg) for the dense Cholesky and dense solves,
  * hand-derived fixtures under tests/golden/ (each with its citation),
  * closed forms (Toeplitz kron I spectrum; scalar Thomas recurrence),
  * structural facts of the multi-stage permutation (fill pattern, counts),
  * invariants (log-det of every ordering, uniqueness of the Cholesky factor).

The mutation tests at the end plant plausible mistakes (transposed operand,
dropped term, wrong sign, wrong stride) in a copy of the oracle's C source and
check that at least one pin fails for each.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import gen


# ---------------------------------------------------------------- helpers ---

def permuted_dense(A, order, n):
    idx = np.concatenate([np.arange(o * n, (o + 1) * n) for o in order])
    return A[np.ix_(idx, idx)]


def predicted_nd_pairs(N):
    """Off-diagonal blocks of the P_inf factor, predicted from Sec. 4.3:
    at level l (stride s = 2^(l-1)) the surviving nodes s, 2s, 3s, ... couple
    pairwise as (k s, (k+1) s), k = 1 .. floor(N/s) - 1 (1-based). In the factor
    the nonzero block sits in the column of whichever of the two is eliminated
    at that level (the odd multiple of s). Returned as 0-based (row, col)."""
    out = set()
    s = 1
    while s <= N:
        for k in range(1, N // s):
            a, b = k * s, (k + 1) * s
            col, row = (a, b) if k % 2 == 1 else (b, a)
            out.add((row - 1, col - 1))
        s *= 2
    return out


def thomas(d, e, rhs):
    """Scalar symmetric tridiagonal solve T_N(d, e) y = rhs (textbook recurrence)."""
    N = len(rhs)
    c = np.zeros(N)
    g = np.zeros(N)
    c[0] = e / d
    g[0] = rhs[0] / d
    for i in range(1, N):
        den = d - e * c[i - 1]
        c[i] = e / den
        g[i] = (rhs[i] - e * g[i - 1]) / den
    y = np.zeros(N)
    y[-1] = g[-1]
    for i in range(N - 2, -1, -1):
        y[i] = g[i] - c[i] * y[i + 1]
    return y


# ------------------------------------------------------------ pin checks ---
# Each returns None on success and raises AssertionError (or an oracle error) otherwise.

def check_chol_vs_lapack(seed=0):
    rng = np.random.default_rng(seed)
    for n in (1, 2, 3, 7, 16):
        M = rng.standard_normal((n, n))
        A = M @ M.T + n * np.eye(n)
        np.testing.assert_allclose(oracle.chol(A), np.linalg.cholesky(A), rtol=1e-13, atol=1e-13)


def check_seq_factor_vs_dense(N=6, n=3, seed=1):
    D, B = gen.bt_random(N, n, delta=0.5, seed=seed)
    Dh, Eh = oracle.seq_factor(D, B)
    A = oracle.assemble(D, B)
    Lref = np.linalg.cholesky(A)
    for i in range(N):
        np.testing.assert_allclose(Dh[i], Lref[i * n:(i + 1) * n, i * n:(i + 1) * n], rtol=1e-12, atol=1e-12)
    for i in range(N - 1):
        np.testing.assert_allclose(Eh[i], Lref[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n], rtol=1e-12,
                                   atol=1e-12)


def check_seq_solve_vs_lapack(N=5, n=3, m=2, seed=2):
    D, B = gen.bt_random(N, n, delta=0.1, seed=seed)
    b = gen.rhs(N, n, m, seed=seed)
    x = oracle.solve(D, B, b)
    A = oracle.assemble(D, B)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(x, oracle.gepp_solve(A, b), rtol=1e-10, atol=1e-12)


def check_nd_factor_vs_dense(N=11, n=2, seed=3):
    D, B = gen.bt_random(N, n, delta=0.2, seed=seed)
    order, Ld, pairs, Loff = oracle.nd_factor(D, B)
    A = oracle.assemble(D, B)
    L = np.linalg.cholesky(permuted_dense(A, order, n))
    pos = np.empty(N, dtype=int)
    pos[order] = np.arange(N)
    for i in range(N):
        p = pos[i]
        np.testing.assert_allclose(Ld[i], L[p * n:(p + 1) * n, p * n:(p + 1) * n], rtol=1e-12, atol=1e-12)
    seen = set()
    for (r, c), blk in zip(pairs, Loff):
        pr, pc = pos[r], pos[c]
        assert pr > pc
        np.testing.assert_allclose(blk, L[pr * n:(pr + 1) * n, pc * n:(pc + 1) * n], rtol=1e-11, atol=1e-12)
        seen.add((pr, pc))
    # every nonzero block of the dense factor is listed
    for pr in range(N):
        for pc in range(pr):
            if np.abs(L[pr * n:(pr + 1) * n, pc * n:(pc + 1) * n]).max() > 1e-12:
                assert (pr, pc) in seen


def check_resid_vs_dense(N=4, n=3, m=2, seed=4):
    D, B = gen.bt_random(N, n, delta=1.0, seed=seed)
    # make the upper triangles of D garbage: only the lower triangle may be read
    Dg = D.copy()
    for i in range(N):
        Dg[i][np.triu_indices(n, 1)] = 1e3
    x = gen.rhs(N, n, m, seed=seed + 1)
    b = gen.rhs(N, n, m, seed=seed + 2)
    A = oracle.assemble(D, B)
    r, a, xn = oracle.resid(Dg, B, x, b)
    assert math.isclose(r, np.abs(b - A @ x).max(), rel_tol=1e-12)
    assert math.isclose(a, np.abs(A).sum(axis=1).max(), rel_tol=1e-12)
    assert math.isclose(xn, np.abs(x).max(), rel_tol=1e-15)


def check_nd_order_golden(golden_dir):
    with open(os.path.join(golden_dir, "nd_order_N20.json")) as f:
        g = json.load(f)
    order, levels = oracle.nd_order(g["N"])
    assert list(order + 1) == g["order_1based"]
    assert levels == g["levels"]


def check_worked_example(golden_dir):
    with open(os.path.join(golden_dir, "nd_worked_example_N3.json")) as f:
        g = json.load(f)
    D, B = np.array(g["D"]), np.array(g["B"])
    order, Ld, pairs, Loff = oracle.nd_factor(D, B)
    assert list(order) == g["order_0based"]
    np.testing.assert_allclose(Ld, np.array(g["Ldiag"]), rtol=1e-15)
    got = {(int(r), int(c)): blk for (r, c), blk in zip(pairs, Loff)}
    assert len(got) == len(g["Loff"])
    for e in g["Loff"]:
        np.testing.assert_allclose(got[(e["row"], e["col"])], np.array(e["value"]), rtol=1e-15)
    assert math.isclose(math.exp(oracle.logdet_from_diag(Ld)), g["det"], rel_tol=1e-14)
    x = oracle.solve(D, B, np.array(g["b"]))
    np.testing.assert_allclose(x, np.array(g["x"]), atol=1e-15)


def check_toeplitz_closed_form(N=13, n=2, d=3.0, e=1.2):
    D, B = gen.toeplitz_kron(N, n, d, e)
    k = np.arange(1, N + 1)
    logdet = n * np.log(d + 2 * e * np.cos(k * np.pi / (N + 1))).sum()
    Dh, _ = oracle.seq_factor(D, B)
    assert math.isclose(oracle.logdet_from_diag(Dh), logdet, rel_tol=1e-13)
    _, Ld, _, _ = oracle.nd_factor(D, B)
    assert math.isclose(oracle.logdet_from_diag(Ld), logdet, rel_tol=1e-13)
    rhs = gen.rhs(N, n, 1, seed=5)[:, 0]
    x = oracle.solve(D, B, rhs)
    for comp in range(n):
        np.testing.assert_allclose(x[comp::n], thomas(d, e, rhs[comp::n]), rtol=1e-12, atol=1e-13)


def check_arrow_assemble_vs_blocks(N=4, n=3, m=2, seed=6):
    D, B, C, A = gen.arrow(N, n, m, seed=seed)
    Ag = A.copy()
    Ag[np.triu_indices(m, 1)] = 7e3  # only the lower triangle of A may be read
    M = oracle.arrow_assemble(D, B, C, Ag)
    ref = np.block([[oracle.assemble(D, B), C.T], [C, A]])
    np.testing.assert_array_equal(M, ref)


def check_arrow_solve_vs_lapack(N=5, n=2, m=3, seed=7):
    D, B, C, A = gen.arrow(N, n, m, seed=seed)
    b = np.random.default_rng(seed).standard_normal(N * n + m)
    x = oracle.arrow_solve(D, B, C, A, b)
    M = np.block([[oracle.assemble(D, B), C.T], [C, A]])
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-10, atol=1e-12)


def check_arrow_resid_vs_dense(N=4, n=3, m=2, seed=8):
    D, B, C, A = gen.arrow(N, n, m, seed=seed)
    rng = np.random.default_rng(seed)
    x, b = rng.standard_normal(N * n + m), rng.standard_normal(N * n + m)
    M = np.block([[oracle.assemble(D, B), C.T], [C, A]])
    r, a, xn = oracle.arrow_resid(D, B, C, A, x, b)
    assert math.isclose(r, np.abs(b - M @ x).max(), rel_tol=1e-12)
    assert math.isclose(a, np.abs(M).sum(axis=1).max(), rel_tol=1e-12)
    assert math.isclose(xn, np.abs(x).max(), rel_tol=1e-15)
    # a residual that lives in the border rows only (the block-tridiagonal rows are satisfied)
    b2 = M @ x
    b2[N * n:] += rng.standard_normal(m) * 1e-3
    r2, _, _ = oracle.arrow_resid(D, B, C, A, x, b2)
    assert math.isclose(r2, np.abs(b2 - M @ x).max(), rel_tol=1e-6)


# ------------------------------------------------------------ the tests ---


@pytest.mark.parametrize("N,p", [(10, 2), (101, 4), (1000, 8), (57, 3), (6, 2)])
def test_partition_sizes_follow_proposition_1(N, p):
    n1, nk = oracle.partition_sizes(N, p)
    assert n1 + (p - 1) * (nk + 1) == N and n1 >= 1 and nk >= 1
    # the continuous optimum balances the two parallel-phase costs at ratio 19/7
    n1s = (19 * N - 19 * p + 19) / (7 * p + 12)
    nks = (7 * N - 7 * p + 7) / (7 * p + 12)
    assert math.isclose(n1s / nks, 19 / 7) and math.isclose(n1s + (p - 1) * (nks + 1), N)
    assert abs(nk - nks) < 1.0 + 1e-12
    # no other integer split does better on the larger phase cost
    cost = lambda a, b: max(7 / 3 * a - 1, 19 / 3 * b - 1)
    for b in range(1, N):
        a = N - (p - 1) * (b + 1)
        if a >= 1:
            assert cost(n1, nk) <= cost(a, b) + 1e-9 or abs(b - nks) >= 1.0


@pytest.mark.parametrize("N,p,n", [(7, 2, 2), (12, 3, 3), (9, 1, 2), (20, 4, 2)])
def test_partition_order_factor_equals_dense_cholesky_of_permuted(N, p, n):
    D, B = gen.bt_random(N, n, delta=0.3, seed=N + p)
    order, Ld, pairs, Loff = oracle.partition_factor(D, B, p)
    assert sorted(order.tolist()) == list(range(N))
    n1, nk = oracle.partition_sizes(N, p)
    assert list(order[:n1]) == list(range(n1))  # chunk 1 first, in natural order
    A = oracle.assemble(D, B)
    L = np.linalg.cholesky(permuted_dense(A, order, n))
    pos = np.empty(N, dtype=int)
    pos[order] = np.arange(N)
    for i in range(N):
        np.testing.assert_allclose(Ld[i], L[pos[i] * n:(pos[i] + 1) * n, pos[i] * n:(pos[i] + 1) * n], rtol=1e-12,
                                   atol=1e-12)
    for (r, c), blk in zip(pairs, Loff):
        np.testing.assert_allclose(blk, L[pos[r] * n:(pos[r] + 1) * n, pos[c] * n:(pos[c] + 1) * n], rtol=1e-11,
                                   atol=1e-12)
    # fill: each chunk k > 1 couples its pivot with every later node of the chunk, and consecutive pivots
    # couple through the last node of the chunk between them
    expect = (N - 1) + (p - 1) * (nk - 1) + max(p - 2, 0)
    assert len(pairs) == expect


def test_arrow_assemble_places_the_border():
    check_arrow_assemble_vs_blocks()


@pytest.mark.parametrize("N,n,m", [(1, 1, 1), (5, 2, 3), (7, 4, 5)])
def test_arrow_solve_matches_lapack(N, n, m):
    check_arrow_solve_vs_lapack(N, n, m, seed=N + m)


def test_arrow_resid_matches_dense():
    check_arrow_resid_vs_dense()


def test_arrow_with_zero_border_decouples():
    """C = 0: the bordered system splits into Psi x_T = b_T (Alg. 1 solve) and A x_A = b_A."""
    D, B, C, A = gen.arrow(6, 3, 4, seed=9)
    C = np.zeros_like(C)
    b = np.random.default_rng(9).standard_normal(18 + 4)
    x = oracle.arrow_solve(D, B, C, A, b)
    np.testing.assert_allclose(x[:18], oracle.solve(D, B, b[:18]), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(x[18:], np.linalg.solve(A, b[18:]), rtol=1e-12, atol=1e-13)


def test_arrow_generator_is_spd_with_schur_complement_above_identity():
    D, B, C, A = gen.arrow(8, 3, 4, delta=0.5, seed=10)
    M = oracle.arrow_assemble(D, B, C, A)
    assert np.linalg.eigvalsh(M).min() > 0
    T = oracle.assemble(D, B)
    S = A - C @ np.linalg.solve(T, C.T)
    assert np.linalg.eigvalsh(S).min() >= 1.0 - 1e-9

def test_chol_matches_lapack():
    check_chol_vs_lapack()


def test_chol_reports_first_bad_pivot():
    A = np.array([[4.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]])  # second pivot 1 - 1 = 0
    with pytest.raises(oracle.NotSPD) as ei:
        oracle.chol(A)
    assert ei.value.info == 2


def test_gepp_matches_lapack_and_pivots():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((9, 9))
    A[0, 0] = 0.0  # forces a row exchange at step 1
    b = rng.standard_normal((9, 3))
    np.testing.assert_allclose(oracle.gepp_solve(A, b), np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


def test_dense_chol_matches_lapack():
    D, B = gen.bt_random(4, 3, seed=9)
    A = oracle.assemble(D, B)
    np.testing.assert_allclose(oracle.dense_chol(A), np.linalg.cholesky(A), rtol=1e-12, atol=1e-13)


def test_assemble_is_symmetric_block_tridiagonal():
    D, B = gen.bt_random(5, 2, seed=10)
    A = oracle.assemble(D, B)
    np.testing.assert_array_equal(A, A.T)
    np.testing.assert_array_equal(A[2:4, 0:2], B[0])
    assert np.all(A[4:6, 0:2] == 0)


@pytest.mark.parametrize("N,n", [(1, 3), (2, 2), (6, 3), (8, 1)])
def test_seq_factor_equals_dense_cholesky(N, n):
    check_seq_factor_vs_dense(N, n)


@pytest.mark.parametrize("N,n,m", [(1, 4, 1), (5, 3, 2), (8, 2, 3)])
def test_seq_solve_equals_lapack_and_gepp(N, n, m):
    check_seq_solve_vs_lapack(N, n, m)


def test_resid_matches_dense():
    check_resid_vs_dense()


def test_nd_order_matches_hand_written_N20(golden_dir):
    check_nd_order_golden(golden_dir)


@pytest.mark.parametrize("N", list(range(1, 65)))
def test_nd_order_is_a_permutation_with_floor_log2_plus_1_levels(N):
    order, levels = oracle.nd_order(N)
    assert sorted(order) == list(range(N))
    assert levels == int(math.floor(math.log2(N))) + 1


def test_worked_example_N3(golden_dir):
    check_worked_example(golden_dir)


@pytest.mark.parametrize("N,n", [(3, 1), (7, 2), (11, 2), (16, 3), (21, 2)])
def test_nd_factor_equals_dense_cholesky_of_permuted(N, n):
    check_nd_factor_vs_dense(N, n, seed=N)


@pytest.mark.parametrize("N", list(range(1, 65)))
def test_nd_fill_pattern_matches_prediction(N):
    D, B = gen.bt_random(N, 1, seed=N)
    order, Ld, pairs, Loff = oracle.nd_factor(D, B)
    got = {(int(r), int(c)) for r, c in pairs}
    pred = predicted_nd_pairs(N)
    assert got == pred
    # counts: off-diagonal blocks = sum over levels (floor(N/s) - 1); fill = that - (N - 1)
    etot = sum(N // (2 ** l) - 1 for l in range(int(math.log2(N)) + 1))
    assert len(got) == etot
    if N & (N - 1) == 0:  # N = 2^k: fill = N - log2(N) - 1
        assert etot - (N - 1) == N - int(math.log2(N)) - 1


def test_identity_order_reproduces_alg1():
    D, B = gen.bt_random(9, 3, seed=11)
    Ld, pairs, Loff = oracle.bs_chol(D, B, np.arange(9))
    Dh, Eh = oracle.seq_factor(D, B)
    np.testing.assert_allclose(Ld, Dh, rtol=1e-13, atol=1e-14)
    assert sorted((int(r), int(c)) for r, c in pairs) == [(i + 1, i) for i in range(8)]
    for (r, c), blk in zip(pairs, Loff):
        np.testing.assert_allclose(blk, Eh[c], rtol=1e-13, atol=1e-14)


def test_logdet_is_order_invariant():
    D, B = gen.bt_random(13, 3, delta=0.05, seed=12)
    sign, ref = np.linalg.slogdet(oracle.assemble(D, B))
    assert sign > 0
    Dh, _ = oracle.seq_factor(D, B)
    _, Ld, _, _ = oracle.nd_factor(D, B)
    rng = np.random.default_rng(0)
    Lr, _, _ = oracle.bs_chol(D, B, rng.permutation(13))
    for L in (Dh, Ld, Lr):
        assert math.isclose(oracle.logdet_from_diag(L), ref, rel_tol=1e-12)


def test_toeplitz_closed_form():
    check_toeplitz_closed_form()


def test_zero_coupling_gives_blockdiag_and_zero_fill():
    D, B = gen.bt_random(12, 3, seed=13)
    B[:] = 0.0
    order, Ld, pairs, Loff = oracle.nd_factor(D, B)
    for i in range(12):
        np.testing.assert_allclose(Ld[i], np.linalg.cholesky(D[i]), rtol=1e-13)
    assert np.all(Loff == 0.0)


def test_N2_nd_equals_natural_order():
    D, B = gen.bt_random(2, 4, seed=14)
    order, Ld, pairs, Loff = oracle.nd_factor(D, B)
    assert list(order) == [0, 1]
    Dh, Eh = oracle.seq_factor(D, B)
    np.testing.assert_array_equal(Ld, Dh)
    np.testing.assert_array_equal(Loff[0], Eh[0])


def test_reconstruction_identity_and_its_sensitivity():
    D, B = gen.bt_random(17, 3, delta=0.1, seed=15)
    order, Ld, pairs, Loff = oracle.nd_factor(D, B)
    assert oracle.bs_reconstruct(D, B, order, Ld, pairs, Loff) < 1e-14
    bad = Loff.copy()
    bad[3] = bad[3].T
    assert oracle.bs_reconstruct(D, B, order, Ld, pairs, bad) > 1e-6


def test_nd_and_sequential_solutions_agree():
    N, n = 33, 3
    D, B = gen.bt_random(N, n, delta=0.01, seed=16)
    b = gen.rhs(N, n, 2, seed=16)
    x_seq = oracle.solve(D, B, b)
    # solve with the ND factor: P^T L L^T P x = b, dense on this small case
    order, Ld, pairs, Loff = oracle.nd_factor(D, B)
    M = N * n
    pos = np.empty(N, dtype=int)
    pos[order] = np.arange(N)
    L = np.zeros((M, M))
    for i in range(N):
        p = pos[i]
        L[p * n:(p + 1) * n, p * n:(p + 1) * n] = Ld[i]
    for (r, c), blk in zip(pairs, Loff):
        L[pos[r] * n:(pos[r] + 1) * n, pos[c] * n:(pos[c] + 1) * n] = blk
    idx = np.concatenate([np.arange(o * n, (o + 1) * n) for o in order])
    y = np.linalg.solve(L, b[idx])
    z = np.linalg.solve(L.T, y)
    x_nd = np.empty_like(z)
    x_nd[idx] = z
    np.testing.assert_allclose(x_nd, x_seq, rtol=1e-9, atol=1e-11)
    assert oracle.relres(D, B, x_seq, b) < 1e-15


def test_generator_is_spd_with_eigenvalues_above_delta():
    for delta in (1.0, 1e-2):
        D, B = gen.bt_random(10, 4, delta=delta, seed=17)
        w = np.linalg.eigvalsh(oracle.assemble(D, B))
        assert w.min() >= delta * (1 - 1e-9)


def test_mpc_generator_is_G_Gt_of_the_dynamics():
    """The MPC blocks equal G G^T for the constraint matrix G of
    x_{k+1} - A_k x_k - Bu_k u_k = 0 (variables x_1..x_N, u_0..u_{N-1}), built here
    column by column; G has full row rank, so Psi is SPD."""
    N, n = 7, 4
    D, B, A, Bu = gen.mpc(N, n, seed=18, return_parts=True)
    h = n // 2
    G = np.zeros((N * n, N * n + N * h))
    xcol = lambda k: slice((k - 1) * n, k * n)  # x_k, k = 1..N
    ucol = lambda k: slice(N * n + k * h, N * n + (k + 1) * h)  # u_k, k = 0..N-1
    for k in range(N):
        rows = slice(k * n, (k + 1) * n)
        G[rows, xcol(k + 1)] = np.eye(n)
        if k >= 1:
            G[rows, xcol(k)] = -A[k]
        G[rows, ucol(k)] = -Bu[k]
    np.testing.assert_allclose(oracle.assemble(D, B), G @ G.T, rtol=1e-13, atol=1e-14)
    assert np.linalg.eigvalsh(G @ G.T).min() > 0
    assert np.allclose(np.abs(np.linalg.eigvals(A)).max(axis=1), 0.95)


# -------------------------------------------------------- mutation tests ---

MUTATIONS = [
    # (tag, original text, planted mistake, which pin must catch it)
    ("chol_transposed_index", "v -= L[i * ldl + k] * L[j * ldl + k];", "v -= L[i * ldl + k] * L[k * ldl + j];",
     "chol"),
    ("trsm_transposed_operand", "for (int k = 0; k < j; ++k) v -= x[k] * L[j * n + k];",
     "for (int k = 0; k < j; ++k) v -= x[k] * L[k * n + j];", "seq"),
    ("syrk_dropped", "    gemm_nt_sub(n, Ehat + (i - 1) * bs, Ehat + (i - 1) * bs, S);\n", "\n", "seq"),
    ("gemm_transposed_operand", "v += A[i * n + k] * B[j * n + k];", "v += A[i * n + k] * B[k * n + j];", "seq"),
    ("backsolve_transposed", "for (int k = 0; k < n; ++k) v += E[k * n + r] * xn[k * m + c];",
     "for (int k = 0; k < n; ++k) v += E[r * n + k] * xn[k * m + c];", "solve"),
    ("bs_scatter_orientation", "blk[r * n + c] = p > q ? B[i * bs + r * n + c] : B[i * bs + c * n + r];",
     "blk[r * n + c] = B[i * bs + r * n + c];", "nd"),
    ("bs_update_wrong_sign", "gemm_nt_sub(n, T[(size_t)i * N + k], T[(size_t)j * N + k], *slot);",
     "gemm_nt_sub(n, T[(size_t)j * N + k], T[(size_t)i * N + k], *slot);", "nd"),
    # (a stride mistake that writes fewer entries, so the planted copy stays in bounds)
    ("nd_order_stride", "for (long i = s; i <= N; i += 2 * s)", "for (long i = s; i <= N; i += 4 * s)", "order"),
    ("resid_sign", "v -= B[(i - 1) * bs + r * n + c] * x[((size_t)(i - 1) * n + c) * m + col];",
     "v += B[(i - 1) * bs + r * n + c] * x[((size_t)(i - 1) * n + c) * m + col];", "resid"),
    ("resid_upper_transposed", "v -= B[i * bs + c * n + r] * x[((size_t)(i + 1) * n + c) * m + col];",
     "v -= B[i * bs + r * n + c] * x[((size_t)(i + 1) * n + c) * m + col];", "resid"),
    ("arrow_border_transposed", "out[(size_t)j * M + L + r] = C[(size_t)r * L + j];",
     "out[(size_t)j * M + L + r] = C[(size_t)r * L + (j + 1) % L];", "arrow"),
    ("arrow_resid_border_dropped", "        v -= a * x[L + q];\n", "\n", "arrow"),
    ("arrow_resid_corner_sign", "      v -= a * x[L + c];", "      v += a * x[L + c];", "arrow"),
    # block-banded: the upper blocks taken untransposed; the band's distance index off by one
    ("band_upper_not_transposed", "(size_t)c * b + r]; /* Psi(I, J) = Psi(J, I)^T */",
     "(size_t)r * b + c]; /* Psi(I, J) = Psi(J, I)^T */", "band"),
    ("band_distance_off_by_one", "if (I > J) return A[((size_t)(I - J) * Nb + J) * bb",
     "if (I > J) return A[((size_t)(I - J - 1) * Nb + J) * bb", "band"),
]


def _run_pins(which, golden_dir):
    if which == "chol":
        check_chol_vs_lapack()
    elif which == "seq":
        check_seq_factor_vs_dense()
        check_seq_solve_vs_lapack()
    elif which == "solve":
        check_seq_solve_vs_lapack()
    elif which == "nd":
        check_nd_factor_vs_dense()
        check_worked_example(golden_dir)
    elif which == "order":
        check_nd_order_golden(golden_dir)
    elif which == "resid":
        check_resid_vs_dense()
    elif which == "arrow":
        check_arrow_assemble_vs_blocks()
        check_arrow_solve_vs_lapack()
        check_arrow_resid_vs_dense()
    elif which == "band":
        check_band_scalar_example()
        check_band_w1_is_block_tridiagonal()
        check_band_resid_vs_dense()


# ---------------------------------------------------------------- block-banded pins
def check_band_scalar_example():
    """b = 1, w = 2, Nb = 4: the pentadiagonal matrix written out by hand from Psi(i+k, i) = A_k[i]
    (A_0 = 10, 11, 12, 13; A_1 = 1, 2, 3; A_2 = 4, 5)."""
    A = np.zeros((3, 4, 1, 1))
    A[0, :, 0, 0] = [10, 11, 12, 13]
    A[1, :3, 0, 0] = [1, 2, 3]
    A[2, :2, 0, 0] = [4, 5]
    A[1, 3] = A[2, 2] = A[2, 3] = 99.0  # outside the matrix: never read
    ref = np.array([[10, 1, 4, 0],
                    [1, 11, 2, 5],
                    [4, 2, 12, 3],
                    [0, 5, 3, 13]], dtype=float)
    assert np.array_equal(oracle.band_assemble(A), ref)
    # a non-symmetric 2 x 2 off-diagonal block keeps its orientation: Psi(1, 0) = A_1[0], Psi(0, 1) = its transpose
    A2 = np.zeros((2, 2, 2, 2))
    A2[0] = np.eye(2) * 9
    A2[1, 0] = [[1, 2], [3, 4]]
    M = oracle.band_assemble(A2)
    assert np.array_equal(M[2:, :2], [[1, 2], [3, 4]]) and np.array_equal(M[:2, 2:], [[1, 3], [2, 4]])


def check_band_w1_is_block_tridiagonal():
    A = gen.banded(7, 3, 1, seed=2)
    assert np.array_equal(oracle.band_assemble(A), oracle.assemble(A[0], A[1, :6]))


def check_band_resid_vs_dense():
    for (Nb, b, w) in [(9, 2, 3), (6, 3, 2), (5, 4, 1)]:
        A = gen.banded(Nb, b, w, seed=Nb)
        M = oracle.band_assemble(A)
        rng = np.random.default_rng(1)
        x = rng.standard_normal((Nb * b, 2))
        rhs = rng.standard_normal((Nb * b, 2))
        r, a, xn = oracle.band_resid(A, x, rhs)
        assert abs(r - np.abs(rhs - M @ x).max()) <= 1e-12 * max(1.0, r)
        assert abs(a - np.abs(M).sum(axis=1).max()) <= 1e-12 * a
        assert xn == np.abs(x).max()


def test_band_oracle_pins():
    check_band_scalar_example()
    check_band_w1_is_block_tridiagonal()
    check_band_resid_vs_dense()


@pytest.mark.parametrize("Nb,b,w", [(1, 3, 2), (5, 2, 2), (7, 3, 3), (9, 2, 4), (8, 4, 2)])
def test_band_group_is_the_same_matrix(Nb, b, w):
    """The block-tridiagonal view of the band is Psi itself, padded with an identity (and generated band
    matrices are SPD, with every eigenvalue >= delta)."""
    A = gen.banded(Nb, b, w, delta=0.5, seed=3)
    M = oracle.band_assemble(A)
    assert np.linalg.eigvalsh(M).min() >= 0.5 - 1e-12
    Dg, Bg = oracle.band_group(A, w)
    G = oracle.assemble(Dg, Bg)
    L = Nb * b
    assert np.array_equal(G[:L, :L], M)
    assert np.array_equal(G[L:, L:], np.eye(G.shape[0] - L)) and not G[L:, :L].any()
    rhs = np.random.default_rng(0).standard_normal((L, 1))
    x = oracle.band_solve(A, rhs)
    assert oracle.band_relres(A, x, rhs) <= 1e-14
    assert np.allclose(x, np.linalg.solve(M, rhs), rtol=0, atol=1e-12 * np.abs(x).max())


@pytest.mark.parametrize("tag,old,new,which", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tag, old, new, which, golden_dir):
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation anchor for {tag} not found exactly once"
    _run_pins(which, golden_dir)  # the real oracle passes
    with oracle.use_variant(src.replace(old, new), tag):
        with pytest.raises((AssertionError, oracle.NotSPD, ZeroDivisionError, ValueError, IndexError)):
            _run_pins(which, golden_dir)


def test_mpc_torch_generator_is_spd_with_radius_095():
    torch = pytest.importorskip("torch")
    D, B = gen.mpc_torch(9, 6, seed=3, device="cpu")
    A = -B.numpy()
    assert np.allclose(np.abs(np.linalg.eigvals(A)), 0.95)
    w = np.linalg.eigvalsh(oracle.assemble(D.numpy(), B.numpy()))
    assert w.min() > 0
