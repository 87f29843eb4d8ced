"""Host-side checks of libbtc.so (no GPU needed): exported symbols, the level
planner of the multi-stage permutation, and its flop/byte tallies."""
import math
import subprocess

import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, build


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return btc.load()


def test_library_exports_every_header_symbol():
    names = btc.header_symbols()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", btc.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [s for s in names if s not in exported]
    assert not missing, missing
    lib = btc.load()
    for s in names:
        assert getattr(lib, s) is not None


def test_version_and_last_error():
    assert btc.btc_version() >= 100
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_describe(0, 4)
    assert ei.value.code == btc.ERR_ARG
    assert "invalid" in btc.load().btc_last_error().decode()


def test_describe_rejects_oversized_blocks():
    assert btc.btc_describe(16, 96, btc.F64)["np"] == 96
    assert btc.btc_describe(16, 128, btc.F32)["np"] == 128
    # blocks above 128 run as blocked nodes of tile tasks, on the tensor-core dtypes only, up to 256
    for dt in (btc.MIXED_TF32, btc.MIXED_BF16):
        assert btc.btc_describe(16, 129, dt)["np"] == 256
        assert btc.btc_describe(16, 256, dt)["np"] == 256
    for n, dt in ((97, btc.F64), (129, btc.F32), (129, btc.MIXED_F32), (257, btc.MIXED_TF32),
                  (257, btc.MIXED_BF16)):
        with pytest.raises(btc.BtcError) as ei:
            btc.btc_describe(16, n, dt)
        assert ei.value.code == btc.ERR_UNSUPPORTED


@pytest.mark.parametrize("N", list(range(1, 130)) + [255, 256, 257, 1000, 1024, 4096])
def test_schedule_is_the_multistage_permutation(N):
    order, levels = btc.btc_schedule(N)
    ref, nlev = oracle.nd_order(N)  # independent restatement of Sec. 4.3
    assert list(order) == list(ref)
    assert levels.max() == nlev == int(math.floor(math.log2(N))) + 1
    # within level l the eliminated nodes are the odd multiples of 2^(l-1) (1-based)
    for node, l in zip(order + 1, levels):
        s = 2 ** (l - 1)
        assert node % s == 0 and (node // s) % 2 == 1


def test_schedule_golden_N20(golden_dir):
    import json, os
    with open(os.path.join(golden_dir, "nd_order_N20.json")) as f:
        g = json.load(f)
    order, levels = btc.btc_schedule(20)
    assert list(order + 1) == g["order_1based"]


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 20, 64, 100, 1024, 4096])
def test_block_counts(N):
    d = btc.btc_describe(N, 4)
    brute = 0
    s = 1
    while s <= N:
        surv = list(range(s, N + 1, s))
        brute += len(surv) - 1
        s *= 2
    assert d["offdiag_blocks"] == brute
    assert d["fill_blocks"] == brute - (N - 1)
    if N & (N - 1) == 0:
        assert d["fill_blocks"] == N - int(math.log2(N)) - 1


@pytest.mark.parametrize("N,n", [(64, 16), (1024, 64), (4096, 8), (37, 5)])
def test_flop_tallies(N, n):
    d = btc.btc_describe(N, n)
    n3 = float(n) ** 3
    # Sec. 3.1: the sequential Alg. 1 costs (7/3 N - 2) n^3
    assert d["seq_factor_flops"] == pytest.approx((7.0 / 3.0 * N - 2.0) * n3)
    # Alg. 5 with Table 1 costs: potrf per node, trsm + syrk per off-diagonal block, gemm per fill block
    assert d["factor_flops"] == pytest.approx((N / 3.0 + 2 * d["offdiag_blocks"] + 2 * d["fill_blocks"]) * n3)
    assert d["critical_path_flops"] <= d["critical_path_formula"] + 1e-6 * n3
    assert d["solve_flops_per_rhs"] == pytest.approx(2 * N * n * n + 4 * d["offdiag_blocks"] * n * n)


def test_table_counts_from_the_scope_table():
    # ND flops / n^3 for N = 64, 1024, 4096 (levels 7, 11, 13)
    for N, lv, F, E, nd in [(64, 7, 57, 120, 375.33), (1024, 11, 1013, 2036, 6439.33), (4096, 13, 4083, 8178,
                                                                                            25887.33)]:
        d = btc.btc_describe(N, 1)
        assert (d["levels"], d["fill_blocks"], d["offdiag_blocks"]) == (lv, F, E)
        assert d["factor_flops"] == pytest.approx(nd, abs=0.01)


def alg5_critical_path(N):
    """Brute-force p = infinity cost of Alg. 5 in units of n^3: per level, the
    largest per-node sum of Table 1 costs over the steps whose conditions hold
    (deferred syrk x2, potrf, trsm x2, syrk, gemm)."""
    total = 0.0
    s = 1
    while s <= N:
        best = 0.0
        for i in range(s, N + 1, 2 * s):
            c = 1.0 / 3.0
            if s > 1 and i <= N - s / 2:
                c += 1
            if s > 1 and i + s <= N - s / 2:
                c += 1
            if i + s <= N:
                c += 2  # trsm + syrk
            if i > s:
                c += 1  # trsm
            if i > s and i + s <= N:
                c += 2  # gemm
            best = max(best, c)
        total += best
        s *= 2
    return total


@pytest.mark.parametrize("N", [2, 3, 7, 20, 64, 100, 1000, 1024, 4095])
def test_critical_path_against_alg5_conditions_and_the_paper_bound(N):
    d = btc.btc_describe(N, 1)
    assert d["critical_path_flops"] == pytest.approx(alg5_critical_path(N))
    # The closed form of Sec. 4.3 (p = infinity) charges every middle level the full
    # 22/3; it is an upper bound, exact on the first and last levels.
    lg = int(math.floor(math.log2(N)))
    assert d["critical_path_formula"] == pytest.approx(16 / 3 + 22 / 3 * (lg - 1) + 4 / 3)
    assert d["critical_path_flops"] <= d["critical_path_formula"] + 1e-9


def test_padding_rule():
    assert btc.btc_describe(10, 12)["np"] == 16
    assert btc.btc_describe(10, 24)["np"] == 32
    assert btc.btc_describe(10, 48)["np"] == 48
    assert btc.btc_describe(10, 64)["np"] == 64
    assert btc.btc_describe(10, 65)["np"] == 96
    assert btc.btc_describe(10, 1)["np"] == 8
