"""btc_residual_noalloc: the residual/norm entry point for callers that cannot
allocate device memory (no cudaMalloc, cudaMallocAsync or library allocation
inside the call; its scratch is a fixed device array in libbtc.so).

Checked through the C ABI against the allocating btc_residual on two calls in
a row with different inputs (the second call must not see stale scratch),
within the residual tolerance used elsewhere (1e-13 relative; the two share
the arithmetic, so equality is expected). This file is collected last on
purpose, so that a run stopping at its first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2601_03754_gb300 import btc, build, gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    btc.load()


def _case(N, n, m, seed):
    D, B = gen.bt_random(N, n, delta=1e-2, seed=seed)
    x = gen.rhs(N, n, m, seed=seed + 1)
    b = gen.rhs(N, n, m, seed=seed + 2)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return to(D), to(B), to(x), to(b)


def test_noalloc_residual_matches_allocating_entry_point_twice():
    cases = [(300, 24, 2, 1), (1024, 64, 1, 2)]
    for N, n, m, seed in cases:  # two calls in a row, different sizes and values
        D, B, x, b = _case(N, n, m, seed)
        ref = btc.btc_residual(N, n, m, D, B, x, b)
        got = btc.btc_residual_noalloc(N, n, m, D, B, x, b)
        for r, g in zip(ref, got):
            assert abs(g - r) <= 1e-13 * abs(r), (N, n, ref, got)
    # and once more on the first case after the larger one overwrote the scratch
    D, B, x, b = _case(*cases[0])
    ref = btc.btc_residual(300, 24, 2, D, B, x, b)
    got = btc.btc_residual_noalloc(300, 24, 2, D, B, x, b)
    assert np.allclose(got, ref, rtol=1e-13, atol=0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    D, B, x, b = _case(4, 8, 1, 3)
    with pytest.raises(btc.BtcError) as ei:
        btc.btc_residual_noalloc(65537, 8, 1, D, B, x, b)
    assert ei.value.code == btc.ERR_ARG
    assert "65536" in str(ei.value)
