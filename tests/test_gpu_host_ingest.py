"""btc_factor_solve_host with page-locked host inputs: the level-1 eliminations read D (lower
triangles only) and B over the CPU-GPU link and fill the device copies that the FP64 residuals
use. The factor and the solution must be exactly those of the same call with device inputs, and
of the copy path that pageable inputs take."""
import numpy as np
import pytest

from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import dev, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _device_reference(N, n, m, D, B, b, dt):
    p = btc.btc_plan(N, n, dt)
    x = torch.zeros((N * n, m), dtype=torch.float64, device="cuda")
    it, rel, _ = btc.btc_factor_solve_refined(p, dev(D, torch.float64), dev(B, torch.float64), dev(b, torch.float64),
                                              x, m, tol=1e-11, maxit=30)
    return x.cpu().numpy(), it, rel, btc.btc_get_factor(p)


@pytest.mark.parametrize("dt", [btc.MIXED_F32, btc.F64], ids=["mixed", "f64"])
@pytest.mark.parametrize("N,n,m,delta", [(2, 16, 1, 1.0), (257, 16, 2, 1e-3), (300, 32, 1, 1.0), (129, 48, 1, 1e-2),
                                         (1024, 64, 1, 1.0), (65, 96, 1, 1.0), (97, 33, 1, 1.0), (40, 7, 2, 1e-2)])
def test_pinned_inputs_give_the_device_result(N, n, m, delta, dt):
    if dt == btc.F64 and n > 96:
        pytest.skip("FP64 blocks up to 96")
    D, B = gen.bt_random(N, n, delta=delta, seed=N + n)
    b = gen.rhs(N, n, m, seed=N)
    x_ref, it_ref, rel_ref, f_ref = _device_reference(N, n, m, D, B, b, dt)
    Dg = D.copy()
    for i in range(N):  # only the lower triangles may be read
        Dg[i][np.triu_indices(n, 1)] = np.nan
    Dh, Bh, bh = _pinned(Dg), _pinned(B), _pinned(b)
    p = btc.btc_plan(N, n, dt)
    for rep in range(3):  # tuning call, graph capture, replay
        xh = torch.zeros((N * n, m), dtype=torch.float64).pin_memory()
        it, rel, rc = btc.btc_factor_solve_host(p, Dh, Bh, bh, xh, m, 1e-11, 30)
        assert rc == btc.OK
        assert np.array_equal(xh.numpy(), x_ref), rep
        assert (it, rel) == (it_ref, rel_ref), rep
    f = btc.btc_get_factor(p)
    assert np.array_equal(f[0], f_ref[0]) and np.array_equal(f[1], f_ref[1])
    # pageable inputs take the copy path: same result
    q = btc.btc_plan(N, n, dt)
    xq = np.zeros_like(b)
    it2, rel2, _ = btc.btc_factor_solve_host(q, Dg, B, b, xq, m, 1e-11, 30)
    assert np.array_equal(xq, x_ref) and (it2, rel2) == (it_ref, rel_ref)


def test_new_values_in_the_same_pinned_buffers_are_read():
    N, n, m = 300, 32, 1
    D, B = gen.bt_random(N, n, delta=1.0, seed=5)
    b = gen.rhs(N, n, m, seed=5)
    Dh, Bh, bh = _pinned(D), _pinned(B), _pinned(b)
    p = btc.btc_plan(N, n, btc.MIXED_F32)
    xh = torch.zeros((N * n, m), dtype=torch.float64).pin_memory()
    for _ in range(2):
        btc.btc_factor_solve_host(p, Dh, Bh, bh, xh, m)
    # scale the matrix in place: the solution scales by the inverse
    Dh.mul_(2.0)
    Bh.mul_(2.0)
    x2 = torch.zeros_like(xh).pin_memory()
    it, rel, rc = btc.btc_factor_solve_host(p, Dh, Bh, bh, x2, m)
    assert rc == btc.OK and rel <= 1e-10
    x_ref, _, _, _ = _device_reference(N, n, m, 2.0 * D, 2.0 * B, b, btc.MIXED_F32)
    assert np.abs(x2.numpy() - x_ref).max() <= 1e-9 * np.abs(x_ref).max()
    assert np.abs(2.0 * x2.numpy() - xh.numpy()).max() <= 1e-8 * np.abs(xh.numpy()).max()


def test_single_block_and_tensor_core_paths_copy_first():
    for N, n, dt in ((1, 16, btc.MIXED_F32), (40, 128, btc.MIXED_TF32)):
        D, B = gen.bt_random(N, n, delta=1.0, seed=7)
        b = gen.rhs(N, n, 1, seed=7)
        Bz = B if B.size else np.zeros((1, n, n))
        p = btc.btc_plan(N, n, dt)
        xh = torch.zeros((N * n, 1), dtype=torch.float64).pin_memory()
        it, rel, rc = btc.btc_factor_solve_host(p, _pinned(D), _pinned(Bz), _pinned(b), xh, 1, 1e-11, 30)
        assert rc == btc.OK and rel <= 1e-11
