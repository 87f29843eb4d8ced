"""The captured-graph form of btc_factor_solve_refined (device-side refinement
loop) against plain launches: same solution bitwise, same number of steps and
final residual, on replay, after a pointer change (re-capture), when the
iteration limit stops the loop, and when a pivot fails."""
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


def _plans(N, n, dt, stream=None):
    pg = btc.btc_plan(N, n, dt, stream)
    pp = btc.btc_plan(N, n, dt, stream)
    btc.btc_plan_set_graphs(pp, False)
    return pg, pp


@pytest.mark.parametrize("dt", [btc.F64, btc.MIXED_F32], ids=["f64", "mixed"])
@pytest.mark.parametrize("N,n,m,delta", [(1, 8, 1, 1.0), (64, 16, 1, 1e-2), (333, 32, 3, 1e-4), (1024, 64, 1, 1.0)])
def test_graph_matches_plain_launches(N, n, m, delta, dt):
    D, B = gen.bt_random(N, n, delta=delta, seed=N + m)
    b = gen.rhs(N, n, m, seed=N)
    Dd, Bd = dev(D, torch.float64), dev(B if B.size else np.zeros((1, n, n)), torch.float64)
    bd = dev(b, torch.float64)
    s = torch.cuda.Stream()
    pg, pp = _plans(N, n, dt, s)
    xp = torch.zeros_like(bd)
    torch.cuda.synchronize()
    ref = btc.btc_factor_solve_refined(pp, Dd, Bd, bd, xp, m, tol=1e-11)
    for rep in range(3):  # first call tunes, then capture, then replays
        xg = torch.zeros_like(bd)
        torch.cuda.synchronize()
        got = btc.btc_factor_solve_refined(pg, Dd, Bd, bd, xg, m, tol=1e-11)
        assert torch.equal(xg, xp) and got[:2] == ref[:2], rep
    # new output pointer: re-captured
    xg2 = torch.full_like(bd, 7.0)
    torch.cuda.synchronize()
    got = btc.btc_factor_solve_refined(pg, Dd, Bd, bd, xg2, m, tol=1e-11)
    assert torch.equal(xg2, xp) and got[:2] == ref[:2]
    # the factor left behind serves later solves (the copies are made on torch's stream; the plans
    # run on s, so wait for them first)
    xs = bd.clone()
    xs2 = bd.clone()
    torch.cuda.synchronize()
    btc.btc_solve(pg, xs, m)
    btc.btc_solve(pp, xs2, m)
    s.synchronize()
    assert torch.equal(xs, xs2)


def test_graph_iteration_limit_and_failed_pivot():
    N, n, dt = 200, 16, btc.MIXED_F32
    D, B = gen.bt_random(N, n, delta=1e-4, seed=5)
    b = gen.rhs(N, n, 1, seed=5)
    Dd, Bd, bd = dev(D, torch.float64), dev(B, torch.float64), dev(b, torch.float64)
    pg, pp = _plans(N, n, dt)
    res = []
    for p in (pp, pg, pg, pg):
        x = torch.zeros_like(bd)
        it, rel, rc = btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, 1, tol=1e-30, maxit=2, allow_not_converged=True)
        assert rc == btc.ERR_NOT_CONVERGED and it == 2
        res.append((x.clone(), rel))
    for x, rel in res[1:]:
        assert torch.equal(x, res[0][0]) and rel == res[0][1]
    D[77] = -np.eye(n)
    Dbad = dev(D, torch.float64)
    for p in (pp, pg):
        x = torch.zeros_like(bd)
        with pytest.raises(btc.BtcError) as ei:
            btc.btc_factor_solve_refined(p, Dbad, Bd, bd, x, 1)
        assert ei.value.code == btc.ERR_NOT_SPD
