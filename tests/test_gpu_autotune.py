"""Configurations of the persistent factorization (register-budget variant x
CTAs per SM) and the autotuner that chooses among them.

The configuration changes only which CTA runs which item and when, never the
arithmetic of an item, so every configuration must give bitwise the same
factor and solution."""
import numpy as np
import pytest

from paper_2601_03754_gb300 import btc, build, gen
from gpu_helpers import dev, need_gpu, tdtype, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    build.build()
    btc.load()


def _run(p, Dd, Bd, b, dt):
    x = dev(b, tdtype(dt))
    btc.btc_factor_solve(p, Dd, Bd, x, b.shape[1])
    rc, _, _ = btc.btc_info(p)
    assert rc == btc.OK
    return btc.btc_get_factor(p), x.cpu().numpy()


@pytest.mark.parametrize("dt", [btc.F64, btc.F32, btc.MIXED_F32], ids=["f64", "f32", "mixed"])
@pytest.mark.parametrize("N,n", [(1, 8), (100, 8), (257, 16), (300, 32), (129, 48), (500, 64)])
def test_every_configuration_gives_the_same_result(N, n, dt):
    D, B = gen.bt_random(N, n, delta=1.0, seed=N + n)
    b = gen.rhs(N, n, 2, seed=N)
    Dd, Bd = dev(D, tdtype(dt)), dev(B if B.size else np.zeros((1, n, n)), tdtype(dt))
    p = btc.btc_plan(N, n, dt)
    btc.btc_plan_set_autotune(p, False)
    ref_f, ref_x = _run(p, Dd, Bd, b, dt)
    variants = btc.btc_plan_flow_configs(p)
    assert variants and all(c >= 1 and m >= 1 for c, m in variants)
    for cap, most in variants:
        for ctas in sorted({1, most}):
            btc.btc_plan_set_flow_config(p, cap, ctas)
            f, x = _run(p, Dd, Bd, b, dt)
            assert np.array_equal(f[0], ref_f[0]) and np.array_equal(f[1], ref_f[1]), (cap, ctas)
            assert np.array_equal(x, ref_x), (cap, ctas)
    # right-looking variant (Alg. 6) under every configuration as well: its two atomic updates of a
    # diagonal block within a level land in either order, so results agree to rounding, not bitwise
    btc.btc_plan_set_variant(p, btc.VARIANT_RIGHT_LOOKING)
    btc.btc_plan_set_flow_config(p, variants[0][0], 0)
    _, x0 = _run(p, Dd, Bd, b, dt)
    tol = 1e-4 if dt == btc.F32 else (1e-4 if dt == btc.MIXED_F32 else 1e-11)
    for cap, most in variants[1:]:
        btc.btc_plan_set_flow_config(p, cap, most)
        _, x = _run(p, Dd, Bd, b, dt)
        assert np.abs(x - x0).max() <= tol * np.abs(x0).max(), cap


def test_autotuner_picks_a_compiled_configuration_and_remembers_it():
    N, n, dt = 700, 32, btc.MIXED_F32
    D, B = gen.bt_random(N, n, delta=1.0, seed=3)
    b = gen.rhs(N, n, 1, seed=3)
    Dd, Bd = dev(D, torch.float64), dev(B, torch.float64)
    p0 = btc.btc_plan(N, n, dt)
    btc.btc_plan_set_autotune(p0, False)
    f_ref, x_ref = _run(p0, Dd, Bd, b, dt)
    caps = dict(btc.btc_plan_flow_configs(p0))
    p = btc.btc_plan(N, n, dt)
    assert btc.btc_plan_tuning(p)[2] is False and btc.btc_plan_tuning_interlaced(p)[2] is False
    # the interlaced call tunes its own launch; its trial runs do not disturb the right-hand side
    _, x = _run(p, Dd, Bd, b, dt)
    cap, ctas, tuned = btc.btc_plan_tuning_interlaced(p)
    assert tuned and np.array_equal(x, x_ref)
    assert cap in caps and ctas >= 1
    assert btc.btc_plan_tuning(p)[2] is False, "the plain launch is tuned on its first use"
    btc.btc_factor(p, Dd, Bd)
    pcap, pctas, ptuned = btc.btc_plan_tuning(p)
    assert ptuned and pcap in caps and 1 <= pctas <= caps[pcap]
    f = btc.btc_get_factor(p)
    assert np.array_equal(f[0], f_ref[0]) and np.array_equal(f[1], f_ref[1])
    q = btc.btc_plan(N, n, dt)  # same shape: the remembered configurations, no new timing runs
    _run(q, Dd, Bd, b, dt)
    assert btc.btc_plan_tuning_interlaced(q) == (cap, ctas, True)
    btc.btc_factor(q, Dd, Bd)
    assert btc.btc_plan_tuning(q) == (pcap, pctas, True)
    with pytest.raises(btc.BtcError):
        btc.btc_plan_set_flow_config(q, 5, 1)
