"""Shared helpers of the GPU parity tests: device transfer and oracle comparison."""
import numpy as np
import pytest

import oracle
from paper_2601_03754_gb300 import btc, gen

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def tdtype(dt):
    return torch.float32 if dt == btc.F32 else torch.float64


def factor_on_gpu(D, B, dt):
    N, n = D.shape[0], D.shape[1]
    p = btc.btc_plan(N, n, dt)
    Dd = dev(D, tdtype(dt))
    Bd = dev(B if B.size else np.zeros((1, n, n)), tdtype(dt))
    btc.btc_factor(p, Dd, Bd)
    return p, Dd, Bd


def compare_factor_with_oracle(p, D, B, tol):
    """Every GPU factor block against the oracle's P_inf-order block Cholesky.

    The GPU stores each off-diagonal block as U(e, o) = L(o, e)^T, with e the node
    eliminated at that level; the oracle lists L(row, col) with row eliminated
    after col. Returns (max abs error relative to max|L|, reconstruction error of
    the GPU factor)."""
    Dh, U, pairs = btc.btc_get_factor(p)
    order, Ld, opairs, Loff = oracle.nd_factor(D, B)
    scale = max(np.abs(Ld).max(), np.abs(Loff).max() if Loff.size else 0.0)
    err = np.abs(Dh.astype(np.float64) - Ld).max() / scale
    ref = {(int(r), int(c)): blk for (r, c), blk in zip(opairs, Loff)}
    assert len(ref) == len(pairs)
    gl_pairs, gl_blocks = [], []
    for (e, o), u in zip(pairs, U):
        blk = ref[(int(o), int(e))]
        err = max(err, np.abs(u.astype(np.float64).T - blk).max() / scale)
        gl_pairs.append((int(o), int(e)))
        gl_blocks.append(u.astype(np.float64).T)
    rec = oracle.bs_reconstruct(D, B, order, Dh.astype(np.float64), np.array(gl_pairs, dtype=np.int32).reshape(-1, 2),
                                np.array(gl_blocks).reshape(-1, D.shape[1], D.shape[1]))
    return err, rec
