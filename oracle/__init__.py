"""FP64 CPU oracle for block-tridiagonal Cholesky factor + solve.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers. The product library never imports this package, and this package
imports nothing from the product.

The arithmetic lives in ``oracle.c`` (plain C, double precision, textbook
loops; see its header for which paper passage each routine restates). This
module compiles it with gcc on first use and wraps it with numpy arrays.

Array conventions (all float64, C-contiguous, 0-based node indices):
  D  [N, n, n]   diagonal blocks; only the lower triangle of each is read.
  B  [N-1, n, n] sub-diagonal blocks, B[i] = Psi(i+1, i) (the paper's E_i).
  x, b [N*n, m]  right-hand sides / solutions, row-major.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _compile(src: str, out: str) -> None:
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (plain C, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        _compile(_SRC, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    lib.orc_chol.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int]
    lib.orc_seq_factor.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
    lib.orc_seq_solve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
    lib.orc_seq_solve.restype = None
    lib.orc_assemble.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
    lib.orc_assemble.restype = None
    lib.orc_dense_chol.argtypes = [ctypes.c_int, _dp, _dp]
    lib.orc_gepp_solve.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
    lib.orc_nd_order.argtypes = [ctypes.c_int, _ip]
    lib.orc_bs_chol.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp, _dp, _dp, ctypes.c_int, _ip, _dp]
    lib.orc_bs_reconstruct.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp, _dp, _dp, ctypes.c_int, _ip,
                                       _dp]
    lib.orc_bs_reconstruct.restype = ctypes.c_double
    lib.orc_resid.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
    lib.orc_resid.restype = None
    if hasattr(lib, "orc_arrow_assemble"):  # absent from planted-mistake variants of older source text
        lib.orc_arrow_assemble.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        lib.orc_arrow_assemble.restype = None
        lib.orc_arrow_resid.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp,
                                        _dp]
        lib.orc_arrow_resid.restype = None
    if hasattr(lib, "orc_band_assemble"):
        lib.orc_band_assemble.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
        lib.orc_band_assemble.restype = None
        lib.orc_band_resid.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.orc_band_resid.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


class use_variant:
    """Context manager that swaps in a library compiled from modified oracle
    source text (used by tests that plant a mistake in the oracle and check
    that the pins catch it). Restores the real oracle on exit."""

    def __init__(self, source_text: str, tag: str):
        os.makedirs(_BUILD, exist_ok=True)
        self.src = os.path.join(_BUILD, f"variant_{tag}.c")
        self.out = os.path.join(_BUILD, f"libvariant_{tag}.so")
        with open(self.src, "w") as f:
            f.write(source_text)

    def __enter__(self):
        global _lib
        _compile(self.src, self.out)
        _load()
        self.saved = _lib
        _lib = _bind(ctypes.CDLL(self.out))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_dp)


def _pi(a):
    return a.ctypes.data_as(_ip)


class NotSPD(ArithmeticError):
    """A pivot was not positive; ``info`` carries the oracle's failure code."""

    def __init__(self, info):
        super().__init__(f"matrix not positive definite (info={info})")
        self.info = info


def chol(A):
    """Unblocked Cholesky-Crout of one SPD matrix (lower triangle read)."""
    A = _f64(A)
    n = A.shape[0]
    L = np.zeros_like(A)
    info = _load().orc_chol(n, _p(A), n, _p(L), n)
    if info:
        raise NotSPD(info)
    return L


def seq_factor(D, B):
    """Alg. 1 (Sec. 3): natural-order factor. Returns (Dhat [N,n,n], Ehat [N-1,n,n])."""
    D, B = _f64(D), _f64(B)
    N, n = D.shape[0], D.shape[1]
    if B.size == 0:
        B = np.zeros((max(N - 1, 0), n, n))
    Dh = np.zeros_like(D)
    Eh = np.zeros((max(N - 1, 0), n, n))
    info = _load().orc_seq_factor(N, n, _p(D), _p(B) if B.size else _p(np.zeros(1)), _p(Dh),
                                  _p(Eh) if Eh.size else _p(np.zeros(1)))
    if info:
        raise NotSPD(info)
    return Dh, Eh


def seq_solve(Dh, Eh, b):
    """Solve Psi x = b with the Alg. 1 factor; b is [N*n, m] (or [N*n])."""
    Dh, Eh = _f64(Dh), _f64(Eh)
    N, n = Dh.shape[0], Dh.shape[1]
    b = _f64(b)
    vec = b.ndim == 1
    x = b.reshape(N * n, -1).copy()
    m = x.shape[1]
    _load().orc_seq_solve(N, n, m, _p(Dh), _p(Eh) if Eh.size else _p(np.zeros(1)), _p(x))
    return x.reshape(-1) if vec else x


def solve(D, B, b):
    """x = Psi^{-1} b via Alg. 1 factor + block substitution."""
    Dh, Eh = seq_factor(D, B)
    return seq_solve(Dh, Eh, b)


def assemble(D, B):
    """Dense symmetric Psi of size (N n) x (N n)."""
    D, B = _f64(D), _f64(B)
    N, n = D.shape[0], D.shape[1]
    A = np.zeros((N * n, N * n))
    _load().orc_assemble(N, n, _p(D), _p(B) if B.size else _p(np.zeros(1)), _p(A))
    return A


def dense_chol(A):
    A = _f64(A)
    M = A.shape[0]
    L = np.zeros_like(A)
    info = _load().orc_dense_chol(M, _p(A), _p(L))
    if info:
        raise NotSPD(info)
    return L


def gepp_solve(A, b):
    """Gaussian elimination with partial pivoting (brute force, tiny inputs)."""
    A = _f64(A)
    b = _f64(b)
    vec = b.ndim == 1
    bb = b.reshape(A.shape[0], -1).copy()
    x = np.zeros_like(bb)
    info = _load().orc_gepp_solve(A.shape[0], bb.shape[1], _p(A), _p(bb), _p(x))
    if info:
        raise ZeroDivisionError(f"singular at step {info}")
    return x.reshape(-1) if vec else x


def nd_order(N):
    """P_inf elimination order (0-based nodes) and the number of levels."""
    order = np.zeros(N, dtype=np.int32)
    levels = _load().orc_nd_order(N, _pi(order))
    return order, levels


def bs_chol(D, B, order):
    """Right-looking block Cholesky of P Psi P^T for an arbitrary order.

    Returns (Ldiag [N,n,n] by node, pairs [nnz,2] (row node, col node), Loff [nnz,n,n])
    where Loff[e] = L(pairs[e,0], pairs[e,1]) and the row node is eliminated
    after the column node.
    """
    D, B = _f64(D), _f64(B)
    N, n = D.shape[0], D.shape[1]
    order = np.ascontiguousarray(order, dtype=np.int32)
    cap = max(4 * N, 8)
    while True:
        Ld = np.zeros_like(D)
        pairs = np.zeros((cap, 2), dtype=np.int32)
        Loff = np.zeros((cap, n, n))
        ret = _load().orc_bs_chol(N, n, _pi(order), _p(D), _p(B) if B.size else _p(np.zeros(1)), _p(Ld), cap,
                                  _pi(pairs), _p(Loff))
        if ret == -1:
            cap *= 4
            continue
        if ret < -1:
            raise NotSPD(-ret - 2)
        return Ld, pairs[:ret].copy(), Loff[:ret].copy()


def bs_reconstruct(D, B, order, Ldiag, pairs, Loff):
    """||P Psi P^T - L L^T||_F / ||Psi||_F, block-sparse."""
    D, B = _f64(D), _f64(B)
    N, n = D.shape[0], D.shape[1]
    order = np.ascontiguousarray(order, dtype=np.int32)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32)
    Ldiag, Loff = _f64(Ldiag), _f64(Loff)
    return _load().orc_bs_reconstruct(N, n, _pi(order), _p(D), _p(B) if B.size else _p(np.zeros(1)), _p(Ldiag),
                                      pairs.shape[0], _pi(pairs) if pairs.size else _pi(np.zeros(2, np.int32)),
                                      _p(Loff) if Loff.size else _p(np.zeros(1)))


def resid(D, B, x, b):
    """(||b - Psi x||_inf, ||Psi||_inf, ||x||_inf) with max over RHS columns."""
    D, B = _f64(D), _f64(B)
    N, n = D.shape[0], D.shape[1]
    x = _f64(x).reshape(N * n, -1)
    b = _f64(b).reshape(N * n, -1)
    out = np.zeros(3)
    _load().orc_resid(N, n, x.shape[1], _p(D), _p(B) if B.size else _p(np.zeros(1)), _p(x), _p(b), _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def relres(D, B, x, b):
    """||b - Psi x||_inf / (||Psi||_inf ||x||_inf)."""
    r, a, xn = resid(D, B, x, b)
    return r / (a * xn) if a * xn > 0 else r


def nd_factor(D, B):
    """The nested-dissection factor: bs_chol in the P_inf order."""
    order, _ = nd_order(D.shape[0])
    return (order,) + bs_chol(D, B, order)


def logdet_from_diag(Ldiag):
    """log det Psi = 2 sum log diag(L)."""
    d = np.diagonal(np.asarray(Ldiag), axis1=-2, axis2=-1)
    return float(2.0 * np.log(d).sum())


# ---------------------------------------------------------------- arrow (bordered) systems
# Psi_a = [[Psi, C^T], [C, A]]: the block-tridiagonal Psi bordered by m dense coupling rows C
# [m, N n] and a dense block A [m, m] (lower triangle read). Vectors have N n + m entries.

def arrow_assemble(D, B, C, A):
    """Dense bordered matrix of size N n + m."""
    D, B, C, A = _f64(D), _f64(B), _f64(C), _f64(A)
    N, n, m = D.shape[0], D.shape[1], C.shape[0]
    M = N * n + m
    out = np.zeros((M, M))
    _load().orc_arrow_assemble(N, n, m, _p(D), _p(B) if B.size else _p(np.zeros(1)), _p(C), _p(A), _p(out))
    return out


def arrow_solve(D, B, C, A, b):
    """x = Psi_a^{-1} b by Gaussian elimination with partial pivoting on the assembled matrix (the plain
    definition; small inputs)."""
    return gepp_solve(arrow_assemble(D, B, C, A), b)


def arrow_resid(D, B, C, A, x, b):
    """(||b - Psi_a x||_inf, ||Psi_a||_inf, ||x||_inf) for one right-hand side, without assembling."""
    D, B, C, A = _f64(D), _f64(B), _f64(C), _f64(A)
    N, n, m = D.shape[0], D.shape[1], C.shape[0]
    out = np.zeros(3)
    _load().orc_arrow_resid(N, n, m, _p(D), _p(B) if B.size else _p(np.zeros(1)), _p(C), _p(A),
                            _p(_f64(x).reshape(-1)), _p(_f64(b).reshape(-1)), _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def arrow_relres(D, B, C, A, x, b):
    r, a, xn = arrow_resid(D, B, C, A, x, b)
    return r / (a * xn) if a * xn > 0 else r


# ---------------------------------------------------------------- block-banded systems (conclusion)
def band_assemble(A):
    """Dense block-banded Psi from A [w+1, Nb, b, b], A[k, i] = Psi(i+k, i)."""
    A = _f64(A)
    w, Nb, b = A.shape[0] - 1, A.shape[1], A.shape[2]
    out = np.zeros((Nb * b, Nb * b))
    _load().orc_band_assemble(Nb, b, w, _p(A), _p(out))
    return out


def band_resid(A, x, rhs):
    """(||rhs - Psi x||_inf, ||Psi||_inf, ||x||_inf) for the block-banded Psi, maxima over columns."""
    A = _f64(A)
    w, Nb, b = A.shape[0] - 1, A.shape[1], A.shape[2]
    x = _f64(x).reshape(Nb * b, -1)
    rhs = _f64(rhs).reshape(Nb * b, -1)
    out = np.zeros(3)
    _load().orc_band_resid(Nb, b, w, x.shape[1], _p(A), _p(x), _p(rhs), _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def band_relres(A, x, rhs):
    r, a, xn = band_resid(A, x, rhs)
    return r / (a * xn) if a * xn > 0 else r


def band_solve(A, rhs):
    """x = Psi^{-1} rhs by the dense Cholesky of the assembled band (the plain definition; small inputs)."""
    M = band_assemble(A)
    L = dense_chol(M)
    y = np.linalg.solve(L, _f64(rhs).reshape(M.shape[0], -1))
    return np.linalg.solve(L.T, y)


def band_group(A, w):
    """The block-tridiagonal view of a block-banded Psi: w consecutive block rows per super-row,
    D'_I(p, q) = Psi(Iw + p, Iw + q), B'_I(p, q) = Psi((I+1)w + p, Iw + q); a ragged last super-row is
    padded with identity blocks. Plain index bookkeeping (no arithmetic) -> (D' [N, wb, wb], B' [N-1, wb, wb])."""
    A = _f64(A)
    Nb, b = A.shape[1], A.shape[2]
    N, n = -(-Nb // w), w * b

    def blk(I, J):  # block (I, J) of Psi, or None outside the band / matrix
        if I >= Nb or J >= Nb or abs(I - J) > w:
            return None
        if I == J:
            lo = np.tril(A[0, I])
            return lo + np.tril(lo, -1).T
        return A[I - J, J] if I > J else A[J - I, I].T

    Dg = np.zeros((N, n, n))
    Bg = np.zeros((max(N - 1, 0), n, n))
    for I in range(N):
        for p in range(w):
            for q in range(w):
                v = blk(I * w + p, I * w + q)
                if v is not None:
                    Dg[I, p * b:(p + 1) * b, q * b:(q + 1) * b] = v
                elif p == q:
                    Dg[I, p * b:(p + 1) * b, q * b:(q + 1) * b] = np.eye(b)
                if I + 1 < N:
                    v = blk((I + 1) * w + p, I * w + q)
                    if v is not None:
                        Bg[I, p * b:(p + 1) * b, q * b:(q + 1) * b] = v
    return Dg, Bg


# ---------------------------------------------------------------- partition permutation (Sec. 4.1)
def partition_sizes(N, p):
    """Chunk sizes (N_1, N_k) of the partition permutation with p chunks and p - 1 pivots (Sec. 4.1,
    Proposition 1): N_k* = (7N - 7p + 7) / (7p + 12) rounded down and up, N_1 = N - (p - 1)(N_k + 1),
    keeping the pair whose larger phase cost max((7/3) N_1 - 1, (19/3) N_k - 1) is smaller. Chunks of
    k > 1 hold at least one node; p = 1 is the sequential order."""
    if p <= 1:
        return N, 0
    best = None
    nk_star = (7 * N - 7 * p + 7) / (7 * p + 12)
    for nk in (int(np.floor(nk_star)), int(np.ceil(nk_star))):
        nk = max(nk, 1)
        n1 = N - (p - 1) * (nk + 1)
        if n1 < 1:
            continue
        cost = max(7.0 / 3.0 * n1 - 1.0, 19.0 / 3.0 * nk - 1.0)
        if best is None or cost < best[0]:
            best = (cost, n1, nk)
    if best is None:
        raise ValueError(f"{p} chunks do not fit in N = {N}")
    return best[1], best[2]


def partition_order(N, p):
    """Elimination order of Psi_p (0-based nodes): the interiors of the p chunks (chunk 1 = nodes
    0 .. N_1-1; chunk k > 1 = the N_k nodes after pivot A_k), each in ascending order, then the pivots
    A_2 .. A_p in ascending order (the sequential phase)."""
    n1, nk = partition_sizes(N, p)
    chunks = [list(range(n1))]
    pivots = []
    v = n1
    for _ in range(p - 1):
        pivots.append(v)
        chunks.append(list(range(v + 1, v + 1 + nk)))
        v += 1 + nk
    assert v == N
    order = [i for c in chunks for i in c] + pivots
    return np.asarray(order, dtype=np.int32)


def partition_factor(D, B, p):
    """The factor of Psi_p: bs_chol in the partition order."""
    order = partition_order(D.shape[0], p)
    return (order,) + bs_chol(D, B, order)
