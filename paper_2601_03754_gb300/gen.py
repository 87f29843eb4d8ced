"""Seeded synthetic inputs for block-tridiagonal SPD systems.

This module builds inputs only: it holds none of the factorization or solve
arithmetic, imports nothing else from this package, and serves both the CUDA
path and the CPU oracle, so the two always see the same numbers.

Recipes (all float64, 0-based blocks, B[i] couples blocks i+1 and i):

``bt_random(N, n, delta, seed)``
    B_i entries iid N(0, 1/n); M_i entries iid N(0, 1);
    D_i = M_i M_i^T / n + (||B_{i-1}||_2 + ||B_i||_2 + delta) I, with
    B_{-1} = B_{N-1} = 0. Every eigenvalue of Psi is then >= delta (the
    shift dominates the Gershgorin-style bound sum_i ||B_i|| (|x_i| - |x_{i+1}|)^2
    >= 0), so Psi is SPD; delta controls the conditioning.

``mpc(N, n, seed)``
    Reduced (dual) KKT Hessian G G^T of an equality-constrained LQ problem with
    dynamics x_{k+1} = A_k x_k + Bu_k u_k, Q = R = I: A_k Gaussian scaled to
    spectral radius 0.95, Bu_k of size n x n/2 with entries iid N(0, 1/n).
    Diagonal blocks D_0 = I + Bu_0 Bu_0^T, D_k = I + A_k A_k^T + Bu_k Bu_k^T;
    sub-diagonal blocks B_k = -A_{k+1}.

``arrow(N, n, m, delta, seed)``
    A bordered ("arrow") system [[Psi, C^T], [C, A]]: Psi from bt_random(N, n,
    delta); C of size m x N n with entries iid N(0, 1/(N n)); A = K K^T/m +
    (||C||_2^2 / delta + 1) I with K iid N(0, 1). Since every eigenvalue of Psi
    is >= delta, C Psi^{-1} C^T <= ||C||_2^2 / delta, so the Schur complement
    A - C Psi^{-1} C^T >= I and the bordered matrix is SPD.

``rhs(N, n, m, seed)``
    Right-hand sides [N n, m] with iid N(0, 1) entries.

``batch_specs(count, seed)`` / ``request_stream(...)``
    Size mixes for batched and served workloads.
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed):
    return np.random.default_rng(seed)


def spectral_norms(B):
    """Largest singular value of each block of B [k, n, n] (0 for an empty stack)."""
    if B.shape[0] == 0:
        return np.zeros(0)
    return np.linalg.norm(B, ord=2, axis=(1, 2))


def bt_random(N: int, n: int, delta: float = 1.0, seed: int = 0):
    """Random block-diagonally-dominant SPD block-tridiagonal system -> (D, B)."""
    rng = _rng(seed)
    B = rng.standard_normal((max(N - 1, 0), n, n)) / math.sqrt(n)
    M = rng.standard_normal((N, n, n))
    D = np.matmul(M, np.swapaxes(M, 1, 2)) / n
    s = spectral_norms(B)
    shift = np.full(N, float(delta))
    if N > 1:
        shift[:-1] += s
        shift[1:] += s
    D += shift[:, None, None] * np.eye(n)[None]
    return np.ascontiguousarray(D), np.ascontiguousarray(B)


def spectral_norms_torch(B):
    """Largest singular value of each block of B [k, n, n] (a torch tensor on
    any device): sqrt of the largest eigenvalue of B^T B from a batched
    symmetric eigensolver on the host CPU (fast and exact to rounding, unlike a
    batched SVD on the GPU for many small blocks)."""
    import torch
    Bc = B.detach().to("cpu")
    w = torch.linalg.eigvalsh(Bc.transpose(1, 2) @ Bc)
    return w[:, -1].clamp_min(0).sqrt().to(B.device)


def bt_random_torch(N: int, n: int, delta: float = 1.0, seed: int = 0, device="cuda", dtype=None):
    """The bt_random recipe drawn with torch's generator directly on `device`
    (for large batched workloads; the numbers differ from bt_random's)."""
    import torch
    dtype = dtype or torch.float64
    gen_ = torch.Generator(device=device)
    gen_.manual_seed(seed)
    B = torch.randn((max(N - 1, 0), n, n), generator=gen_, device=device, dtype=dtype) / math.sqrt(n)
    M = torch.randn((N, n, n), generator=gen_, device=device, dtype=dtype)
    D = M @ M.transpose(1, 2) / n
    shift = torch.full((N,), float(delta), device=device, dtype=dtype)
    if N > 1:
        s = spectral_norms_torch(B)
        shift[:-1] += s
        shift[1:] += s
    D += shift[:, None, None] * torch.eye(n, device=device, dtype=dtype)[None]
    return D.contiguous(), B.contiguous()


def mpc_torch(N: int, n: int, seed: int = 0, device="cuda"):
    """MPC-like reduced KKT Hessian drawn on `device` for large serving pools.
    Same structure as mpc(); the stable dynamics are A_k = 0.95 Q_k with Q_k a
    random orthogonal matrix (QR of a Gaussian), so every eigenvalue of A_k has
    modulus 0.95 without a per-block eigenvalue solve."""
    import torch
    if n % 2:
        raise ValueError("mpc generator needs an even block size (inputs of size n/2)")
    g_ = torch.Generator(device=device)
    g_.manual_seed(seed)
    G = torch.randn((N, n, n), generator=g_, device=device, dtype=torch.float64)
    Q, Rr = torch.linalg.qr(G)
    Q = Q * torch.sign(torch.diagonal(Rr, dim1=1, dim2=2))[:, None, :]
    A = 0.95 * Q
    Bu = torch.randn((N, n, n // 2), generator=g_, device=device, dtype=torch.float64) / math.sqrt(n)
    D = torch.eye(n, device=device, dtype=torch.float64)[None] + Bu @ Bu.transpose(1, 2)
    D[1:] += A[1:] @ A[1:].transpose(1, 2)
    B = -A[1:].clone()
    return D.contiguous(), B.contiguous()


def _stable_dynamics(rng, count, n, radius=0.95):
    A = rng.standard_normal((count, n, n))
    if count == 0:
        return A
    rho = np.abs(np.linalg.eigvals(A)).max(axis=1)
    return A * (radius / rho)[:, None, None]


def mpc(N: int, n: int, seed: int = 0, return_parts: bool = False):
    """MPC-like reduced KKT Hessian -> (D, B); see the module docstring.

    With ``return_parts`` also returns the dynamics (A [N,n,n], Bu [N,n,n/2]).
    """
    if n % 2:
        raise ValueError("mpc generator needs an even block size (inputs of size n/2)")
    rng = _rng(seed)
    A = _stable_dynamics(rng, N, n)  # A[k] for k = 0..N-1; A[0] unused by D_0
    Bu = rng.standard_normal((N, n, n // 2)) / math.sqrt(n)
    eye = np.eye(n)[None]
    D = eye + np.matmul(Bu, np.swapaxes(Bu, 1, 2))
    D[1:] += np.matmul(A[1:], np.swapaxes(A[1:], 1, 2))
    B = -A[1:].copy()
    if return_parts:
        return np.ascontiguousarray(D), np.ascontiguousarray(B), A, Bu
    return np.ascontiguousarray(D), np.ascontiguousarray(B)


def rhs(N: int, n: int, m: int = 1, seed: int = 0):
    """Right-hand sides [N n, m], iid N(0, 1)."""
    return _rng(seed + 7919).standard_normal((N * n, m))


def toeplitz_kron(N: int, n: int, d: float, e: float):
    """D_i = d I, B_i = e I: Psi = T_N(d, e) kron I_n (closed-form spectrum)."""
    D = np.tile(d * np.eye(n), (N, 1, 1))
    B = np.tile(e * np.eye(n), (max(N - 1, 0), 1, 1))
    return D, B


def batch_specs(count: int = 512, seed: int = 0, sizes=(8, 16, 32, 64), nmin: int = 32, nmax: int = 2048):
    """(N_k, n_k) pairs: n uniform over `sizes`, N log-uniform in [nmin, nmax]."""
    rng = _rng(seed + 104729)
    ns = rng.choice(np.asarray(sizes), size=count)
    Ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count)).round().astype(int)
    Ns = np.clip(Ns, nmin, nmax)
    return [(int(N), int(n)) for N, n in zip(Ns, ns)]


def request_stream(rate: float, count: int, seed: int = 0, sizes=(12, 24, 48, 96), nmin: int = 50,
                   nmax: int = 5000, resolve_frac: float = 0.3):
    """Poisson arrivals of factor+solve requests.

    Returns a list of dicts with arrival time t (s), N, n, and `resolve_of`
    (index of an earlier factor request whose factor is reused with a new
    right-hand side, or -1).
    """
    rng = _rng(seed + 15485863)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    factors = []
    for k in range(count):
        if factors and rng.uniform() < resolve_frac:
            src = int(factors[rng.integers(len(factors))])
            out.append(dict(t=float(t[k]), N=out[src]["N"], n=out[src]["n"], resolve_of=src, seed=k))
        else:
            n = int(rng.choice(np.asarray(sizes)))
            N = int(np.clip(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))), nmin, nmax))
            out.append(dict(t=float(t[k]), N=N, n=n, resolve_of=-1, seed=k))
            factors.append(k)
    return out


def arrow(N: int, n: int, m: int, delta: float = 1.0, seed: int = 0):
    """Bordered block-tridiagonal SPD system -> (D, B, C [m, N n], A [m, m])."""
    D, B = bt_random(N, n, delta=delta, seed=seed)
    rng = _rng(seed + 7919)
    C = rng.standard_normal((m, N * n)) / math.sqrt(N * n)
    K = rng.standard_normal((m, m))
    cn = np.linalg.norm(C, ord=2) if m > 0 else 0.0
    A = K @ K.T / max(m, 1) + (cn * cn / delta + 1.0) * np.eye(m)
    return D, B, np.ascontiguousarray(C), np.ascontiguousarray(A)


def banded(Nb: int, b: int, w: int, delta: float = 1.0, seed: int = 0):
    """Random block-banded SPD system with lower block bandwidth w -> A [w+1, Nb, b, b], A[k, i] = Psi(i+k, i).

    Off-diagonal blocks N(0, 1/b); each diagonal block M M^T / b shifted by the spectral norms of the
    2w off-diagonal blocks of its block row plus delta (block diagonal dominance: SPD, every eigenvalue
    >= delta by the block Gershgorin bound). Blocks with i + k >= Nb are zero."""
    rng = _rng(seed)
    A = np.zeros((w + 1, Nb, b, b))
    for k in range(1, w + 1):
        if Nb > k:
            A[k, :Nb - k] = rng.standard_normal((Nb - k, b, b)) / math.sqrt(b)
    M = rng.standard_normal((Nb, b, b))
    A[0] = np.matmul(M, np.swapaxes(M, 1, 2)) / b
    shift = np.full(Nb, float(delta))
    for k in range(1, w + 1):
        if Nb > k:
            s = spectral_norms(A[k, :Nb - k])
            shift[:Nb - k] += s  # block (i+k, i) lies in block row i + k and (transposed) in block row i
            shift[k:] += s
    A[0] += shift[:, None, None] * np.eye(b)[None]
    return np.ascontiguousarray(A)
