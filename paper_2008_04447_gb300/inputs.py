"""Seeded synthetic inputs for RQRCP / TRQRCP / TUXV.

This module only draws random numbers and assembles test matrices; it holds
none of the factorisation arithmetic.  Both the CUDA path's tests/benchmark
and the CPU oracle take their inputs from here.

Recipes (all FP64 on the host unless a ``torch`` generator is used):

* ``omega(l, m, seed)``: the Gaussian compression matrix, i.i.d. N(0, 1)
  entries (Sec. 3: a GIID matrix with E||Omega a||^2 = l ||a||^2).
* ``haar(m, r, rng)``: m x r with orthonormal columns, Haar distributed: QR of
  a Gaussian matrix with the signs of diag(R) moved into Q (Mezzadri, 2007).
* ``graded(m, n, decades, seed)``: A = U diag(s) V^T with s_i = 10^(-decades*i/r),
  i = 1..r, r = min(m, n), U and V Haar.  The full-factorisation workloads
  (1000^2 with 8 decades, 16384^2 with 12 decades).
* ``lowrank_plus_noise(m, n, r, noise, seed)``: s_i = i^-2 for i <= r with Haar
  factors, plus ``noise`` * N(0, 1) entries.  The truncated / TUXV workload.
* ``batch_shapes(count, seed)``: the many-small-problems mix: m log-uniform in
  [64, 2048], n log-uniform in [64, min(m, 1024)], k uniform in [16, 128]
  clamped to floor(min(m, n) / 2).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["rng", "omega", "haar", "graded", "lowrank_plus_noise", "batch_shapes",
           "haar_torch", "graded_torch", "lowrank_plus_noise_torch", "omega_torch"]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def omega(l: int, m: int, seed: int) -> np.ndarray:
    """l x m i.i.d. N(0, 1), FP64, C-contiguous (row i = one sketch row)."""
    return rng(seed).standard_normal((l, m))


def haar(m: int, r: int, g: np.random.Generator) -> np.ndarray:
    """m x r matrix with Haar-distributed orthonormal columns (r <= m)."""
    z = g.standard_normal((m, r))
    q, rr = np.linalg.qr(z)
    d = np.sign(np.diag(rr))
    d[d == 0] = 1.0
    return q * d


def graded(m: int, n: int, decades: float, seed: int) -> np.ndarray:
    """U diag(10^(-decades*i/r)) V^T, i = 1..r = min(m, n); FP64 m x n."""
    g = rng(seed)
    r = min(m, n)
    s = 10.0 ** (-decades * np.arange(1, r + 1) / r)
    u = haar(m, r, g)
    v = haar(n, r, g)
    return (u * s) @ v.T


def lowrank_plus_noise(m: int, n: int, r: int, noise: float, seed: int) -> np.ndarray:
    """U diag(i^-2) V^T (i <= r, Haar U, V) + noise * N(0,1); FP64 m x n."""
    g = rng(seed)
    r = min(r, m, n)
    s = np.arange(1, r + 1, dtype=np.float64) ** -2.0
    u = haar(m, r, g)
    v = haar(n, r, g)
    a = (u * s) @ v.T
    if noise:
        a += noise * g.standard_normal((m, n))
    return a


def batch_shapes(count: int, seed: int, m_range=(64, 2048), n_cap=1024, k_range=(16, 128)):
    """List of (m, n, k) for the batched mix (see module docstring)."""
    g = rng(seed)
    out = []
    for _ in range(count):
        m = int(round(math.exp(g.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        n_hi = min(m, n_cap)
        n = int(round(math.exp(g.uniform(math.log(m_range[0]), math.log(max(n_hi, m_range[0]))))))
        n = max(1, min(n, n_hi))
        k = int(g.integers(k_range[0], k_range[1] + 1))
        k = max(1, min(k, min(m, n) // 2))
        out.append((m, n, k))
    return out


# --- device-side generators for the large workloads (torch is plumbing here) ---

def _torch():
    import torch
    _preload_linalg(torch)
    return torch


def _preload_linalg(torch):
    """Load torch's CUDA linear-algebra library by path before its first use.

    torch opens it lazily by name; under some profilers' injection that lookup
    fails, so it is opened here once, globally, from torch's own lib folder.
    """
    import ctypes
    import os
    lib = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(lib) and not getattr(_preload_linalg, "done", False):
        ctypes.CDLL(lib, mode=ctypes.RTLD_GLOBAL)
        _preload_linalg.done = True


def omega_torch(l: int, m: int, seed: int, device="cuda", dtype=None):
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randn((l, m), generator=g, device=device, dtype=dtype or torch.float64)


def haar_torch(m: int, r: int, g, device="cuda"):
    torch = _torch()
    z = torch.randn((m, r), generator=g, device=device, dtype=torch.float64)
    q, rr = torch.linalg.qr(z)
    d = torch.sign(torch.diagonal(rr))
    d[d == 0] = 1.0
    return q * d


def graded_torch(m: int, n: int, decades: float, seed: int, device="cuda"):
    """Device FP64 copy of the ``graded`` recipe (same construction, torch RNG)."""
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    r = min(m, n)
    s = 10.0 ** (-decades * torch.arange(1, r + 1, device=device, dtype=torch.float64) / r)
    u = haar_torch(m, r, g, device)
    v = haar_torch(n, r, g, device)
    return (u * s) @ v.T


def lowrank_plus_noise_parts_torch(m: int, n: int, r: int, noise: float, seed: int, device="cuda"):
    """The parts of ``lowrank_plus_noise_torch``: Haar U (m x r), sigma_i = i^-2,
    Haar V (n x r) and the noise matrix (None when noise is 0), drawn in the
    same order from the same generator."""
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    r = min(r, m, n)
    s = torch.arange(1, r + 1, device=device, dtype=torch.float64) ** -2.0
    u = haar_torch(m, r, g, device)
    v = haar_torch(n, r, g, device)
    nz = noise * torch.randn((m, n), generator=g, device=device, dtype=torch.float64) if noise else None
    return u, s, v, nz


def lowrank_plus_noise_torch(m: int, n: int, r: int, noise: float, seed: int, device="cuda"):
    u, s, v, nz = lowrank_plus_noise_parts_torch(m, n, r, noise, seed, device)
    a = (u * s) @ v.T
    if nz is not None:
        a += nz
    return a
