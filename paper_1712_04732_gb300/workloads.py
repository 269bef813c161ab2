"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws positions and
charges (numpy PCG64), so that the CUDA path and the FP64 oracle can be fed
the very same arrays.  The paper's own workloads are synthetic as well:
positions uniform in the box and charges uniform in [-1, 1] (Secs. 5.2, 7.1,
7.2); Sec. 7.3 adds dense clouds.

Named workloads (the sizes the tests and the benchmark use):

* ``lattice_3p``    D = 3, N = 1000 uniform, alternating +-1 charges, xi = 8,
                    M = 32, truncated Gaussian P = 8, FP64 (plus the NaCl cell).
* ``free_0p``       D = 0, N = 20000 uniform, q ~ U(-1,1) shifted to zero sum,
                    M = 48, PKB P = 8, xi = 8, extension lambda = 2 (M~ = 64,
                    FFT 128^3), FP32 and FP64, phi + F.
* ``slab_2p``       D = 2, N = 100000 uniform, M = 64, PKB P = 6 (FP32) and
                    P = 10 (FP64), xi = 16.
* ``wire_1p``       D = 1, N = 1.2e6 (1e6 uniform + 2e5 in ten Gaussian blobs,
                    sigma = 0.03), M = 128, PKB P = 8, xi = 32, FP32.
* ``batch_3p2p``    64 systems, N log-uniform in [1e3, 1e5], D in {3, 2}.
"""
from __future__ import annotations

import numpy as np

WORKLOADS = {
    "lattice_3p": dict(D=3, N=1000, L=1.0, xi=8.0, M=32, P=8, window="gaussian",
                       charges="alternating"),
    "free_0p": dict(D=0, N=20000, L=1.0, xi=8.0, M=48, P=8, window="pkb",
                    charges="uniform", lam=2.0),
    "slab_2p": dict(D=2, N=100000, L=1.0, xi=16.0, M=64, P=6, window="pkb",
                    charges="uniform", P_fp64=10),
    "wire_1p": dict(D=1, N=1200000, L=1.0, xi=32.0, M=128, P=8, window="pkb",
                    charges="uniform", clustered=True),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_positions(N: int, L: float = 1.0, seed: int = 1) -> np.ndarray:
    """N points uniform in [0, L)^3, float64, shape (N, 3)."""
    x = rng(seed).random((N, 3)) * L
    return np.minimum(x, np.nextafter(L, 0.0))


def uniform_charges(N: int, seed: int = 1, neutral: bool = True) -> np.ndarray:
    """q ~ U(-1, 1); with ``neutral`` the mean is subtracted (zero net charge)."""
    q = rng(seed + 7919).uniform(-1.0, 1.0, N)
    if neutral:
        q -= q.mean()
    return q


def alternating_charges(N: int) -> np.ndarray:
    """+1, -1, +1, ... (neutral for even N)."""
    q = np.ones(N)
    q[1::2] = -1.0
    return q


def nacl_cell(n: int = 8, L: float = 1.0):
    """Rock-salt cell: n^3 ions on a cubic lattice of spacing a = L/n with
    charges (-1)^(i+j+k)."""
    idx = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    x = idx * (L / n)
    q = np.where(idx.sum(1) % 2 == 0, 1.0, -1.0)
    return x.astype(np.float64), q


def clustered_positions(N_uniform: int, N_blobs: int, n_blobs: int = 10, sigma: float = 0.03,
                        L: float = 1.0, seed: int = 1) -> np.ndarray:
    """N_uniform points uniform in [0,L)^3 plus N_blobs points in n_blobs Gaussian
    clouds (std sigma*L, centres uniform in [0.15, 0.85]^3 L), redrawn until every
    point lies inside the box."""
    g = rng(seed + 104729)
    xu = g.random((N_uniform, 3)) * L
    centres = (0.15 + 0.7 * g.random((n_blobs, 3))) * L
    per = np.full(n_blobs, N_blobs // n_blobs)
    per[: N_blobs % n_blobs] += 1
    blobs = []
    for c, m in zip(centres, per):
        pts = np.empty((0, 3))
        while pts.shape[0] < m:
            cand = c + sigma * L * g.standard_normal((2 * (m - pts.shape[0]) + 8, 3))
            ok = np.all((cand >= 0.0) & (cand < L), axis=1)
            pts = np.concatenate([pts, cand[ok]])
        blobs.append(pts[:m])
    x = np.concatenate([xu] + blobs)
    return np.minimum(x, np.nextafter(L, 0.0))


def make(name: str, seed: int = 1, N: int | None = None):
    """(x, q, spec) for a named workload; ``N`` overrides the particle count
    (the clustered share stays 1/6 of the total)."""
    spec = dict(WORKLOADS[name])
    if N is not None:
        spec["N"] = N
    n = spec["N"]
    if spec.get("clustered"):
        nb = n // 6
        x = clustered_positions(n - nb, nb, L=spec["L"], seed=seed)
    else:
        x = uniform_positions(n, spec["L"], seed)
    if spec["charges"] == "alternating":
        q = alternating_charges(n)
    else:
        q = uniform_charges(n, seed)
    return x, q, spec


def batch_systems(n_sys: int = 64, seed: int = 1, n_min: float = 1e3, n_max: float = 1e5):
    """Independent systems with N log-uniform in [n_min, n_max], alternating D in
    {3, 2}; returns a list of (x, q, D)."""
    g = rng(seed + 15485863)
    out = []
    for i in range(n_sys):
        n = int(10 ** g.uniform(np.log10(n_min), np.log10(n_max)))
        n += n & 1
        x = uniform_positions(n, 1.0, seed * 1000 + i)
        q = uniform_charges(n, seed * 1000 + i)
        out.append((x, q, 3 if i % 2 == 0 else 2))
    return out
