"""Seeded synthetic Ising instances (inputs only; no simulated-bifurcation arithmetic).

The paper's workloads are Sherrington-Kirkpatrick (SK) instances with all-to-all
couplings J_ij = J_ji drawn from {-1, +1} with equal probability and J_ii = 0
(Results, "SB with thermal fluctuation" and the K2000 / 700-spin studies).  The
named benchmark instances (K2000 and the 100 instances of 700 spins) are not
available, so seeded instances of the same shape and distribution stand in.

This module is shared by the tests, the benchmark and the smoke check.  It holds
only input generation: no force, update, energy or schedule code lives here, so
the CUDA path and the CPU oracle share nothing but their inputs.
"""
from __future__ import annotations

import numpy as np


def sk_pm1(n: int, seed: int) -> np.ndarray:
    """Symmetric +/-1 couplings with zero diagonal, float32 [n, n], row-major.

    One fair bit per unordered pair i < j (numpy PCG64 stream `seed`), mirrored
    to j < i.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2, size=(n, n), dtype=np.int8)
    upper = np.triu(bits * np.int8(2) - np.int8(1), 1)
    j = upper + upper.T
    return j.astype(np.float32)


def sk_gauss(n: int, seed: int) -> np.ndarray:
    """Symmetric N(0, 1) couplings with zero diagonal, float32 [n, n].

    Drawn in float64 (numpy PCG64 stream `seed`), upper triangle mirrored, then
    rounded once to float32.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(size=(n, n))
    upper = np.triu(g, 1)
    return (upper + upper.T).astype(np.float32)


def batch_sizes(count: int, seed: int, lo: int = 100, hi: int = 2000) -> list[int]:
    """Uneven instance sizes N_b uniform on the integers [lo, hi]."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(lo, hi + 1, size=count)]


def sk_batch(count: int, seed: int, lo: int = 100, hi: int = 2000,
             gaussian: bool = False) -> list[np.ndarray]:
    """`count` SK instances of uneven size; instance b uses stream seed*1000003+b."""
    sizes = batch_sizes(count, seed, lo, hi)
    gen = sk_gauss if gaussian else sk_pm1
    return [gen(n, seed * 1000003 + b) for b, n in enumerate(sizes)]


def sign_matrix(rows: int, cols: int, seed: int) -> np.ndarray:
    """Random +/-1 int8 matrix, used to probe exact integer products."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 2, size=(rows, cols), dtype=np.int8) * 2 - 1).astype(np.int8)
