"""Seeded synthetic inputs shared by the tests, the oracle runs and the bench.

This module holds no arithmetic of the method: it only draws initial data and
initial iterates (numpy PCG64 streams keyed by an integer seed) and evaluates
the closed-form initial conditions of the workloads on their grid points.
"""
from __future__ import annotations

import numpy as np


def grid_points_1d(n: int, bc: str) -> np.ndarray:
    """Vertex grid (n interior points of [0,1]) for "ss"; cell centres for "neumann"."""
    if bc == "ss":
        return np.arange(1, n + 1) / (n + 1)
    return (np.arange(n) + 0.5) / n


def u0_sine_modes(n: int, modes=((1, 1.0), (3, 0.5))) -> np.ndarray:
    """sum_k a_k sin(k pi x) on the vertex grid: sin(pi x) + 0.5 sin(3 pi x) by default."""
    x = grid_points_1d(n, "ss")
    return sum(a * np.sin(k * np.pi * x) for k, a in modes)


def u0_uniform(nspace: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """i.i.d. uniform[lo, hi] values."""
    return np.random.default_rng(seed).uniform(lo, hi, nspace)


def u0_ch(nspace: int, seed: int, amp: float = 0.1) -> np.ndarray:
    """amp * uniform[-1, 1] minus its mean (zero-mass spinodal data)."""
    v = amp * np.random.default_rng(seed).uniform(-1.0, 1.0, nspace)
    return v - v.mean()


def random_iterate(nt: int, nspace: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """A seeded uniform[lo, hi] initial iterate U^0 of shape (nt, nspace)."""
    return np.random.default_rng(seed).uniform(lo, hi, (nt, nspace))
