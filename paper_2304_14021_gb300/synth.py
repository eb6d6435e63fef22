"""Seeded synthetic inputs shared by the tests, the oracle runs and the bench.

This module holds no arithmetic of the method: it only draws initial data and
initial iterates (numpy PCG64 streams keyed by an integer seed) and evaluates
the closed-form initial conditions of the workloads on their grid points.
"""
from __future__ import annotations

import numpy as np


def grid_points_1d(n: int, bc: str) -> np.ndarray:
    """Vertex grid (n interior points of [0,1]) for "ss"; cell centres for
    "neumann"; n vertices including both ends for "neumann_v"."""
    if bc == "ss":
        return np.arange(1, n + 1) / (n + 1)
    if bc == "neumann_v":
        return np.arange(n) / (n - 1)
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


def batched_instances(n: int, seed: int, alpha: float = 1e-2, max_dof: int | None = None) -> list[dict]:
    """n seeded independent problems mixing the three equations:
    equation uniform over {biharmonic, linear_ch, cahn_hilliard}, dim uniform
    over {1, 2}; 1-D nx = 2^U{6..12}, 2-D nx = ny = 2^U{6..9}; N_t = 2^U{4..9};
    eps ~ U[0.01, 0.1], beta ~ U[0, 1/sqrt 3]; cell-centred Neumann grids;
    alpha fixed.  Final times: biharmonic 0.01; linearized CH
    min(0.1, ln(0.1/alpha) / (beta^4 / (4 eps^2))) so that the growing modes stay
    within alpha * growth <= 0.1; Cahn-Hilliard one window of T = 2 eps^2.
    Initial data: biharmonic a random mix of three cosine modes, linearized CH
    uniform[-0.05, 0.05], Cahn-Hilliard 0.1 uniform[-1, 1] minus its mean.
    Each item: {"problem": dict of solver keywords, "u0": array, "dof": int}."""
    rng = np.random.default_rng(seed)
    eqs = ["biharmonic", "linear_ch", "cahn_hilliard"]
    out = []
    while len(out) < n:
        eq = eqs[rng.integers(0, 3)]
        dim = int(rng.integers(1, 3))
        nx = 2 ** int(rng.integers(6, 13)) if dim == 1 else 2 ** int(rng.integers(6, 10))
        ny = nx if dim == 2 else 1
        nt = 2 ** int(rng.integers(4, 10))
        eps = float(rng.uniform(0.01, 0.1))
        beta = float(rng.uniform(0.0, 1.0 / np.sqrt(3.0)))
        if eq == "biharmonic":
            T = 0.01
        elif eq == "linear_ch":
            grow = beta ** 4 / (4.0 * eps ** 2)
            T = 0.1 if grow == 0.0 else float(min(0.1, np.log(0.1 / alpha) / grow))
        else:
            T = 2.0 * eps ** 2
        ns = nx * ny
        if max_dof is not None and ns * nt > max_dof:
            continue
        x = (np.arange(nx) + 0.5) / nx
        if eq == "biharmonic":
            ks = rng.integers(1, 6, size=3)
            amp = rng.uniform(-1.0, 1.0, size=3)
            if dim == 1:
                u0 = sum(a * np.cos(k * np.pi * x) for k, a in zip(ks, amp))
            else:
                y = x
                u0 = sum(a * np.outer(np.cos(k * np.pi * y), np.cos(k * np.pi * x)).ravel() for k, a in zip(ks, amp))
        elif eq == "linear_ch":
            u0 = rng.uniform(-0.05, 0.05, ns)
        else:
            v = 0.1 * rng.uniform(-1.0, 1.0, ns)
            u0 = v - v.mean()
        prob = dict(equation=eq, dim=dim, nx=nx, ny=ny, bc="neumann", eps=eps, beta=beta, T=T, nt=nt,
                    n_windows=1, alpha=alpha)
        out.append({"problem": prob, "u0": np.ascontiguousarray(u0, dtype=np.float64), "dof": ns * nt})
    return out
