"""Writes exact_iterations_linear_ch_256.json: the residual history of the
PinT iteration (Eq. 2.8 applied to the residual of Eq. 2.6, from the zero
iterate) evaluated in FP64 by the oracle, for the 2-D linearized
Cahn-Hilliard benchmark configuration.  The GPU's mixed forms compute the
residual, scaling and update FP64-accurately and the transforms in FP32, so
they should stop within one iteration of this count; a transform whose
rounding leaks into the stiff high modes (which the next residual
multiplies by up to ~c2 Lambda_max^2 dt) shows up as extra iterations.

Case: cell-centred homogeneous Neumann 256 x 256 on [0,1]^2, eps = 0.05,
beta = 0.5, T = 0.1, N_t = 128 (one window), theta = 1, u0 = uniform
[-0.05, 0.05] (synth.u0_uniform, seed 0), alpha in {1e-2, 1e-3}.  Recorded per
alpha: the relative residual ||r_k|| / ||b|| for k = 0..6.

Only oracle/ and the seeded input generator are used.  Run from the repository
root:  python tests/golden/make_exact_iterations_linear_ch_256.py   (a minute or two).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pint_oracle as O  # noqa: E402
from paper_2304_14021_gb300 import synth  # noqa: E402

ITERS = 6


def main() -> None:
    out = {"case": "linear_ch 2-D neumann 256x256 eps 0.05 beta 0.5 T 0.1 nt 128 theta 1, u0 uniform[-0.05,0.05] seed 0, "
                   "zero initial iterate", "history": {}}
    for alpha in (1e-2, 1e-3):
        p = O.Problem(equation=O.LINEAR_CH, dim=2, nx=256, ny=256, bc="neumann", eps=0.05, beta=0.5, T=0.1, nt=128,
                      n_windows=1, theta=1.0, alpha=alpha)
        u0 = synth.u0_uniform(p.nspace, -0.05, 0.05, 0)
        bn = O.rhs_norm(p, u0)
        U = np.zeros((p.nt, p.nspace))
        hist = []
        for _ in range(ITERS + 1):
            r = O.residual(p, u0, U)
            hist.append(float(np.linalg.norm(r) / bn))
            U = U + O.diagonalized_apply_separable(p, alpha, r, None)
        out["history"][f"{alpha:g}"] = hist
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exact_iterations_linear_ch_256.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
