"""Writes ch_config3_64x64.json: reference values of the oracle's sequential solution
for the Cahn-Hilliard configuration of the benchmark set at a size the CPU oracle
finishes (fully implicit backward Euler, Eq. 4.5, solved step by step by Newton's
method; Sec. 4.1 defines PinT-I as converging to this solution).

Case: 2-D Cahn-Hilliard on [0,1]^2, cell-centred homogeneous Neumann 64 x 64,
eps = 0.02, dt = 1e-4, 2048 steps (8 windows of 256), u0 = 0.1 uniform[-1,1]
minus its mean (synth.u0_ch, seed 0).  Recorded: the mass and discrete energy
(Eq. 1.5) of every 16th time level, and the solution at 64 sampled points
(every 64th grid point) at the end of every window.

Only oracle/ and the seeded input generator are used.  Run from the repository
root:  python tests/golden/make_ch_config3_64.py   (a few minutes).
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pint_oracle as O  # noqa: E402
from paper_2304_14021_gb300 import synth  # noqa: E402

NX, EPS, DT, NT, WINDOWS = 64, 0.02, 1e-4, 256, 8
EVERY_LEVEL, EVERY_POINT = 16, 64


def main() -> None:
    p = O.Problem(equation=O.CAHN_HILLIARD, dim=2, nx=NX, ny=NX, bc="neumann", eps=EPS, T=NT * WINDOWS * DT, nt=NT,
                  n_windows=WINDOWS)
    u = synth.u0_ch(p.nspace, 0)
    levels, mass, energy, ends = [], [], [], []
    for n in range(1, NT * WINDOWS + 1):
        u, _ = O.ch_step_newton(p, u)
        if n % EVERY_LEVEL == 0:
            levels.append(n)
            mass.append(O.discrete_mass(p, u))
            energy.append(O.discrete_energy(p, u))
        if n % NT == 0:
            ends.append({"level": n, "values": [float(v) for v in u[::EVERY_POINT]]})
            print(f"level {n}: energy {energy[-1]:.12g}", flush=True)
    out = {
        "about": "Oracle reference values (sequential backward-Euler Newton, Eq. 4.5) for the 2-D Cahn-Hilliard "
                 "benchmark configuration at 64 x 64; written by make_ch_config3_64.py from oracle/ only.",
        "case": {"equation": "cahn_hilliard", "dim": 2, "nx": NX, "ny": NX, "bc": "neumann", "eps": EPS, "dt": DT,
                 "nt": NT, "n_windows": WINDOWS, "u0": "synth.u0_ch(4096, seed 0)"},
        "citation": "Sec. 4.1 (Eq. 4.5: the fully implicit scheme whose solution PinT-I converges to); "
                    "Sec. 1 Eq. 1.5 (the energy); Sec. 5.3-5.4 (mass and energy of the 2-D runs)",
        "levels": levels, "mass": mass, "energy": energy,
        "sample_every_point": EVERY_POINT, "window_ends": ends,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ch_config3_64x64.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
