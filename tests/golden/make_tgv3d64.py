"""Write tests/golden/tgv3d64_oracle.npz: the FP64 oracle's velocity after 5000
steps of the classical 3D Taylor-Green vortex on a periodic 64^3 D3Q19 lattice
(u0 = 0.02) for tau in {0.51, 0.52, 0.55, 0.6}, at 1024 seeded sample cells,
plus the mean kinetic energy over all cells.  Calls only the oracle.

    python tests/golden/make_tgv3d64.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as orc  # noqa: E402
from paper_2307_11752_gb300 import inputs as I  # noqa: E402

N, U0, STEPS, TAUS, SAMPLES = 64, 0.02, 5000, (0.51, 0.52, 0.55, 0.6), 4096
KEEP = 4  # store every 4th of the 4096 drawn cells (1024 cells)


def main():
    m = I.periodic_box(N, N, N)
    cells = I.random_fluid_cells(7, m, SAMPLES)[::KEEP]
    out = {"cells": cells, "n": N, "u0": U0, "steps": STEPS, "taus": np.array(TAUS)}
    for tau in TAUS:
        lat = orc.Lattice(orc.D3Q19, m, tau, periodic=7)
        f = lat.init_equilibrium(*I.tgv3d(N, U0))
        lat.step(f, STEPS)
        rho, u = lat.moments(f)
        key = f"tau{tau:.2f}"
        out[key + "_u"] = u.reshape(3, -1)[:, cells]
        out[key + "_energy"] = float((0.5 * (u ** 2).sum(axis=0)).mean())
        print(key, "mean energy", out[key + "_energy"], flush=True)
    np.savez_compressed(os.path.join(HERE, "tgv3d64_oracle.npz"), **out)


if __name__ == "__main__":
    main()
