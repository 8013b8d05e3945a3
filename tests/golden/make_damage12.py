"""Writes damage12.npz: the FP64 oracle's trajectory of a 12^3 four-grain
polycrystal through damage nucleation and crack growth, for the GPU parity
test of the damaged regime (tests/test_gpu_parity.py).

Calls only the oracle and the seeded input generators.  The workload:
periodic Voronoi grains (seed 31), Table 1 material with tau_c0 = 250 MPa,
full storage of the plastic work (xi_store = 1) and G_crit = 7e-4 N/mm, so
that W_crit is reached at the first tensile peak and the drive of Eq. zeta
turns positive one cycle later; an R = -1 uniaxial-strain cycle of 0.6 %
in 24 increments, repeated; the paper's tolerances.  Damage appears at
increment 25, grows through 28 and runs across the cell at 29-30 at a
fixed load (tens of staggered iterations).  Stored: the statistics of
increments 1-30, phi after increments 25-30 and the degraded stress
g(phi) P after increments 28 and 30, the stress rounded to FP32 (a
relative 6e-8, far below the test's bar for it) to keep the file small.

    python tests/golden/make_damage12.py      # about 8 minutes on one core
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2304_01125_gb300 import inputs as I  # noqa: E402

N_GRID = (12, 12, 12)
INCREMENTS = 30
KEEP_PHI = range(24, 30)  # increments 25-30 (0-based)
KEEP_P = (27, 29)  # increments 28 and 30
STATS = ("stag_it", "newton_it", "lin_it_total", "pf_it_total", "cracked")


def setup():
    gid, eul = I.voronoi(N_GRID, 4, 31)
    mat = I.material("baseline", tau_c0=250.0, G_crit=7e-4, xi_store=1.0)
    prog = I.uniaxial_cycle_program(0.006, 24, 2)[:INCREMENTS]
    return gid, eul, mat, prog, I.solver_options("paper")


def main():
    gid, eul, mat, prog, opts = setup()
    r = O.RVE(N_GRID, I.VOXEL_MM, gid, eul, mat, opts)
    out = {"stats": np.zeros((INCREMENTS, len(STATS)))}
    t0 = time.time()
    for k, (Fb, dt) in enumerate(prog):
        s, st = r.run_increment(Fb, dt)
        assert s == 0, (k, st)
        out["stats"][k] = [st[key] for key in STATS]
        if k in KEEP_PHI:
            out[f"phi_{k}"] = r.field("phi")
        if k in KEEP_P:
            out[f"P_{k}"] = r.field("P").astype(np.float32)
        print(k + 1, {key: st[key] for key in STATS}, f"{time.time() - t0:.0f}s", flush=True)
    np.savez_compressed(os.path.join(HERE, "damage12.npz"), **out)


if __name__ == "__main__":
    main()
