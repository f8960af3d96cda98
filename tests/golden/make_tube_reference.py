"""Writes tests/golden/tube256_axis_phi.txt with the FP64 oracle only: the
capillary-tube workload of the Washburn test (Sec. IV.A, Type-I Zou-He
pressure drive; D3Q19 tube of radius 8 in a 20 x 20 cross-section, 256
long, red in the first 32 layers, rho_in / rho_out = 1.01 / 0.99, theta =
90 deg with Scheme-I, tau = 1) run for 20000 steps from its sharp initial
state. Recorded every 4000 steps: the phase field along the tube, averaged
over the four lattice lines nearest the axis (256 values), and the
interface position (red volume over the cross-section's fluid nodes).

Run from the repository root:  python tests/golden/make_tube_reference.py
(about 1e9 node updates; a few minutes on 8 cores)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2407_10914_gb300 import analysis as A  # noqa: E402
from paper_2407_10914_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                   "tube256_axis_phi.txt")
EVERY, STEPS = 4000, 20000


def axis_profile(phi):
    """Mean of phi over the four (y, z) lines nearest the axis (9.5, 9.5)."""
    return phi[9:11, 9:11, :].mean(axis=(0, 1))


def main():
    case = W.tube_3d()
    o = O.Oracle(19, case.solid, case.periodic)
    o.set_params(**case.params)
    o.init_state(case.phi0)
    lines = ["# FP64 oracle, capillary tube 256 x 20 x 20, r = 8, Type-I "
             "rho 1.01/0.99, Scheme-I theta 90, tau 1 (workloads.tube_3d()).",
             "# Written by tests/golden/make_tube_reference.py (oracle only).",
             "# Per record: 'step <n> z <interface position>' then the 256 "
             "axis-averaged phi values."]
    for k in range(STEPS // EVERY):
        o.step(EVERY)
        phi = o.fields()["phi"]
        z = A.interface_position(phi, 0, case.solid)
        lines.append(f"step {(k + 1) * EVERY} z {z:.12e}")
        lines.append(" ".join(f"{v:.9e}" for v in axis_profile(phi)))
        print(lines[-2], flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
