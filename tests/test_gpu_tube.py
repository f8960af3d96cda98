"""The capillary-tube workload run in full on the GPU (Sec. IV.A, Type-I
pressure drive; 256 x 20 x 20, r = 8, 20000 steps from the sharp initial
state): the phase field along the tube stays within 1e-4 of the FP64
oracle's full run (tests/golden/tube256_axis_phi.txt, written by
make_tube_reference.py with the oracle only), and the interface advances
at the speed of the Washburn law for equal viscosities, Eq. (47) with
cos(theta) = 0: dz/dt = r^2 dP / (8 mu L), within 10 % for the nominal
radius (the lattice tube is a staircase; its effective radius is
reported)."""
import os

import numpy as np
import pytest

from paper_2407_10914_gb300 import analysis as A
from paper_2407_10914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden",
                    "tube256_axis_phi.txt")


def golden():
    recs = []
    lines = [ln for ln in open(GOLD) if not ln.startswith("#")]
    for head, vals in zip(lines[0::2], lines[1::2]):
        _, step, _, z = head.split()
        recs.append((int(step), float(z),
                     np.array([float(v) for v in vals.split()])))
    return recs


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_10914_gb300 import build, lbm
    build.build()
    return lbm


def test_tube_full_run(lbm):
    case = W.tube_3d()
    s = lbm.Session(19, case.solid, case.periodic)
    s.set_params(**case.params)
    s.init_state(case.phi0.astype(np.float32))
    ts, zs = [], []
    done = 0
    for step, z_ref, prof_ref in golden():
        s.step(step - done)
        done = step
        phi = s.macros()["phi"].cpu().numpy()
        prof = phi[9:11, 9:11, :].mean(axis=(0, 1))
        assert np.abs(prof - prof_ref).max() <= 1e-4, step
        z = A.interface_position(phi, 0, case.solid)
        assert abs(z - z_ref) <= 1e-3, (step, z, z_ref)
        ts.append(step)
        zs.append(z)
    U = np.polyfit(ts[1:], zs[1:], 1)[0]
    p = case.params
    dP = (p["rho_in"] - p["rho_out"]) / 3
    mu = p["rho0"] * (p["tau_r"] - 0.5) / 3
    L = case.solid.shape[2] - 1
    r = case.info["radius"]
    U_ref = r * r * dP / (8 * mu * L)
    r_eff = np.sqrt(8 * mu * L * U / dP)
    print(f"interface speed {U:.4e} vs Eq. 47 {U_ref:.4e}; r_eff {r_eff:.3f}")
    assert abs(U / U_ref - 1) < 0.10, (U, U_ref, r_eff)
