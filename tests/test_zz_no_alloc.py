"""lbm_colour_mass_noalloc: the colour-mass reduction for callers that
cannot allocate device memory (they run under a device-memory budget that
another framework reserved up front, or under a policy that forbids
allocation after start-up). Its red and blue masses must match lbm_reduce's
LBM_MASS_R / LBM_MASS_B on the same state within the tolerance of the mass
reductions in test_gpu_parity.py (1e-6 of the total mass), on two calls in
a row, each on a different state."""
import numpy as np
import pytest

from paper_2407_10914_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["d3q19", "d2q9"])
def test_colour_mass_noalloc_matches_reduce(which):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_10914_gb300 import build, lbm
    build.build()
    if which == "d3q19":
        case = W.droplet_3d(side=24, radius=7.0, theta_deg=70.0, wetting=2,
                            shape=(19, 24, 29))
    else:
        case = W.droplet_2d(nx=70, ny=33, radius=11.0)
    s = lbm.Session(case.lattice, case.solid, case.periodic)
    s.set_params(**case.params)
    s.init_state(case.phi0.astype(np.float32))
    s.step(17)
    for call in range(2):
        pops = s.get_populations()
        red, blue = lbm.lbm_colour_mass_noalloc(case.lattice, pops, s.stream())
        ref_r = s.reduce(lbm.LBM_MASS_R)
        ref_b = s.reduce(lbm.LBM_MASS_B)
        tol = 1e-6 * (ref_r + ref_b)
        assert abs(red - ref_r) <= tol, (call, red, ref_r)
        assert abs(blue - ref_b) <= tol, (call, blue, ref_b)
        s.step(9)
