"""Washburn Case-I on the GPU (Sec. IV.A.1): the wetting fluid b enters the
paper's 12 x 12 x 101 tube of radius 5 at equal end pressures and displaces
r (viscosity ratio 1/5); the interface path follows Eq. (49). Measured area
errors (the paper's metric, from the settled start to t* = 60) are 0.03-0.3 %
at 45-75 deg with either wetting scheme; the bound below is 1 %."""
import numpy as np
import pytest

from paper_2407_10914_gb300 import washburn as Wb
from paper_2407_10914_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_10914_gb300 import build, lbm
    build.build()
    return lbm


@pytest.mark.parametrize("wetting", [1, 2])
@pytest.mark.parametrize("theta", [45.0, 75.0])
def test_case1_follows_washburn(lbm, theta, wetting):
    case = W.washburn_tube(theta, wetting)

    def make(params):
        s = lbm.Session(19, case.solid, case.periodic)
        s.set_params(**params)
        s.init_state(case.phi0.astype(np.float32))
        return s

    r = Wb.run_case1(make, case, theta, wetting, tstar_end=60.0)
    assert len(r["tstar"]) > 20
    assert np.all(np.diff(r["zstar"]) > -1e-3)  # the interface advances
    assert r["area_error"] < 0.01, r["area_error"]


def test_case2_pressure_driven(lbm):
    """Case-II (Sec. IV.A.2): neutral wetting, a pressure drop imposed by the
    Zou-He densities (Type-I) or an equivalent body force (Type-II). The
    path follows Eq. (49) within 8 % (measured 3.5-5 %: the staircase tube
    of radius 5 carries a little less flux than a round one), and the two
    drives agree within 1 %."""
    case = W.washburn_tube(90.0, 1)

    def make(params):
        s = lbm.Session(19, case.solid, case.periodic)
        s.set_params(**params)
        s.init_state(case.phi0.astype(np.float32))
        return s

    dp = 0.02 * 2 * case.info["length"] * case.params["gamma"] / 25.0
    r1 = Wb.run_case2(make, case, dp, "typeI", tstar_end=60.0)
    r2 = Wb.run_case2(make, case, dp, "typeII", tstar_end=60.0)
    for r in (r1, r2):
        assert r["area_error"] < 0.08, r["area_error"]
        assert np.all(np.diff(r["zstar"]) > -1e-3)
    n = min(len(r1["zstar"]), len(r2["zstar"]))
    assert np.abs(r1["zstar"][:n] - r2["zstar"][:n]).max() < 0.01
