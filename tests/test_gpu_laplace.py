"""The Laplace law on the GPU (Sec. III.A): drops of radius 8-17 in a
periodic 64^3 box with the paper's viscosity ratio and lattice tension
(1/45, i.e. 0.02 N/m in its unit system); the slope of the time-averaged
jump against 2/R is the tension within 3 % (measured 1 %), each drop
within 5 %."""
import numpy as np
import pytest

from paper_2407_10914_gb300 import laplace as Lp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_10914_gb300 import build, lbm
    build.build()
    return lbm


def test_laplace_slope_gpu(lbm):
    def make(case):
        s = lbm.Session(19, case.solid, case.periodic)
        s.set_params(**case.params)
        s.init_state(case.phi0.astype(np.float32))
        return s

    r = Lp.sweep(make, 64, (8.0, 11.0, 14.0, 17.0), steps=6000)
    assert r["error"] < 0.03, r
    g = r["gamma_lbm_input"]
    for dp, R in zip(r["dp_lbm"], r["radii"]):
        assert abs(dp * R / (2 * g) - 1) < 0.05, (dp, R)
    assert r["gamma_phys_sim"] == pytest.approx(0.02 * (1 + (r["gamma_lbm_sim"]
                                                              / g - 1)),
                                                rel=1e-9)
