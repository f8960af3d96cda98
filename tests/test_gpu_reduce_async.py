"""lbm_reduce_async + lbm_reduce_value give what lbm_reduce gives, for every
reduction kind, read back step after step into page-locked host memory
without waiting between steps (the same kernel and the same host formula,
so the doubles are equal)."""
import numpy as np
import pytest

from paper_2407_10914_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_10914_gb300 import build
    build.build()
    return torch


def test_async_reductions_equal_synchronous(torch):
    from paper_2407_10914_gb300 import lbm
    pack = W.sphere_pack((41, 37, 29), 0.3, rmin=3.0, rmax=6.0, seed=21,
                         reservoir=4)
    case = W.porous_3d(pack=pack, drive="typeI", theta_deg=45.0, wetting=1,
                       rho_in=1.02, rho_out=0.98)
    kinds = [lbm.LBM_MASS_R, lbm.LBM_MASS_B, lbm.LBM_SW_COUNT,
             lbm.LBM_SW_SMOOTH, lbm.LBM_DP, lbm.LBM_CA_R, lbm.LBM_CA_B]
    a = lbm.Session(case.lattice, case.solid, case.periodic)
    b = lbm.Session(case.lattice, case.solid, case.periodic)
    for s in (a, b):
        s.set_params(**case.params)
        s.init_state(case.phi0.astype(np.float32))
    steps = 6
    raw = torch.zeros((steps, len(kinds), 4), dtype=torch.float64).pin_memory()
    at = raw.data_ptr()
    for t in range(steps):
        a.step(1)
        for j, kind in enumerate(kinds):
            lbm.lbm_reduce_async(a.h, kind, at + 32 * (t * len(kinds) + j),
                                 a.stream())
    torch.cuda.synchronize()
    for t in range(steps):
        b.step(1)
        for j, kind in enumerate(kinds):
            want = b.reduce(kind)
            got = lbm.lbm_reduce_value(b.h, kind,
                                       at + 32 * (t * len(kinds) + j))
            assert got == want, (t, kind, got, want)
