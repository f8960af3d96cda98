"""Failure detection of the C-ABI, made on the host: every fault here is an
argument, a state or a value that the library must refuse or report, and
none of them faults the GPU. Argument errors return LBM_ERR_ARG before
anything is enqueued (and the handle keeps working); a call out of order
returns LBM_ERR_STATE; a workspace too small LBM_ERR_NOMEM; a non-finite
value injected into the state is caught by the FP64 reductions
(LBM_ERR_NONFINITE)."""
import numpy as np
import pytest

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


def small():
    return W.droplet_3d(side=16, radius=5.0, theta_deg=60.0, wetting=2)


BAD_PARAMS = [dict(tau_r=0.5), dict(tau_b=0.3), dict(beta=1.5),
              dict(beta=-0.1), dict(gamma=-1.0), dict(rho0=0.0),
              dict(theta_deg=0.0), dict(theta_deg=180.0), dict(wetting=3),
              dict(flow_axis=3), dict(zou_he=2), dict(collision=2),
              dict(g=(float("nan"), 0.0, 0.0)),
              dict(zou_he=1, flow_axis=0)]  # x is periodic in the drop case


@pytest.mark.parametrize("bad", BAD_PARAMS, ids=[str(b) for b in BAD_PARAMS])
def test_bad_parameters_refused(lbm, bad):
    case = small()
    s = lbm.Session(19, case.solid, case.periodic)
    s.set_params(**case.params)
    s.init_state(case.phi0.astype(np.float32))
    before = s.get_populations().cpu().numpy()
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        s.set_params(**dict(case.params, **bad))
    # the refused call left the handle as it was: it still steps
    s.step(2)
    after = s.get_populations().cpu().numpy()
    assert np.isfinite(after).all() and not np.array_equal(before, after)


def test_calls_out_of_order(lbm):
    case = small()
    s = lbm.Session(19, case.solid, case.periodic)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        s.step(1)  # no parameters, no state
    s.set_params(**case.params)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_STATE"):
        s.step(1)  # no state yet
    s.init_state(case.phi0.astype(np.float32))
    s.step(1)


def test_bad_geometry_and_workspace(lbm):
    import torch
    case = small()
    nz, ny, nx = case.solid.shape
    solid = np.ones_like(case.solid)  # no fluid node
    ws = lbm.lbm_workspace_bytes(19, nx, ny, nz, case.solid)
    buf = torch.empty(ws, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(lbm.LbmError, match="LBM_ERR_ARG"):
        lbm.lbm_init_geometry(19, nx, ny, nz, solid, 7, 0, buf, stream)
    small_buf = torch.empty(ws // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LbmError, match="LBM_ERR_NOMEM"):
        lbm.lbm_init_geometry(19, nx, ny, nz, case.solid, 7, 0, small_buf,
                              stream)
    assert lbm.lbm_workspace_bytes(19, nx, ny, 0, None) == 0
    assert lbm.lbm_workspace_bytes(7, nx, ny, nz, None) == 0


def test_non_finite_state_is_reported(lbm):
    """A NaN injected into one population (host-side, through the public
    set_populations) spreads through the step; the FP64 mass reduction
    reports it instead of returning a number."""
    case = small()
    s = lbm.Session(19, case.solid, case.periodic)
    s.set_params(**case.params)
    s.init_state(case.phi0.astype(np.float32))
    s.step(3)
    f = s.get_populations().cpu().numpy()
    fl = np.argwhere(case.solid == 0)[len(np.argwhere(case.solid == 0)) // 2]
    f[0, 5, fl[0], fl[1], fl[2]] = np.nan
    s.set_populations(f)
    s.step(2)
    with pytest.raises(lbm.LbmError, match="LBM_ERR_NONFINITE"):
        s.reduce(lbm.LBM_MASS_R)
    # a clean state makes the handle usable again
    s.init_state(case.phi0.astype(np.float32))
    s.step(1)
    assert np.isfinite(s.reduce(lbm.LBM_MASS_R))
