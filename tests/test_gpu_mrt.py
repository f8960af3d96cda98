"""The MRT collision on the GPU (collision = 1: Eq. 2 in moment space with
the rates of Eqs. 4, 15 and 16) against the FP64 oracle's MRT, which its
own pins fix to the printed M (Eq. A.3), A.4/A.5 and the slip-free
Poiseuille channel.

Same method as the single-rate parity tests: a developed oracle state,
rounded to float32, is loaded into both sides and both take one step
(populations within 1e-6 per colour); 100 steps compare the phase field
(1e-4). The body-forced channel checks the property that sets the MRT rates
apart on the GPU as well: no wall slip, where the single-rate collision at
the same viscosity slips by a fraction of a percent of the peak velocity."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10914_gb300 import workloads as W

from test_gpu_parity import (CASES, TOL_POP, developed, gpu_session,
                             oracle_for, rel_err)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_10914_gb300 import build
    build.build()
    return torch


def mrt(case):
    """The same workload with the MRT collision."""
    c = W.Case(case.name + "_mrt", case.lattice, case.solid, case.periodic,
               case.phi0, dict(case.params, collision=1), case.steps,
               case.info)
    return c


MRT_CASES = [(n + "_mrt", mrt(c), d) for n, c, d in CASES if c.lattice == 19]


@pytest.mark.parametrize("name,case,dev", MRT_CASES,
                         ids=[c[0] for c in MRT_CASES])
def test_one_step_populations_mrt(torch, name, case, dev):
    o, f32 = developed(case, dev)
    s = gpu_session(torch, case)
    s.set_populations(torch.from_numpy(f32))
    o.step(1)
    s.step(1)
    got = s.get_populations().cpu().numpy().astype(np.float64)
    err = rel_err(got, o.pops)
    assert max(err) <= TOL_POP, err
    # the test sees the MRT rates: the single-rate step from the same state
    # misses the MRT result by well over the tolerance (5e-5 on the slow
    # tube flow, more elsewhere)
    b = gpu_session(torch, W.Case(case.name, 19, case.solid, case.periodic,
                                  case.phi0, dict(case.params, collision=0)))
    b.set_populations(torch.from_numpy(f32))
    b.step(1)
    other = b.get_populations().cpu().numpy().astype(np.float64)
    assert max(rel_err(other, o.pops)) > 10 * TOL_POP


# The Type-I Scheme-I pack is held to the one-step bar only: from its
# developed state a difference of a few 1e-6 (float32 against float64) flips
# the direction of Scheme-I's result at one wall node within 60 steps (the
# secant's last update divides by f(v1) - f(v2), whose sign sets the
# direction where Eq. 28 has no root), and the two runs then separate to
# 2e-3 in phi by step 100. The FP64 oracle started from the float32 state
# of step 50 separates from its own run in the same way; a tenth of that
# difference does not.
LONG_MRT = [c for c in MRT_CASES if c[0] != "porous_typeI_schemeI_mrt"][:3]


@pytest.mark.parametrize("name,case,dev", LONG_MRT,
                         ids=[c[0] for c in LONG_MRT])
def test_hundred_steps_phase_field_mrt(torch, name, case, dev):
    o, f32 = developed(case, dev)
    s = gpu_session(torch, case)
    s.set_populations(torch.from_numpy(f32))
    o.step(100)
    s.step(100)
    phi = s.macros()["phi"].cpu().numpy()
    fl = o.geometry()[0] >= 2
    err = np.abs(phi[fl] - o.fields()["phi"][fl]).max()
    assert err <= 1e-4, err


def test_mrt_channel_has_no_slip_gpu(torch):
    """Body-forced D3Q19 channel between halfway bounce-back walls at
    y0 = 0.5 and y1 = ny - 1.5, tau = 0.6: with MRT the steady float32
    profile is the parabola g/(2 nu)(y - y0)(y1 - y) to 1e-3 of its peak
    (float32 accumulation leaves about 3e-4; the FP64 oracle meets it to
    round-off); the single-rate collision misses it by its slip
    g(16L - 3)/(24 nu), L = (tau - 1/2)^2, about 3.5e-3 of the peak."""
    g, ny, tau = 1e-5, 19, 0.6
    nu = (tau - 0.5) / 3
    y = np.arange(ny, dtype=float)[1:-1]
    expect = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    peak = expect.max()
    dev = {}
    for coll in (1, 0):
        case = W.channel_3d(ny=ny, g=g, tau=tau, collision=coll)
        s = gpu_session(torch, case)
        s.init_state(case.phi0.astype(np.float32))
        s.step(30000)
        u = s.macros()["u"].cpu().numpy()
        dev[coll] = np.abs(u[0][:, 1:-1, :] - expect[None, :, None]).max()
        assert np.abs(u[1:, :, 1:-1, :]).max() <= 1e-4 * peak
    assert dev[1] <= 1e-3 * peak, dev
    slip = abs(g * (16 * (tau - 0.5) ** 2 - 3) / (24 * nu))
    assert dev[0] >= 0.5 * slip, dev


def test_mrt_refused_where_undefined(torch):
    """MRT is defined for D3Q19 only (Appendix A), and the adjoint does not
    differentiate it: both are refused with LBM_ERR_ARG."""
    from paper_2407_10914_gb300 import lbm
    case = W.channel_2d(nx=4, ny=9)
    s = gpu_session(torch, case)
    with pytest.raises(lbm.LbmError):
        s.set_params(**dict(case.params, collision=1))
    case3 = W.channel_3d(collision=1)
    s3 = gpu_session(torch, case3)
    s3.init_state(case3.phi0.astype(np.float32))
    ws = torch.empty(lbm.lbm_adj_workspace_bytes(s3.h), dtype=torch.uint8,
                     device="cuda")
    with pytest.raises(lbm.LbmError):
        lbm.lbm_adj_create(s3.h, ws)
