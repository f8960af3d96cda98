"""The hand-written adjoint of the step on the GPU (FP32) against the FP64
tangent-linear oracle: the smooth saturation after n steps and its
gradient with respect to the contact angle and the body force; the
checkpoint interval does not change the gradient; the autograd wrapper
returns the same numbers; cases outside the adjoint's scope are refused."""
import math

import numpy as np
import pytest

from oracle import oracle as O
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


def drop(wetting=2, theta=60.0):
    c = W.droplet_2d(nx=40, ny=24, radius=9.0, theta_deg=theta,
                     wetting=wetting, steps=40)
    c.params["g"] = (2e-4, 0.0, 0.0)
    return c


CASES = [("drop2d_schemeII", drop(), 40),
         ("drop2d_nowetting", drop(wetting=0), 30),
         ("pack3d_small", W.adjoint_pack(n=(22, 18, 16), steps=12), 12),
         ("pack3d_medium", W.adjoint_pack(n=(40, 36, 32), slab=6, steps=60), 60)]


def session(torch, case):
    from paper_2407_10914_gb300 import lbm
    s = lbm.Session(case.lattice, case.solid, case.periodic, "fp32")
    s.set_params(**case.params)
    return s


def tlm(case, steps, g_axis=0, freeze=0.0, cmin=0.0):
    t = O.TangentLinear(case.lattice, case.solid, case.periodic, g_axis)
    t.set_params(**case.params)
    t.set_freeze(freeze)
    t.set_cmin(cmin)
    t.init_state(case.phi0)
    t.step(steps)
    return t.sw()


def compare(torch, case, steps, freeze, cmin):
    """Every gradient component within 1e-3 of the FP64 tangent-linear
    value, relative to the size of the gradient it belongs to: theta on its
    own, g as a vector (a component that nearly cancels, like g_x on a
    drop symmetric in x, is measured against |dJ/dg|). Both sides take the
    same linearisation (freeze: Scheme-II, cmin: the normal n_c)."""
    from paper_2407_10914_gb300.adjoint import Run
    refs = [tlm(case, steps, a, freeze, cmin)
            for a in range(2 if case.lattice == 9 else 3)]
    J_ref, dth_ref = refs[0][0], refs[0][1]
    dg_ref = np.array([r[2] for r in refs] + [0.0] * (3 - len(refs)))
    run = Run(session(torch, case), case.phi0, steps, freeze_sin=freeze,
              c_min=cmin)
    J = run.forward()
    dth, dg = run.backward()
    assert J == pytest.approx(J_ref, rel=2e-5)
    scale = np.abs(dg_ref).max()
    assert scale > 1e-6
    assert np.abs(dg - dg_ref).max() <= 1e-3 * scale, (dg, dg_ref)
    if case.params["wetting"]:
        assert abs(dth_ref) > 1e-6
        assert dth == pytest.approx(dth_ref, rel=1e-3), (dth, dth_ref)
    else:
        assert dth == 0.0 and dth_ref == 0.0


@pytest.mark.parametrize("name,case,steps", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_tangent_linear(torch, name, case, steps):
    """The exact derivative (no regularisation) on short runs."""
    compare(torch, case, steps, 0.0, 0.0)


def test_regularised_adjoint_matches_regularised_tangent_linear(torch):
    """The default regularised linearisation, on both sides, over a run long
    enough for wetting nodes with n_c almost along n_w."""
    case = W.adjoint_pack(n=(40, 36, 32), slab=6, steps=150)
    compare(torch, case, 150, 0.05, 1e-3)


def test_checkpoint_interval_does_not_change_the_gradient(torch):
    from paper_2407_10914_gb300.adjoint import Run
    case, steps = CASES[2][1], CASES[2][2]
    out = []
    for every in (1, 3, steps):
        run = Run(session(torch, case), case.phi0, steps, every=every,
                  freeze_sin=0.0, c_min=0.0)
        run.forward()
        dth, dg = run.backward()
        out.append((dth, dg[0]))
    for dth, dg in out[1:]:
        assert dth == pytest.approx(out[0][0], rel=1e-5)
        assert dg == pytest.approx(out[0][1], rel=1e-5)


def test_autograd_function(torch):
    from paper_2407_10914_gb300.adjoint import Run, SwGradient
    case, steps = CASES[0][1], CASES[0][2]
    s = session(torch, case)
    th = torch.tensor(case.params["theta_deg"], dtype=torch.float64,
                      requires_grad=True)
    g = torch.tensor(case.params["g"], dtype=torch.float64, requires_grad=True)
    J = SwGradient.apply(th, g, s, case.params, case.phi0, steps)
    J.backward()
    run = Run(session(torch, case), case.phi0, steps)
    J2 = run.forward()
    dth, dg = run.backward()
    assert float(J.detach()) == pytest.approx(J2, rel=1e-7)
    # atomics sum in any order: two sweeps agree to float32 rounding of
    # the gradient's largest component
    assert float(th.grad) == pytest.approx(dth * math.pi / 180.0, rel=1e-5)
    assert np.abs(g.grad.numpy() - dg).max() <= 1e-5 * np.abs(dg).max()


def test_adjoint_refuses_cases_out_of_scope(torch):
    from paper_2407_10914_gb300 import lbm
    for case in (drop(wetting=1, theta=120.0),
                 W.tube_3d(nx=24, red_len=8, rho_in=1.02, rho_out=0.98)):
        s = session(torch, case)
        ws = torch.empty(lbm.lbm_adj_workspace_bytes(s.h), dtype=torch.uint8,
                         device="cuda")
        with pytest.raises(lbm.LbmError):
            lbm.lbm_adj_create(s.h, ws)
