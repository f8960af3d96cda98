"""The oracle's tangent-linear run (its step on forward-mode dual numbers)
against central finite differences of the plain FP64 oracle: dS_w/dtheta and
dS_w/dg_x for the smooth saturation after n steps, on cases where the
contact angle and the body force both act (Scheme-II and Scheme-I drops on
a wall, a periodic pack). This pins the reference that the GPU adjoint is
checked against."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10914_gb300 import workloads as W


def sw_after(case, steps, **over):
    o = O.Oracle(case.lattice, case.solid, case.periodic)
    p = dict(case.params)
    p.update(over)
    o.set_params(**p)
    o.init_state(case.phi0)
    o.step(steps)
    return o.reduce(3)


def tlm_after(case, steps):
    t = O.TangentLinear(case.lattice, case.solid, case.periodic)
    t.set_params(**case.params)
    t.init_state(case.phi0)
    t.step(steps)
    return t.sw()


def richardson(case, steps, key, h):
    """(4 D(h/2) - D(h)) / 3 of central differences D: error O(h^4), so a
    step large enough to keep FP64 round-off of S_w out of the quotient."""
    return (4.0 * central(case, steps, key, h / 2) - central(case, steps, key, h)) / 3.0


def central(case, steps, key, h):
    p = case.params
    if key == "theta":
        th = p["theta_deg"]
        hd = h * 180.0 / math.pi
        return (sw_after(case, steps, theta_deg=th + hd)
                - sw_after(case, steps, theta_deg=th - hd)) / (2 * h)
    g = list(p["g"])
    gp, gm = list(g), list(g)
    gp[0] += h
    gm[0] -= h
    return (sw_after(case, steps, g=tuple(gp))
            - sw_after(case, steps, g=tuple(gm))) / (2 * h)


def drop(wetting, theta):
    c = W.droplet_2d(nx=40, ny=24, radius=9.0, theta_deg=theta,
                     wetting=wetting, steps=40)
    c.params["g"] = (2e-4, 0.0, 0.0)
    return c


CASES = [("drop2d_schemeII", drop(2, 60.0), 40),
         ("drop2d_schemeI", drop(1, 120.0), 40),
         ("pack3d_schemeII", W.adjoint_pack(n=(22, 18, 16), steps=12), 12)]


@pytest.mark.parametrize("name,case,steps", CASES, ids=[c[0] for c in CASES])
def test_tangent_linear_matches_central_differences(name, case, steps):
    J, dth, dg = tlm_after(case, steps)
    assert J == pytest.approx(sw_after(case, steps), rel=1e-13, abs=1e-15)
    fd_th = richardson(case, steps, "theta", 2e-4)
    fd_g = richardson(case, steps, "g", 4e-5)
    assert abs(dth) > 1e-6 and abs(dg) > 1e-6, (dth, dg)  # both act
    assert dth == pytest.approx(fd_th, rel=1e-6), (dth, fd_th)
    assert dg == pytest.approx(fd_g, rel=1e-5), (dg, fd_g)


def test_regularised_linearisation_changes_derivatives_only():
    """freeze_sin / c_min hold directions constant in the linearisation:
    the values (S_w) are those of the plain oracle, and thresholds below
    every node's sin(theta') and |C| leave the derivatives exact."""
    name, case, steps = CASES[0]
    exact = tlm_after(case, steps)

    def run(freeze, cmin):
        t = O.TangentLinear(case.lattice, case.solid, case.periodic)
        t.set_params(**case.params)
        t.set_freeze(freeze)
        t.set_cmin(cmin)
        t.init_state(case.phi0)
        t.step(steps)
        return t.sw()

    tiny = run(1e-12, 1e-12)
    assert tiny == exact
    big = run(1.0, 10.0)
    assert big[0] == pytest.approx(exact[0], rel=1e-13)
    assert big[1] != exact[1]  # the held directions change the derivative
