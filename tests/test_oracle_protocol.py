"""The injected-fluid swap of Sec. II.D.1 (Eqs. 37-38) in the oracle, and
the displacement protocol of Sec. IV.B (paper_2407_10914_gb300.protocol)
driven on the CPU with the oracle as its engine (the oracle has the same
set_params / step / reduce / swap_inlet interface as the GPU session).

Pins of the swap: it is an exact move of mass between colours on the inlet
plane only: every inlet population of the old colour becomes zero, the new
colour's population becomes the old total, nothing else changes, and the
colour masses shift by exactly the inlet's old-colour mass."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10914_gb300 import protocol as P
from paper_2407_10914_gb300 import units as U
from paper_2407_10914_gb300 import workloads as W


def small_case(drive="typeI", shape=(24, 20, 20), seed=5):
    pack = W.sphere_pack(shape, 0.35, rmin=2.5, rmax=4.5, seed=seed,
                         reservoir=3)
    return W.porous_3d(pack=pack, drive=drive, theta_deg=45.0, wetting=1,
                       rho_in=1.01, rho_out=0.99, g_x=1e-4)


def oracle_for(case):
    o = O.Oracle(case.lattice, case.solid, case.periodic)
    o.set_params(**case.params)
    o.init_state(case.phi0)
    return o


def test_swap_inlet_moves_exactly_the_inlet_mass():
    case = small_case()
    o = oracle_for(case)
    o.step(150)  # red has entered through the inlet
    before = o.pops.copy()
    fl = case.solid == 0
    inlet = np.zeros_like(fl)
    inlet[:, :, 0] = fl[:, :, 0]
    assert before[0][:, inlet].sum() > 0  # red at the inlet
    mr, mb = o.reduce(O.MASS_R), o.reduce(O.MASS_B)
    n = o.swap_inlet(1)  # water (b) replaces oil (r)
    assert n == inlet.sum()
    after = o.pops
    # old colour emptied, new colour holds the old total, per population
    assert np.all(after[0][:, inlet] == 0.0)
    np.testing.assert_allclose(after[1][:, inlet],
                               before[0][:, inlet] + before[1][:, inlet],
                               rtol=1e-15, atol=0)
    # nothing else changes
    rest = ~inlet
    np.testing.assert_array_equal(after[:, :, rest], before[:, :, rest])
    # the colour masses shift by the inlet's red mass
    moved = before[0][:, inlet].sum()
    assert o.reduce(O.MASS_R) == pytest.approx(mr - moved, rel=1e-13)
    assert o.reduce(O.MASS_B) == pytest.approx(mb + moved, rel=1e-13)
    assert (o.reduce(O.MASS_R) + o.reduce(O.MASS_B)
            == pytest.approx(mr + mb, rel=1e-14))
    # the inlet phase field is pure b afterwards
    o.step(1)
    with pytest.raises(ValueError):
        o.swap_inlet(2)


def test_swap_inlet_on_another_axis():
    """The inlet is coordinate 0 of the flow axis, whichever axis it is."""
    case = small_case()
    solid = np.ascontiguousarray(np.transpose(case.solid, (2, 1, 0)))
    phi0 = np.ascontiguousarray(np.transpose(case.phi0, (2, 1, 0)))
    o = O.Oracle(19, solid, (True, True, False))
    o.set_params(**dict(case.params, flow_axis=2))
    o.init_state(phi0)
    o.step(60)
    before = o.pops.copy()
    n = o.swap_inlet(1)
    fl = solid == 0
    assert n == fl[0].sum()
    assert np.all(o.pops[0][:, 0][:, fl[0]] == 0.0)
    np.testing.assert_array_equal(o.pops[:, :, 1:], before[:, :, 1:])


def test_drive_parameters():
    case = small_case()
    d1 = P.Displacement(None, case.params, "typeI", length=23.0)
    p = d1.drive_params(0.004)
    assert p["rho_in"] == pytest.approx(case.params["rho_out"] + 0.012)
    assert p["g"] == (0.0, 0.0, 0.0)
    d2 = P.Displacement(None, case.params, "typeII", length=23.0)
    p = d2.drive_params(0.004)
    assert p["rho_in"] == p["rho_out"]
    assert p["g"][0] == pytest.approx(0.004 / 23.0)
    with pytest.raises(ValueError):
        P.Displacement(None, dict(case.params, zou_he=0))


@pytest.mark.parametrize("drive", ["typeI", "typeII"])
def test_protocol_on_the_oracle(drive):
    """Primary drainage lowers S_w, spontaneous imbibition at falling
    pressure raises it back, and forced imbibition swaps the inlet fluid
    and raises it further; P_c carries the sign of the injected fluid and
    converts to Pa with the paper's unit system."""
    case = small_case(drive)
    params = dict(case.params, rho_in=case.params["rho_out"], g=(0, 0, 0),
                  zeta_r=1.0)
    o = O.Oracle(case.lattice, case.solid, case.periodic)
    o.set_params(**params)
    o.init_state(case.phi0)  # full of water (b)
    units = U.Units.from_tau(6e-6, 1000.0, 1e-6, params["tau_b"])
    d = P.Displacement(o, params, drive, length=case.solid.shape[2] - 1,
                       units=units, check_every=200, sw_tol=2e-3,
                       max_steps=600, stop_dsw=0.005)
    curve = d.run(drainage=[0.004, 0.01, 0.02], spontaneous=[0.005, 0.0],
                  forced=[0.004, 0.01])
    stages = [lv.stage for lv in curve]
    assert stages[0] == "drainage" and stages[-1] == "forced"
    dr = [lv for lv in curve if lv.stage == "drainage"]
    sp = [lv for lv in curve if lv.stage == "spontaneous"]
    fo = [lv for lv in curve if lv.stage == "forced"]
    assert dr[-1].sw < 0.9  # oil has entered
    assert all(b.sw <= a.sw + 0.01 for a, b in zip(dr, dr[1:]))
    assert fo[-1].sw > dr[-1].sw  # water came back
    assert all(lv.pc_lbm > 0 for lv in dr) and all(lv.pc_lbm < 0 for lv in fo)
    assert sp[-1].pc_lbm == 0.0
    for lv in curve:
        assert lv.pc_phys == pytest.approx(units.pressure_phys(lv.pc_lbm))
        assert 0.0 <= lv.sw <= 1.0 and 0.0 <= lv.sw_smooth <= 1.0
    # the inlet holds water after the swap
    phi = o.fields()["phi"]
    fl = case.solid[:, :, 0] == 0
    assert np.all(phi[:, :, 0][fl] < 0)
