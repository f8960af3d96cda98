"""Parity of the CUDA step (through the C-ABI) with the FP64 oracle.

Method (the same on every case): the oracle develops a state for a few
hundred steps from the seeded initial condition; that state, rounded to
float32, is loaded into both sides; both take one step; the populations are
compared colour by colour as max|f_gpu - f_ref| / max|f_ref| <= 1e-6.
Longer runs compare the phase field (<= 1e-4) and the contact angle
(<= 0.5 deg)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10914_gb300 import analysis as A
from paper_2407_10914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_POP = 1e-6


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_10914_gb300 import build
    build.build()
    return torch


def oracle_for(case):
    o = O.Oracle(case.lattice, case.solid, case.periodic)
    o.set_params(**case.params)
    o.init_state(case.phi0)
    return o


def developed(case, steps):
    o = oracle_for(case)
    o.step(steps)
    f32 = o.pops.astype(np.float32)
    o.pops = f32.astype(np.float64)
    return o, f32


def gpu_session(torch, case, storage="fp32"):
    from paper_2407_10914_gb300 import lbm
    s = lbm.Session(case.lattice, case.solid, case.periodic, storage)
    s.set_params(**case.params)
    return s


def rel_err(got, ref):
    return [float(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max())
            for c in range(2)]


def small_pack(shape=(41, 37, 29), porosity=0.3, seed=21, reservoir=4):
    nx, ny, nz = shape
    return W.sphere_pack((nx, ny, nz), porosity, rmin=3.0, rmax=6.0, seed=seed,
                         reservoir=reservoir)


def cases():
    out = []
    out.append(("droplet2d_schemeII", W.droplet_2d(), 200))
    out.append(("droplet2d_schemeI_120",
                W.droplet_2d(theta_deg=120.0, wetting=1, nx=97, ny=45,
                             radius=15.0), 200))
    pack = small_pack()
    c = W.porous_3d(pack=pack, drive="typeI", theta_deg=45.0, wetting=1,
                    rho_in=1.02, rho_out=0.98)
    out.append(("porous_typeI_schemeI", c, 150))
    c = W.porous_3d(pack=pack, drive="typeII", theta_deg=40.0, wetting=2,
                    g_x=2e-4, invading="b")
    out.append(("porous_typeII_schemeII", c, 150))
    c = W.tube_3d(nx=45, red_len=12, rho_in=1.02, rho_out=0.98)
    out.append(("tube_typeI", c, 150))
    c = W.droplet_3d(side=26, radius=8.0, theta_deg=130.0, wetting=2,
                     shape=(21, 26, 33))
    out.append(("droplet3d_schemeII", c, 120))
    c = W.laplace_drop(19, 24, 6.0, tau_r=1.0, tau_b=0.6)
    out.append(("laplace3d_periodic", c, 100))
    out.append(("zou_he_periodic_edges", edge_drop(), 40))
    return out


def edge_drop(shape=(14, 18, 24), radius=5.0):
    """A red drop centred on the edge where the Zou-He outlet plane (x = nx-1,
    non-periodic) meets the periodic y faces: the stencils there reach
    positions that are off the box on both axes, which wrap on y and clamp
    on x (reading 13 of the off-box rule), so n_c and the curvature at the
    edge nodes come from the far side of the y period."""
    nz, ny, nx = shape
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    dy = np.minimum(y, ny - y)  # distance to the plane y = 0 across the period
    r2 = (x - (nx - 1)) ** 2 + dy ** 2 + (z - nz / 2.0) ** 2
    phi0 = np.tanh((radius - np.sqrt(r2)) / 1.5)
    solid = np.zeros(shape, np.uint8)
    p = W.base_params(tau_r=1.0, tau_b=0.8, gamma=0.01, beta=0.95,
                      zou_he=1, flow_axis=0, rho_in=1.0, rho_out=1.0,
                      zeta_r=0.0)
    return W.Case("edge_drop", 19, solid, (False, True, True),
                  np.ascontiguousarray(phi0), p)


CASES = cases()


@pytest.mark.parametrize("name,case,dev", CASES, ids=[c[0] for c in CASES])
def test_geometry_matches_oracle(torch, name, case, dev):
    s = gpu_session(torch, case)
    cls, nw = s.geometry()
    o = oracle_for(case)
    cls_ref, _, nw_ref = o.geometry()
    np.testing.assert_array_equal(cls.cpu().numpy(), cls_ref)
    np.testing.assert_allclose(nw.cpu().numpy(), nw_ref * (cls_ref == 3),
                               rtol=0, atol=2e-7)
    nn, nf, nsb, nfb = s.counts
    assert nn == case.n_nodes and nf == (cls_ref >= 2).sum()
    assert nsb == (cls_ref == 1).sum() and nfb == (cls_ref == 3).sum()


@pytest.mark.parametrize("name,case,dev", CASES, ids=[c[0] for c in CASES])
def test_one_step_populations(torch, name, case, dev):
    o, f32 = developed(case, dev)
    s = gpu_session(torch, case)
    s.set_populations(torch.from_numpy(f32))
    # the state is held in its post-recolouring form (f'' and q, v); a
    # float32-rounded state comes back to within float32 rounding
    back = s.get_populations().cpu().numpy()
    assert np.abs(back - f32).max() <= 5e-7 * np.abs(f32).max()
    o.step(1)
    s.step(1)
    got = s.get_populations().cpu().numpy().astype(np.float64)
    err = rel_err(got, o.pops)
    assert max(err) <= TOL_POP, err
    # fields of the step: phi (incl. Eq. 34 at solid-boundary nodes), rho, u
    m = s.macros()
    fo = o.fields()
    cls_ref = o.geometry()[0]
    act = cls_ref >= 1
    np.testing.assert_allclose(m["phi"].cpu().numpy()[act], fo["phi"][act],
                               rtol=0, atol=2e-6)
    fl = cls_ref >= 2
    np.testing.assert_allclose(m["rho"].cpu().numpy()[fl], fo["rho"][fl],
                               rtol=2e-6, atol=0)
    np.testing.assert_allclose(m["u"].cpu().numpy()[:, fl], fo["u"][:, fl],
                               rtol=0, atol=2e-6)


@pytest.mark.parametrize("name,case,dev", CASES[:5], ids=[c[0] for c in CASES[:5]])
def test_hundred_steps_phase_field(torch, name, case, dev):
    o, f32 = developed(case, dev)
    s = gpu_session(torch, case)
    s.set_populations(torch.from_numpy(f32))
    o.step(100)
    s.step(100)
    phi = s.macros()["phi"].cpu().numpy()
    fl = o.geometry()[0] >= 2
    err = np.abs(phi[fl] - o.fields()["phi"][fl]).max()
    assert err <= 1e-4, err


@pytest.mark.parametrize("name,case,dev", CASES[:5], ids=[c[0] for c in CASES[:5]])
def test_reductions_match_oracle(torch, name, case, dev):
    from paper_2407_10914_gb300 import lbm
    o, f32 = developed(case, dev)
    s = gpu_session(torch, case)
    s.set_populations(torch.from_numpy(f32))
    o.step(3)
    s.step(3)
    for kind in range(7):
        g = s.reduce(kind)
        r = o.reduce(kind)
        scale = max(abs(r), 1e-12)
        if kind in (lbm.LBM_MASS_R, lbm.LBM_MASS_B):
            assert abs(g - r) <= 1e-6 * max(scale, o.reduce(0) + o.reduce(1))
        elif kind == lbm.LBM_SW_COUNT:
            n = (o.geometry()[0] >= 2).sum()
            assert abs(g - r) * n <= 3  # phi within 1e-6 of zero may flip
        elif kind in (lbm.LBM_CA_R, lbm.LBM_CA_B):
            # scale: the capillary number of the largest velocity present
            p = case.params
            tau = p["tau_r"] if kind == lbm.LBM_CA_R else p["tau_b"]
            umax = np.abs(o.fields()["u"]).max()
            ca_scale = p["rho0"] * (tau - 0.5) / 3 * umax / p["gamma"]
            assert abs(g - r) <= 1e-4 * ca_scale + 1e-12
        elif kind == lbm.LBM_DP:
            assert abs(g - r) <= 1e-6  # float32 densities near 1, over 3
        else:
            assert abs(g - r) <= 1e-5 * max(scale, 1e-3)


STORAGE_TOL = {"fp16": 1e-4, "bf16": 1e-3}


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("name,case,dev", [CASES[0], CASES[2], CASES[4]],
                         ids=[CASES[0][0], CASES[2][0], CASES[4][0]])
def test_one_step_16bit_storage(torch, storage, name, case, dev):
    """16-bit storage of f''_i (offsets from w_i rho0, scaled by 1/w_i);
    the colour fields q, v and all arithmetic stay float32. Stated error
    after one step from the float32 state: 1e-4 (fp16), 1e-3 (bf16)."""
    o, f32 = developed(case, dev)
    s = gpu_session(torch, case, storage)
    s.set_populations(torch.from_numpy(f32))
    o.step(1)
    s.step(1)
    got = s.get_populations().cpu().numpy().astype(np.float64)
    err = rel_err(got, o.pops)
    print(storage, name, err)
    assert max(err) <= STORAGE_TOL[storage], err


def test_droplet_full_run_phase_and_angle(torch):
    """The D2Q9 droplet workload (128 x 64, R = 24, Scheme-II at 60 deg):
    2000 steps from the sharp initial state on both sides; phase field
    within 1e-4, contact angle within 0.5 deg."""
    case = W.droplet_2d()
    o = oracle_for(case)
    o.step(case.steps)
    s = gpu_session(torch, case)
    s.init_state(case.phi0.astype(np.float32))
    s.step(case.steps)
    phi_g = s.macros()["phi"].cpu().numpy()[0]
    phi_o = o.fields()["phi"][0]
    fl = case.solid[0] == 0
    assert np.abs(phi_g[fl] - phi_o[fl]).max() <= 1e-4
    cx = case.info["centre"][0]
    th_g = A.droplet_contact_angle(phi_g, 0, cx)
    th_o = A.droplet_contact_angle(phi_o, 0, cx)
    assert abs(th_g - th_o) <= 0.5, (th_g, th_o)


def test_mass_conservation_gpu(torch):
    pack = W.sphere_pack((40, 36, 30), 0.45, reservoir=0, side_walls=False,
                         seed=3)
    solid = pack["solid"]
    rng = np.random.default_rng(4)
    phi0 = np.where(rng.random(solid.shape) < 0.5, 1.0, -1.0)
    case = W.Case("pack", 19, solid, (True, True, True), phi0,
                  W.base_params(tau_r=1.0, tau_b=0.6, theta_deg=45.0,
                                wetting=1, gamma=0.02, g=(2e-5, 0, 0)))
    s = gpu_session(torch, case)
    s.init_state(phi0.astype(np.float32))
    m0 = s.reduce(0), s.reduce(1)
    s.step(500)
    assert abs(s.reduce(0) / m0[0] - 1) < 2e-5
    assert abs(s.reduce(1) / m0[1] - 1) < 2e-5


def test_step_timed_equals_step(torch):
    """lbm_step_timed runs the same kernels as lbm_step, with events
    between the passes instead of programmatic dependent launches (where a
    pass's blocks start while its predecessor drains and wait for it on the
    device): the states after 5 steps are bit-identical, on a case small
    enough that every pass's blocks are resident at once (so each pass
    really does wait on the device for the one before it), and every
    kernel that runs on the Type-I pack (all seven) reports a positive
    time."""
    from paper_2407_10914_gb300 import lbm
    case = CASES[2][1]  # porous_typeI_schemeI: Zou-He planes and solids
    a = gpu_session(torch, case)
    b = gpu_session(torch, case)
    for s in (a, b):
        s.init_state(case.phi0.astype(np.float32))
    a.step(5)
    ms = b.step_timed(5)
    assert tuple(ms) == lbm.PASSES
    assert all(v > 0 for v in ms.values()), ms
    fa = a.get_populations().cpu().numpy()
    fb = b.get_populations().cpu().numpy()
    assert np.array_equal(fa, fb)


def test_step_graph_equals_single_steps(torch):
    """lbm_step(n) replays pairs of steps from a recorded CUDA graph: the
    state equals that of n single steps bit for bit, for odd and even n,
    across both orientations of the state buffers, and after new
    parameters (the graph is recorded again)."""
    case = CASES[2][1]  # Zou-He planes and solids: all seven kernels
    a = gpu_session(torch, case)
    b = gpu_session(torch, case)
    for s in (a, b):
        s.init_state(case.phi0.astype(np.float32))
    for n in (7, 4, 5, 2, 9):
        a.step(n)
        for _ in range(n):
            b.step(1)
        assert np.array_equal(a.get_populations().cpu().numpy(),
                              b.get_populations().cpu().numpy()), n
    p = dict(case.params, theta_deg=60.0, rho_in=1.03)
    for s in (a, b):
        s.set_params(**p)
    a.step(6)
    for _ in range(6):
        b.step(1)
    assert np.array_equal(a.get_populations().cpu().numpy(),
                          b.get_populations().cpu().numpy())
    for k in ("rho", "phi", "u"):
        assert np.array_equal(a.macros()[k].cpu().numpy(),
                              b.macros()[k].cpu().numpy()), k
