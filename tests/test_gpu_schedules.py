"""The tile schedule of the step (the default: four tile passes that stage a
halo in shared memory and evaluate Eqs. 34-35 inside the stencil passes)
against the node schedule (seven passes over the compact node lists).

Both sum every term in the same order, so with float32 storage they must
agree bit for bit: populations after several steps (graph-replayed pairs and
plain launches), the phase field with Eq. (34) at the solid-boundary nodes,
rho and u. With 16-bit storage the node schedule also rounds the streamed
populations to the storage type before the collision; there the two agree
to the storage's own rounding (the tolerance of the 16-bit parity tests)."""
import numpy as np
import pytest

from paper_2407_10914_gb300 import workloads as W
from test_gpu_parity import CASES, small_pack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_10914_gb300 import build
    build.build()
    return torch


def pair(case, storage="fp32", params=None, develop=40):
    """Two sessions of the case, one per schedule, holding the same
    developed state."""
    from paper_2407_10914_gb300 import lbm
    p = dict(case.params, **(params or {}))
    a = lbm.Session(case.lattice, case.solid, case.periodic, storage)
    a.set_params(**p)
    a.init_state(case.phi0.astype(np.float32))
    a.step(develop)
    f = a.get_populations()
    b = lbm.Session(case.lattice, case.solid, case.periodic, storage)
    b.set_params(**p)
    b.set_schedule("nodes")
    assert a.schedule == "tiles" and b.schedule == "nodes"
    a.set_populations(f)
    b.set_populations(f)
    return a, b


def fields(s):
    m = s.macros()
    return (s.get_populations().cpu().numpy(), m["phi"].cpu().numpy(),
            m["rho"].cpu().numpy(), m["u"].cpu().numpy())


def where(x, y):
    """Index and values of the largest difference (for the failure message)."""
    k = np.unravel_index(np.argmax(np.abs(x - y)), x.shape)
    return k, float(x[k]), float(y[k])


@pytest.mark.parametrize("name,case,dev", CASES, ids=[c[0] for c in CASES])
def test_schedules_bit_identical_fp32(torch, name, case, dev):
    a, b = pair(case)
    for n in (1, 5):  # a plain step, then graph-replayed pairs and the last
        a.step(n)
        b.step(n)
        for x, y, what in zip(fields(a), fields(b), ("pops", "phi", "rho", "u")):
            assert np.array_equal(x, y), (name, n, what, where(x, y))


MRT_CASES = [c for c in CASES if c[1].lattice == 19][:4]


@pytest.mark.parametrize("name,case,dev", MRT_CASES,
                         ids=[c[0] for c in MRT_CASES])
def test_schedules_bit_identical_mrt(torch, name, case, dev):
    a, b = pair(case, params=dict(collision=1))
    a.step(4)
    b.step(4)
    for x, y, what in zip(fields(a), fields(b), ("pops", "phi", "rho", "u")):
        assert np.array_equal(x, y), (name, what, where(x, y))


@pytest.mark.parametrize("storage,tol", [("fp16", 1e-4), ("bf16", 1e-3)])
def test_schedules_agree_16bit(torch, storage, tol):
    pack = small_pack()
    case = W.porous_3d(pack=pack, drive="typeI", theta_deg=45.0, wetting=1,
                       rho_in=1.02, rho_out=0.98)
    a, b = pair(case, storage)
    a.step(3)
    b.step(3)
    fa, fb = a.get_populations().cpu().numpy(), b.get_populations().cpu().numpy()
    for c in range(2):
        err = np.abs(fa[c] - fb[c]).max() / np.abs(fb[c]).max()
        assert err <= tol, (storage, c, err)


def test_schedule_switch_and_timed_slots(torch):
    """lbm_set_schedule refuses unknown values; lbm_step_timed names the
    tile passes (the slots of Eqs. 34 and 35 stay empty) and runs the same
    kernels as lbm_step."""
    from paper_2407_10914_gb300 import lbm
    case = CASES[2][1]  # porous_typeI_schemeI: Zou-He planes present
    a, b = pair(case)
    L = lbm.load_library()
    assert L.lbm_set_schedule(a.h, 7) == -1
    assert a.schedule == "tiles"
    ms = a.step_timed(3)
    assert set(ms) == {"pull", "planes", "gradient", "curvature", "collide"}
    assert all(v > 0 for v in ms.values())
    b.set_schedule("tiles")
    b.step(3)
    assert np.array_equal(a.get_populations().cpu().numpy(),
                          b.get_populations().cpu().numpy())
