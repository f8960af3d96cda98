"""The periodic-translation symmetry of tests/test_oracle_translation.py on
the CUDA path, stepped as bench.py steps it (graph-replayed step pairs):
translating the solid image and the phase field along a periodic axis and
stepping gives the translated populations. The compact node order, the
tiles and the dense boxes all move relative to the state, so this checks
the index work of the whole path (wrap and clamp of the dense entry box,
halo copies, Zou-He planes, solid-boundary links) at the periodic faces.
Bound: the float32 parity bar, 1e-6 of the largest population (the step's
arithmetic per node does not depend on the order of nodes)."""
import numpy as np
import pytest

from test_oracle_translation import edge_case, edge_case_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_10914_gb300 import build, lbm
    build.build()
    return lbm


def gpu_run(lbm, solid, phi0, p, steps):
    s = lbm.Session(19, solid, (False, True, True))
    s.set_params(**p)
    s.init_state(phi0.astype(np.float32))
    s.step(steps)
    return s.get_populations().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("axis,shift", [(1, 1), (1, 5), (0, 3)],
                         ids=["y1", "y5", "z3"])
def test_gpu_step_commutes_with_periodic_translation(lbm, axis, shift):
    solid, phi0, p = edge_case()
    ref = gpu_run(lbm, solid, phi0, p, 6)
    got = gpu_run(lbm, np.ascontiguousarray(np.roll(solid, shift, axis=axis)),
                  np.ascontiguousarray(np.roll(phi0, shift, axis=axis)), p, 6)
    want = np.roll(ref, shift, axis=axis + 2)
    assert np.abs(got - want).max() <= 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("shift", [1, 7, 20])
def test_gpu_d2q9_step_commutes_with_periodic_translation(lbm, shift):
    solid, phi0, p = edge_case_2d()

    def run(sol, ph):
        s = lbm.Session(9, sol, (True, False, True))
        s.set_params(**p)
        s.init_state(ph.astype(np.float32))
        s.step(8)
        return s.get_populations().cpu().numpy().astype(np.float64)

    ref = run(solid, phi0)
    got = run(np.ascontiguousarray(np.roll(solid, shift, axis=2)),
              np.ascontiguousarray(np.roll(phi0, shift, axis=2)))
    want = np.roll(ref, shift, axis=4)
    assert np.abs(got - want).max() <= 1e-6 * np.abs(ref).max()
