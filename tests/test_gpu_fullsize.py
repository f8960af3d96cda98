"""Parity at the full size of the throughput workload: the 256^3 synthetic
rock (4.6 M fluid nodes, Scheme-I drainage; Type-I Zou-He or Type-II body
force; FP32 storage, and FP16 at its stated 1e-4) stepped by the GPU in the
launch configuration bench.py times (graph replay of step pairs, then the
last step) and by the FP64 oracle, three steps from the same initial
state; every population of every fluid node within the tolerance of the
largest population of its colour. The oracle needs about 12 GB of host
memory and some seconds of the host's cores per case."""
import numpy as np
import pytest

from oracle import oracle as O
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


TOL = {"fp32": 1e-6, "fp16": 1e-4}


@pytest.mark.parametrize("drive,storage", [("typeI", "fp32"),
                                           ("typeII", "fp32"),
                                           ("typeI", "fp16")])
def test_rock_256_three_steps(lbm, drive, storage):
    case = W.porous_3d(n=(256, 256, 256), drive=drive)
    s = lbm.Session(19, case.solid, case.periodic, storage)
    s.set_params(**case.params)
    s.init_state(case.phi0.astype(np.float32))
    s.step(3)
    got = s.get_populations().cpu().numpy()
    del s
    o = O.Oracle(19, case.solid, case.periodic)
    o.set_params(**case.params)
    o.init_state(case.phi0)
    o.step(3)
    ref = o.pops
    fl = case.solid == 0
    for c in range(2):
        scale = np.abs(ref[c]).max()
        worst = 0.0
        for i in range(19):
            d = np.abs(got[c, i][fl].astype(np.float64) - ref[c, i][fl]).max()
            worst = max(worst, float(d))
        assert worst <= TOL[storage] * scale, (c, worst / scale)
