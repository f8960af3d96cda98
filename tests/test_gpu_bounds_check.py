"""The bounds-checked build (liblbmgb_check.so, compiled with
LBM_BOUNDS_CHECK): every gathered index of the step (pull sources,
stencil neighbours, Zou-He plane nodes, solid-boundary links) is checked
against its array, a violation recorded in the domain's error word
(lbm_debug_flags) and the access redirected in bounds. This stands in for
a memory checker, which this GPU pool does not offer. Small cases of every
kind of node and schedule run under it with a clean error word, and give
the populations of the normal build."""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from paper_2407_10914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cases():
    pack = W.sphere_pack((20, 18, 16), 0.35, rmin=2.5, rmax=4.0, seed=9,
                         reservoir=3)
    return [
        W.porous_3d(pack=pack, drive="typeI", theta_deg=45.0, wetting=1,
                    rho_in=1.02, rho_out=0.98),
        W.porous_3d(pack=pack, drive="typeII", theta_deg=40.0, wetting=2,
                    g_x=2e-4, invading="b"),
        W.droplet_2d(nx=16, ny=8, radius=3.0),
        W.droplet_3d(side=12, radius=4.0, theta_deg=120.0, wetting=1),
    ]


RUN = r'''
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
from paper_2407_10914_gb300 import build, lbm
from test_gpu_bounds_check import cases
lib = sys.argv[2]
if lib:
    lbm.load_library(lib)
out = {}
sess = []
for n, c in enumerate(cases()):
    s = lbm.Session(c.lattice, c.solid, c.periodic)
    s.set_params(**dict(c.params, collision=1 if c.lattice == 19 and n == 0
                        else 0))
    s.init_state(c.phi0.astype(np.float32))
    s.step(15)
    out[f"pops{n}"] = s.get_populations().cpu().numpy()
    out[f"flags{n}"] = np.array(lbm.lbm_debug_flags(s.h, s.stream()))
    sess.append(s)
# the persistent batch schedule over the two 3-D drops and a pack
b = lbm.Batch([sess[1], sess[3]])
b.set_config(1, 128, 4)
b.step(3)
out["flags_batch"] = np.array([lbm.lbm_debug_flags(s.h, s.stream())
                               for s in (sess[1], sess[3])])
np.savez(sys.argv[3], **out)
'''


def run(lib, path):
    r = subprocess.run([sys.executable, "-c", RUN, ROOT, lib, path],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(path)


@pytest.fixture(scope="module")
def libs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2407_10914_gb300 import build
    return build.build(), build.build(check=True)


def test_checked_build_is_clean_and_equal(libs):
    normal, checked = libs
    with tempfile.TemporaryDirectory() as d:
        ref = run(normal, os.path.join(d, "normal.npz"))
        got = run(checked, os.path.join(d, "checked.npz"))
    n = len(cases())
    for k in range(n):
        assert int(got[f"flags{k}"]) == 0, k
        assert int(ref[f"flags{k}"]) == 0, k
        a, b = ref[f"pops{k}"], got[f"pops{k}"]
        for c in range(2):
            assert np.abs(a[c].astype(np.float64) - b[c]).max() <= \
                1e-6 * np.abs(a[c]).max(), (k, c)
    assert not got["flags_batch"].any()
