"""Tile shapes of the fluid-node numbering: every shape gives the same
per-node results bit for bit (the shape only moves where a node's values
sit in memory), on ragged boxes whose sizes are no multiple of any tile
extent, with Zou-He planes (whose nodes lead their tiles) and with the
periodic wrap; a batch of domains of different shapes steps like the
domains alone; the autotuner's tile search returns one of its
candidates."""
import numpy as np
import pytest

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


def session(case, tile, storage="fp32"):
    from paper_2407_10914_gb300 import lbm
    s = lbm.Session(case.lattice, case.solid, case.periodic, storage,
                    tile=tile)
    s.set_params(**case.params)
    s.init_state(case.phi0.astype(np.float32))
    return s


def fields(s):
    m = s.macros()
    out = {k: v.cpu().numpy() for k, v in m.items()}
    out["pops"] = s.get_populations().cpu().numpy()
    return out


def cases():
    pack = W.sphere_pack((41, 37, 29), 0.3, rmin=3.0, rmax=6.0, seed=21,
                         reservoir=4)
    return [
        ("porous_typeI", W.porous_3d(pack=pack, drive="typeI", theta_deg=45.0,
                                     wetting=1, rho_in=1.02, rho_out=0.98),
         ((32, 8, 8), (32, 4, 4), (64, 4, 4), (128, 2, 2), (32, 16, 16),
          (32, 1, 1))),
        ("porous_typeII", W.porous_3d(pack=pack, drive="typeII",
                                      theta_deg=40.0, wetting=2, g_x=2e-4,
                                      invading="b"),
         ((32, 8, 8), (64, 8, 8), (32, 4, 8))),
        ("droplet2d", W.droplet_2d(theta_deg=120.0, wetting=1, nx=97, ny=45,
                                   radius=15.0),
         ((64, 32, 1), (32, 32, 1), (128, 16, 1), (32, 1, 1))),
    ]


CASES = cases()


@pytest.mark.parametrize("name,case,tiles", CASES, ids=[c[0] for c in CASES])
def test_every_tile_shape_gives_identical_fields(torch, name, case, tiles):
    ref = session(case, None)
    ref.step(30)
    want = fields(ref)
    for tile in tiles:
        s = session(case, tile)
        assert s.counts == ref.counts
        s.step(30)
        got = fields(s)
        for k in want:
            assert np.array_equal(want[k], got[k]), (tile, k)


def test_batch_of_mixed_tile_shapes(torch):
    from paper_2407_10914_gb300 import lbm
    name, case, tiles = CASES[0]
    alone = [session(case, t) for t in tiles[:3]]
    batched = [session(case, t) for t in tiles[:3]]
    b = lbm.Batch(batched)
    b.set_config(0, 256, 1)
    b.step(12)
    for s in alone:
        s.step(12)
    for a, g in zip(alone, batched):
        assert np.array_equal(a.get_populations().cpu().numpy(),
                              g.get_populations().cpu().numpy())


def test_tile_search_returns_a_candidate(torch):
    from paper_2407_10914_gb300 import autotune
    name, case, tiles = CASES[0]
    r = autotune.tune_tile(lambda t: session(case, t), 19,
                           candidates=tiles[:3], trial_steps=2,
                           use_cache=False)
    assert r["tile"] in tiles[:3]
    assert len(r["trials"]) == 3
    assert all(v > 0 for v in r["trials"].values())
