"""The batched sweep (lbm_batch_*): many cases stepped together give what
stepping each case on its own gives, bit for bit, across odd step counts,
graph replays and cases stepped outside the batch, with one launch per pass
of all cases (mode 0) and with one persistent launch (mode 1). Mode 1
inlines every pass into one kernel, compiled for other register limits;
it is bit-identical because every rounding of the step is pinned (the
shared helpers of stencil.cuh use explicitly rounded operations, so the
compiler cannot contract them differently per kernel). The bounded wait
gives up and reports; the autotuner keeps results identical."""
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


def small_cases():
    """Uneven D3Q19 cases: sessile drops of the sweep (shrunk), a Zou-He
    tube and a forced pack with solids inside."""
    cases = W.batched_droplets(count=4, smin=48, smax=128, steps=10,
                               scale=0.25)
    cases.append(W.tube_3d(nx=40, red_len=10, rho_in=1.02, rho_out=0.98))
    pack = W.sphere_pack((33, 29, 27), 0.35, rmin=3.0, rmax=6.0, seed=5,
                         reservoir=3)
    cases.append(W.porous_3d(pack=pack, drive="typeII", theta_deg=40.0,
                             wetting=2, g_x=2e-4, invading="b"))
    return cases


def sessions(torch, cases, storage="fp32"):
    from paper_2407_10914_gb300 import lbm
    out = []
    for c in cases:
        s = lbm.Session(c.lattice, c.solid, c.periodic, storage)
        s.set_params(**c.params)
        s.init_state(c.phi0.astype(np.float32))
        out.append(s)
    return out


def pops(s):
    return s.get_populations().cpu().numpy()




def agree(r, g):
    """Populations of two sessions are identical."""
    return np.array_equal(pops(r), pops(g))


def same_as_alone(torch, cases, storage, config, calls):
    from paper_2407_10914_gb300 import lbm
    ref = sessions(torch, cases, storage)
    got = sessions(torch, cases, storage)
    b = lbm.Batch(got)
    b.set_config(*config)
    for n in calls:
        b.step(n)
        for s in ref:
            s.step(n)
    assert b.status() == 0
    for r, g, c in zip(ref, got, cases):
        assert agree(r, g), (c.name, config)
        mr, mg = r.macros(), g.macros()
        for k in ("rho", "phi", "u"):
            assert np.array_equal(mr[k].cpu().numpy(), mg[k].cpu().numpy()), k


@pytest.mark.parametrize("config", [(0, 256, 1), (0, 128, 1), (1, 256, 1),
                                    (1, 256, 4), (1, 128, 16)],
                         ids=["levels256", "levels128", "persist256c1",
                              "persist256c4", "persist128c16"])
def test_batch_equals_cases_alone(torch, config):
    # 3 then 4 steps: an odd call, then a second graph; 3 again: a replay
    same_as_alone(torch, small_cases(), "fp32", config, (3, 4, 3))


def test_batch_fp16_storage(torch):
    same_as_alone(torch, small_cases()[:3], "fp16", (1, 256, 4), (2, 3))


def test_case_stepped_outside_the_batch(torch):
    from paper_2407_10914_gb300 import lbm
    cases = small_cases()[:3]
    ref = sessions(torch, cases)
    got = sessions(torch, cases)
    b = lbm.Batch(got)
    b.set_config(1, 256, 4)
    b.step(3)
    got[1].step(1)  # the batch must re-read this case
    b.step(2)
    for s in ref:
        s.step(3)
    ref[1].step(1)
    for s in ref:
        s.step(2)
    for r, g in zip(ref, got):
        assert agree(r, g)


def test_batch_one_step_matches_oracle(torch):
    """Directly against the FP64 oracle: one batched step of a drop."""
    from oracle import oracle as O
    from paper_2407_10914_gb300 import lbm
    case = small_cases()[0]
    s = sessions(torch, [case])[0]
    b = lbm.Batch([s])
    b.set_config(1, 256, 1)
    b.step(1)
    o = O.Oracle(case.lattice, case.solid, case.periodic)
    o.set_params(**case.params)
    o.init_state(case.phi0)
    o.step(1)
    ref = o.pops
    got = pops(s).astype(np.float64)
    fl = case.solid == 0
    for c in range(2):
        err = np.abs(got[c][:, fl] - ref[c][:, fl]).max() / np.abs(ref[c]).max()
        assert err <= 1e-6, (c, err)


def test_bounded_wait_gives_up(torch):
    from paper_2407_10914_gb300 import lbm
    cases = small_cases()[:2]
    ref = sessions(torch, cases)
    got = sessions(torch, cases)
    b = lbm.Batch(got)
    waited = b.check_wait(50.0)
    assert 45.0 <= waited <= 2000.0, waited
    assert b.status() == 0  # the check cleared its own flag
    b.set_config(1, 256, 4)
    b.step(2)  # the context and the batch still work
    for s in ref:
        s.step(2)
    assert b.status() == 0
    for r, g in zip(ref, got):
        assert agree(r, g)


def test_autotune_keeps_results(torch, tmp_path):
    from paper_2407_10914_gb300 import autotune, lbm
    cases = small_cases()[:3]
    ref = sessions(torch, cases)
    got = sessions(torch, cases)
    b = lbm.Batch(got)
    res = autotune.tune(b, trial_steps=2, cache_path=str(tmp_path / "t.json"))
    assert res["config"] in autotune.CANDIDATES and not res["cached"]
    used = res["steps_used"]
    assert used == len(autotune.CANDIDATES) * 3
    b.step(1)
    for s in ref:
        s.step(used + 1)
    for r, g in zip(ref, got):
        assert agree(r, g)
    again = autotune.tune(lbm.Batch(sessions(torch, cases)), trial_steps=2,
                          cache_path=str(tmp_path / "t.json"))
    assert again["cached"] and again["config"] == res["config"]
