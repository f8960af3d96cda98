"""Host-side checks of the C-ABI library that need no GPU: it loads, it
exports every function include/lbmgb.h declares, and argument errors are
reported before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_10914_gb300 import build as B, lbm
    B.build()
    return lbm.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbmgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_header_declarations_are_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2407_10914_gb300 import lbm
    assert sorted(lbm.EXPORTS) == declared_functions()
    for n in lbm.EXPORTS:
        if n != "lbm_last_error":
            assert callable(getattr(lbm, n))


def test_workspace_bytes_host_only(lib):
    from paper_2407_10914_gb300 import lbm
    solid = np.zeros((4, 5, 6), np.uint8)
    n19 = lbm.lbm_workspace_bytes(19, 6, 5, 4, solid, 0)
    n19h = lbm.lbm_workspace_bytes(19, 6, 5, 4, solid, 1)
    assert n19 > 2 * 2 * 19 * 120 * 4 and n19h < n19
    assert lbm.lbm_workspace_bytes(7, 6, 5, 4, solid, 0) == 0
    assert lbm.lbm_workspace_bytes(9, 6, 5, 2, solid, 0) == 0  # D2Q9 needs nz=1
    assert lbm.lbm_workspace_bytes(19, 6, 5, 4, solid, 5) == 0


def test_tile_shapes_host_only(lib):
    """Tile shapes: powers of two, x extent 32..1024, at most 16384 nodes,
    z extent 1 on D2Q9; the default shape is what a null tile gives; the
    per-tile arrays grow with the number of tiles."""
    from paper_2407_10914_gb300 import autotune, lbm
    solid = np.zeros((20, 30, 70), np.uint8)
    args = (19, 70, 30, 20, solid, 0)
    base = lbm.lbm_workspace_bytes(*args)
    assert lbm.lbm_workspace_bytes_tiled(*args, None) == base
    assert lbm.lbm_workspace_bytes_tiled(*args, (32, 8, 8)) == base
    assert lbm.lbm_workspace_bytes_tiled(*args, (32, 1, 1)) > base
    for bad in ((16, 8, 8), (48, 8, 8), (32, 32, 32), (2048, 1, 1),
                (32, 0, 8), (32, 8, -8), (32, 3, 8)):
        assert lbm.lbm_workspace_bytes_tiled(*args, bad) == 0, bad
    s2 = np.zeros((1, 30, 70), np.uint8)
    assert lbm.lbm_workspace_bytes_tiled(9, 70, 30, 1, s2, 0, (64, 32, 1)) \
        == lbm.lbm_workspace_bytes(9, 70, 30, 1, s2, 0)
    assert lbm.lbm_workspace_bytes_tiled(9, 70, 30, 1, s2, 0, (64, 16, 2)) == 0
    h = C.c_void_p()
    sp = solid.ctypes.data_as(C.c_void_p)
    bad = (C.c_int * 3)(16, 8, 8)
    assert lib.lbm_init_geometry_tiled(C.byref(h), 19, 70, 30, 20, sp, 7, 0,
                                       bad, C.c_void_p(256), 1 << 30,
                                       None) == -1
    assert not h.value
    for q, cands in autotune.TILE_CANDIDATES.items():
        assert cands[0] == ((32, 8, 8) if q == 19 else (64, 32, 1))
        for t in cands:
            sh = (20, 30, 70) if q == 19 else (1, 30, 70)
            assert lbm.lbm_workspace_bytes_tiled(
                q, 70, 30, sh[0], np.zeros(sh, np.uint8), 0, t) > 0, t


def test_init_geometry_rejects_bad_arguments(lib):
    h = C.c_void_p()
    solid = np.zeros(8, np.uint8)
    sp = solid.ctypes.data_as(C.c_void_p)
    fake_ws = C.c_void_p(256)  # never touched: the checks come first
    assert lib.lbm_init_geometry(C.byref(h), 7, 2, 2, 2, sp, 7, 0, fake_ws,
                                 1 << 20, None) == -1
    assert lib.lbm_init_geometry(C.byref(h), 19, 2, 2, 2, None, 7, 0,
                                 fake_ws, 1 << 20, None) == -1
    allsolid = np.ones(8, np.uint8)
    assert lib.lbm_init_geometry(C.byref(h), 19, 2, 2, 2,
                                 allsolid.ctypes.data_as(C.c_void_p), 7, 0,
                                 fake_ws, 1 << 20, None) == -1
    assert lib.lbm_init_geometry(C.byref(h), 19, 2, 2, 2, sp, 7, 0,
                                 C.c_void_p(257), 1 << 20, None) == -1
    assert lib.lbm_init_geometry(C.byref(h), 19, 2, 2, 2, sp, 7, 0, fake_ws,
                                 16, None) == -6
    assert not h.value


def test_batch_entry_points_host_only(lib):
    """Batch sizes and argument checks that need no GPU."""
    from paper_2407_10914_gb300 import lbm
    n1 = lbm.lbm_batch_workspace_bytes(1)
    n96 = lbm.lbm_batch_workspace_bytes(96)
    assert lbm.lbm_batch_workspace_bytes(0) == 0
    assert 0 < n1 < n96 < 96 * 4096
    out = C.c_void_p()
    arr = (C.c_void_p * 1)(None)
    # a null handle, no cases, a null workspace: rejected before any CUDA call
    assert lib.lbm_batch_create(C.byref(out), arr, 1, C.c_void_p(256), n1,
                                None) == -1
    assert lib.lbm_batch_create(C.byref(out), arr, 0, C.c_void_p(256), n1,
                                None) == -1
    assert lib.lbm_batch_create(None, arr, 1, C.c_void_p(256), n1, None) == -1
    assert lib.lbm_batch_step(None, 1, None) == -1
    assert lib.lbm_batch_set_config(None, 0, 256, 1, None) == -1
    assert lib.lbm_batch_last_error(None) == b"null batch"


def test_pass_list_matches_header_and_byte_model():
    """lbm_step_timed reports LBM_N_PASSES kernels; the binding names them
    and bench.py's byte model has an entry for each."""
    import importlib.util
    from paper_2407_10914_gb300 import lbm
    src = open(os.path.join(ROOT, "include", "lbmgb.h")).read()
    n = int(re.search(r"#define LBM_N_PASSES (\d+)", src).group(1))
    assert len(lbm.PASSES) == n
    spec = importlib.util.spec_from_file_location(
        "bench_module", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for q in (9, 19):
        pb = bench.pass_bytes(q, 4)
        assert set(pb) == set(lbm.PASSES) == set(bench.PASS_KERNEL)
        assert all(v > 0 for v in pb.values())


def test_noalloc_refuses_host_tensor_before_any_launch():
    """The binding of lbm_colour_mass_noalloc refuses a host tensor (a
    host pointer handed to the kernel would be an illegal access) before it
    reaches the library, GPU or not."""
    torch = pytest.importorskip("torch")
    from paper_2407_10914_gb300 import lbm
    pops = torch.zeros((2, 19, 4, 4, 4), dtype=torch.float32)
    with pytest.raises(lbm.LbmError, match="CUDA tensor"):
        lbm.lbm_colour_mass_noalloc(19, pops, None)
    with pytest.raises(lbm.LbmError, match="lattice"):
        lbm.lbm_colour_mass_noalloc(7, pops, None)


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "bench_traffic", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


def test_recorded_traffic_needs_kernel_workload_and_source(tmp_path,
                                                           monkeypatch):
    """bench.py reports a kernel's DRAM bytes only from a line taken on the
    running kernel source: the kernel, the workload and the source hash must
    all match, and comment lines are skipped."""
    bench = _bench_module()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(
        "# k_stream w1 1 abc\n"
        "k_stream  w1 100 abc\n"
        "k_stream  w1 200 def\n"
        "k_collide w1 300 abc\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.recorded_traffic("k_stream", "w1") == 100
    assert bench.recorded_traffic("k_collide", "w1") == 300
    assert bench.recorded_traffic("k_stream", "w2") is None
    assert bench.recorded_traffic("k_gradient", "w1") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "def")
    assert bench.recorded_traffic("k_stream", "w1") == 200
    assert bench.recorded_traffic("k_collide", "w1") is None


def test_committed_traffic_covers_every_pass_of_the_step():
    """The committed DRAM summary has a line for every kernel of the FP32
    step on the 256^3 rock at the current kernel source (a kernel change
    that was not captured again would leave the roofline's traffic null)."""
    bench = _bench_module()
    for kern in bench.PASS_KERNEL.values():
        t = bench.recorded_traffic(kern, "porous256_drainage_typeI_fp32")
        assert t is not None and t > 0, kern
