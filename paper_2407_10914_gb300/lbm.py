"""Python binding of the C-ABI in ``include/lbmgb.h`` (argument marshalling
only; every step of the method runs in the CUDA library ``liblbmgb.so``).

PyTorch provides the device memory (the workspace and every buffer passed to
the library) and the stream (``torch.cuda.current_stream()``). The module
fails loudly if the library is missing or no GPU is present: there is no
CPU fallback.

The functions ``lbm_*`` mirror the C names one to one; :class:`Session` is
a convenience owner of one domain and its workspace.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbmgb.so")

LBM_OK = 0
STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA",
          -3: "LBM_ERR_STATE", -4: "LBM_ERR_NONFINITE", -5: "LBM_ERR_TIMEOUT",
          -6: "LBM_ERR_NOMEM"}
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
(LBM_MASS_R, LBM_MASS_B, LBM_SW_COUNT, LBM_SW_SMOOTH, LBM_DP, LBM_CA_R,
 LBM_CA_B) = range(7)
EXPORTS = ("lbm_workspace_bytes", "lbm_init_geometry",
           "lbm_workspace_bytes_tiled", "lbm_init_geometry_tiled",
           "lbm_set_params",
           "lbm_init_state", "lbm_step", "lbm_step_timed", "lbm_macros",
           "lbm_reduce", "lbm_reduce_async", "lbm_reduce_value",
           "lbm_get_populations", "lbm_set_populations", "lbm_swap_inlet",
           "lbm_debug_flags",
           "lbm_get_geometry",
           "lbm_counts", "lbm_colour_mass_noalloc", "lbm_last_error",
           "lbm_destroy",
           "lbm_batch_workspace_bytes", "lbm_batch_create",
           "lbm_batch_set_config", "lbm_batch_step", "lbm_batch_status",
           "lbm_batch_check_wait", "lbm_batch_last_error",
           "lbm_batch_destroy",
           "lbm_state_bytes", "lbm_save_state", "lbm_load_state",
           "lbm_adj_workspace_bytes", "lbm_adj_create", "lbm_adj_seed_sw",
           "lbm_adj_step", "lbm_adj_gradients", "lbm_adj_get_lambda",
           "lbm_adj_set_freeze", "lbm_adj_set_cmin", "lbm_adj_last_error",
           "lbm_adj_destroy")


class LbmError(RuntimeError):
    pass


class lbm_params(C.Structure):
    """Mirror of the C struct ``lbm_params``."""
    _fields_ = [("tau_r", C.c_double), ("tau_b", C.c_double),
                ("gamma", C.c_double), ("beta", C.c_double),
                ("rho0", C.c_double), ("theta_deg", C.c_double),
                ("wetting", C.c_int), ("zou_he", C.c_int),
                ("flow_axis", C.c_int),
                ("rho_in", C.c_double), ("rho_out", C.c_double),
                ("zeta_r", C.c_double), ("g", C.c_double * 3),
                ("collision", C.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load ``liblbmgb.so`` (no GPU needed to load it) and declare the
    prototypes of every exported entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LbmError(f"CUDA library not built: {path} (run "
                       "python -m paper_2407_10914_gb300.build)")
    L = C.CDLL(path)
    vp, sz, i64p = C.c_void_p, C.c_size_t, C.POINTER(C.c_int64)
    L.lbm_workspace_bytes.restype = sz
    L.lbm_workspace_bytes.argtypes = [C.c_int] * 4 + [vp, C.c_int]
    L.lbm_init_geometry.restype = C.c_int
    L.lbm_init_geometry.argtypes = [C.POINTER(vp)] + [C.c_int] * 4 + [
        vp, C.c_uint, C.c_int, vp, sz, vp]
    L.lbm_workspace_bytes_tiled.restype = sz
    L.lbm_workspace_bytes_tiled.argtypes = [C.c_int] * 4 + [
        vp, C.c_int, C.POINTER(C.c_int)]
    L.lbm_init_geometry_tiled.restype = C.c_int
    L.lbm_init_geometry_tiled.argtypes = [C.POINTER(vp)] + [C.c_int] * 4 + [
        vp, C.c_uint, C.c_int, C.POINTER(C.c_int), vp, sz, vp]
    L.lbm_set_params.restype = C.c_int
    L.lbm_set_params.argtypes = [vp, C.POINTER(lbm_params)]
    L.lbm_init_state.restype = C.c_int
    L.lbm_init_state.argtypes = [vp, vp, vp]
    L.lbm_step.restype = C.c_int
    L.lbm_step.argtypes = [vp, C.c_int, vp]
    L.lbm_step_timed.restype = C.c_int
    L.lbm_step_timed.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_double)]
    L.lbm_macros.restype = C.c_int
    L.lbm_macros.argtypes = [vp, vp, vp, vp, vp]
    L.lbm_reduce.restype = C.c_int
    L.lbm_reduce.argtypes = [vp, C.c_int, C.POINTER(C.c_double), vp]
    L.lbm_reduce_async.restype = C.c_int
    L.lbm_reduce_async.argtypes = [vp, C.c_int, vp, vp]
    L.lbm_reduce_value.restype = C.c_int
    L.lbm_reduce_value.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_double)]
    L.lbm_get_populations.restype = C.c_int
    L.lbm_get_populations.argtypes = [vp, vp, vp]
    L.lbm_set_populations.restype = C.c_int
    L.lbm_set_populations.argtypes = [vp, vp, vp]
    L.lbm_swap_inlet.restype = C.c_int
    L.lbm_swap_inlet.argtypes = [vp, C.c_int, vp]
    L.lbm_debug_flags.restype = C.c_int
    L.lbm_debug_flags.argtypes = [vp, C.POINTER(C.c_uint), vp]
    L.lbm_get_geometry.restype = C.c_int
    L.lbm_get_geometry.argtypes = [vp, vp, vp, vp]
    L.lbm_counts.restype = C.c_int
    L.lbm_counts.argtypes = [vp, i64p, i64p, i64p, i64p]
    L.lbm_colour_mass_noalloc.restype = C.c_int
    L.lbm_colour_mass_noalloc.argtypes = [C.c_int, C.c_int64, vp,
                                          C.POINTER(C.c_double), vp]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_last_error.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_destroy.argtypes = [vp]
    L.lbm_batch_workspace_bytes.restype = sz
    L.lbm_batch_workspace_bytes.argtypes = [C.c_int]
    L.lbm_batch_create.restype = C.c_int
    L.lbm_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int, vp,
                                   sz, vp]
    L.lbm_batch_set_config.restype = C.c_int
    L.lbm_batch_set_config.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp]
    L.lbm_batch_step.restype = C.c_int
    L.lbm_batch_step.argtypes = [vp, C.c_int, vp]
    L.lbm_batch_status.restype = C.c_int
    L.lbm_batch_status.argtypes = [vp, vp]
    L.lbm_batch_check_wait.restype = C.c_int
    L.lbm_batch_check_wait.argtypes = [vp, C.c_double, C.POINTER(C.c_double),
                                       vp]
    L.lbm_batch_last_error.restype = C.c_char_p
    L.lbm_batch_last_error.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_state_bytes.restype = sz
    L.lbm_state_bytes.argtypes = [vp]
    for f in (L.lbm_save_state, L.lbm_load_state):
        f.restype = C.c_int
        f.argtypes = [vp, vp, vp]
    L.lbm_adj_workspace_bytes.restype = sz
    L.lbm_adj_workspace_bytes.argtypes = [vp]
    L.lbm_adj_create.restype = C.c_int
    L.lbm_adj_create.argtypes = [C.POINTER(vp), vp, vp, sz]
    for f in (L.lbm_adj_seed_sw, L.lbm_adj_step):
        f.restype = C.c_int
        f.argtypes = [vp, vp]
    L.lbm_adj_gradients.restype = C.c_int
    L.lbm_adj_gradients.argtypes = [vp, C.POINTER(C.c_double), vp]
    L.lbm_adj_get_lambda.restype = C.c_int
    L.lbm_adj_get_lambda.argtypes = [vp, vp, vp, vp]
    L.lbm_adj_set_freeze.restype = C.c_int
    L.lbm_adj_set_freeze.argtypes = [vp, C.c_double]
    L.lbm_adj_set_cmin.restype = C.c_int
    L.lbm_adj_set_cmin.argtypes = [vp, C.c_double]
    L.lbm_adj_last_error.restype = C.c_char_p
    L.lbm_adj_last_error.argtypes = [vp]
    L.lbm_adj_destroy.restype = None
    L.lbm_adj_destroy.argtypes = [vp]
    _lib = L
    return L


def _check(st: int, h=None, what: str = ""):
    if st != LBM_OK:
        msg = ""
        if h:
            msg = load_library().lbm_last_error(h).decode()
        raise LbmError(f"{what}: {STATUS.get(st, st)} {msg}")


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise LbmError("no CUDA device: the LBM step runs only on the GPU")
    return torch


def _stream(torch):
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def make_params(**kw) -> lbm_params:
    d = dict(tau_r=1.0, tau_b=1.0, gamma=0.01, beta=0.95, rho0=1.0,
             theta_deg=90.0, wetting=0, zou_he=0, flow_axis=0, rho_in=1.0,
             rho_out=1.0, zeta_r=1.0, g=(0.0, 0.0, 0.0), collision=0)
    for k in kw:
        if k not in d:
            raise KeyError(k)
    d.update(kw)
    return lbm_params(d["tau_r"], d["tau_b"], d["gamma"], d["beta"],
                      d["rho0"], d["theta_deg"], int(d["wetting"]),
                      int(d["zou_he"]), int(d["flow_axis"]), d["rho_in"],
                      d["rho_out"], d["zeta_r"], (C.c_double * 3)(*d["g"]),
                      int(d["collision"]))


# ------------------------------------------------ one-to-one C wrappers
def lbm_workspace_bytes(lattice, nx, ny, nz, solid: Optional[np.ndarray],
                        storage=0) -> int:
    L = load_library()
    sp = None if solid is None else solid.ctypes.data_as(C.c_void_p)
    return int(L.lbm_workspace_bytes(lattice, nx, ny, nz, sp, storage))


def _tile_arg(tile):
    return None if tile is None else (C.c_int * 3)(*[int(t) for t in tile])


def lbm_workspace_bytes_tiled(lattice, nx, ny, nz,
                              solid: Optional[np.ndarray], storage=0,
                              tile=None) -> int:
    """tile: None (the default shape) or (tx, ty, tz)."""
    L = load_library()
    sp = None if solid is None else solid.ctypes.data_as(C.c_void_p)
    return int(L.lbm_workspace_bytes_tiled(lattice, nx, ny, nz, sp, storage,
                                           _tile_arg(tile)))


def lbm_init_geometry(lattice, nx, ny, nz, solid: np.ndarray, periodic_mask,
                      storage, workspace, stream) -> C.c_void_p:
    L = load_library()
    h = C.c_void_p()
    solid = np.ascontiguousarray(solid, np.uint8)
    st = L.lbm_init_geometry(C.byref(h), lattice, nx, ny, nz,
                             solid.ctypes.data_as(C.c_void_p), periodic_mask,
                             storage, _dptr(workspace), workspace.numel(),
                             stream)
    _check(st, None, "lbm_init_geometry")
    return h


def lbm_init_geometry_tiled(lattice, nx, ny, nz, solid: np.ndarray,
                            periodic_mask, storage, tile, workspace,
                            stream) -> C.c_void_p:
    L = load_library()
    h = C.c_void_p()
    solid = np.ascontiguousarray(solid, np.uint8)
    st = L.lbm_init_geometry_tiled(C.byref(h), lattice, nx, ny, nz,
                                   solid.ctypes.data_as(C.c_void_p),
                                   periodic_mask, storage, _tile_arg(tile),
                                   _dptr(workspace), workspace.numel(),
                                   stream)
    _check(st, None, "lbm_init_geometry_tiled")
    return h


def lbm_set_params(h, p: lbm_params):
    _check(load_library().lbm_set_params(h, C.byref(p)), h, "lbm_set_params")


def lbm_init_state(h, phi0, stream):
    _check(load_library().lbm_init_state(h, _dptr(phi0), stream), h,
           "lbm_init_state")


def lbm_step(h, nsteps, stream):
    _check(load_library().lbm_step(h, int(nsteps), stream), h, "lbm_step")


PASSES = ("stream", "zh_fix", "phi_solid", "gradient", "nc_solid",
          "curvature", "collide")


def lbm_step_timed(h, nsteps, stream) -> dict:
    ms = (C.c_double * len(PASSES))()
    _check(load_library().lbm_step_timed(h, int(nsteps), stream, ms), h,
           "lbm_step_timed")
    return dict(zip(PASSES, ms[:]))


def lbm_macros(h, rho, phi, u, stream):
    p = [None if t is None else _dptr(t) for t in (rho, phi, u)]
    _check(load_library().lbm_macros(h, *p, stream), h, "lbm_macros")


def lbm_reduce(h, kind, stream) -> float:
    out = C.c_double()
    _check(load_library().lbm_reduce(h, int(kind), C.byref(out), stream), h,
           "lbm_reduce")
    return out.value


def lbm_reduce_async(h, kind, raw4_ptr, stream):
    """Enqueue a reduction and the copy of its four raw FP64 sums to the host
    address raw4_ptr (an int; page-locked memory for the copy to overlap)."""
    _check(load_library().lbm_reduce_async(h, int(kind), C.c_void_p(raw4_ptr),
                                           stream), h, "lbm_reduce_async")


def lbm_reduce_value(h, kind, raw4_ptr) -> float:
    """The quantity of `kind` from four raw sums at host address raw4_ptr."""
    out = C.c_double()
    _check(load_library().lbm_reduce_value(h, int(kind), C.c_void_p(raw4_ptr),
                                           C.byref(out)), h, "lbm_reduce_value")
    return out.value


def lbm_get_populations(h, dst, stream):
    _check(load_library().lbm_get_populations(h, _dptr(dst), stream), h,
           "lbm_get_populations")


def lbm_set_populations(h, src, stream):
    _check(load_library().lbm_set_populations(h, _dptr(src), stream), h,
           "lbm_set_populations")


def lbm_debug_flags(h, stream) -> int:
    out = C.c_uint(0)
    _check(load_library().lbm_debug_flags(h, C.byref(out), stream), h,
           "lbm_debug_flags")
    return int(out.value)


def lbm_swap_inlet(h, colour: int, stream):
    _check(load_library().lbm_swap_inlet(h, int(colour), stream), h,
           "lbm_swap_inlet")


def lbm_get_geometry(h, cls, nw, stream):
    p = [None if t is None else _dptr(t) for t in (cls, nw)]
    _check(load_library().lbm_get_geometry(h, *p, stream), h,
           "lbm_get_geometry")


def lbm_counts(h):
    v = [C.c_int64() for _ in range(4)]
    _check(load_library().lbm_counts(h, *[C.byref(x) for x in v]), h,
           "lbm_counts")
    return tuple(x.value for x in v)


def lbm_colour_mass_noalloc(lattice, pops, stream):
    """Red and blue masses of a dense float32 population tensor
    (2, Q, ...) on the device, computed without any device allocation by
    the library (for callers that cannot allocate; see the C header).
    The tensor must be a contiguous float32 CUDA tensor on the current
    device with shape (2, Q, ...); anything else is refused here, before
    the library sees a pointer."""
    import torch
    if lattice not in (9, 19):
        raise LbmError("lbm_colour_mass_noalloc: lattice must be 9 or 19")
    if not isinstance(pops, torch.Tensor) or not pops.is_cuda:
        raise LbmError("lbm_colour_mass_noalloc: pops must be a CUDA tensor")
    torch = _torch()
    if pops.device.index != torch.cuda.current_device():
        raise LbmError("lbm_colour_mass_noalloc: pops is not on the "
                       "current device")
    if pops.dtype != torch.float32 or not pops.is_contiguous():
        raise LbmError("lbm_colour_mass_noalloc: pops must be contiguous "
                       "float32")
    if (pops.dim() < 3 or pops.shape[0] != 2 or pops.shape[1] != lattice
            or pops.numel() % (2 * lattice)):
        raise LbmError("lbm_colour_mass_noalloc: pops must have shape "
                       "(2, Q, ...)")
    out = (C.c_double * 2)()
    n = pops.numel() // (2 * lattice)
    _check(load_library().lbm_colour_mass_noalloc(lattice, n, _dptr(pops),
                                                  out, stream),
           None, "lbm_colour_mass_noalloc")
    return out[0], out[1]


def lbm_destroy(h):
    if h:
        load_library().lbm_destroy(h)


# ------------------------------------------------------------ Session
class Session:
    """One domain on the current CUDA device: the workspace (a torch uint8
    tensor), the library handle and the helpers that move fields in and
    out as torch tensors of shape (nz, ny, nx) (x fastest)."""

    def __init__(self, lattice: int, solid: np.ndarray, periodic=(True,) * 3,
                 storage: str = "fp32", device: str = "cuda", tile=None):
        torch = _torch()
        self.torch = torch
        solid = np.ascontiguousarray(solid, np.uint8)
        if solid.ndim == 2:
            solid = solid[None]
        self.q = lattice
        self.shape = solid.shape
        nz, ny, nx = self.shape
        self.N = nx * ny * nz
        self.storage = storage
        self.device = torch.device(device)
        mask = sum((1 << a) for a in range(3) if periodic[a])
        self.tile = None if tile is None else tuple(int(t) for t in tile)
        ws = lbm_workspace_bytes_tiled(lattice, nx, ny, nz, solid,
                                       STORAGE[storage], self.tile)
        if ws == 0:
            raise LbmError("bad domain or tile shape")
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self.h = lbm_init_geometry_tiled(lattice, nx, ny, nz, solid, mask,
                                         STORAGE[storage], self.tile,
                                         self.workspace, self.stream())
        self.counts = lbm_counts(self.h)
        self._solid = solid
        self.n_zou_he = 0

    def stream(self):
        return _stream(self.torch)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lbm_destroy(h)
            self.h = None

    @property
    def n_fluid(self) -> int:
        return int(self.counts[1])

    def set_params(self, **kw):
        lbm_set_params(self.h, make_params(**kw))
        # fluid nodes on the two Zou-He planes of the flow axis (host count)
        self.n_zou_he = 0
        if kw.get("zou_he"):
            ax = 2 - int(kw.get("flow_axis", 0))  # numpy axis of (z, y, x)
            fl = self._solid == 0
            self.n_zou_he = int(np.take(fl, 0, axis=ax).sum()
                                + np.take(fl, -1, axis=ax).sum())

    def init_state(self, phi0):
        t = self.torch.as_tensor(np.asarray(phi0, np.float32).reshape(self.shape)
                                 if isinstance(phi0, np.ndarray) else phi0)
        t = t.to(self.device, self.torch.float32).contiguous()
        lbm_init_state(self.h, t, self.stream())

    def step(self, n: int = 1):
        lbm_step(self.h, n, self.stream())

    def step_timed(self, n: int = 1) -> dict:
        """Per-pass milliseconds summed over n steps (CUDA events)."""
        return lbm_step_timed(self.h, n, self.stream())


    def macros(self):
        t = self.torch
        rho = t.empty(self.shape, dtype=t.float32, device=self.device)
        phi = t.empty_like(rho)
        u = t.empty((3,) + self.shape, dtype=t.float32, device=self.device)
        lbm_macros(self.h, rho, phi, u, self.stream())
        return dict(rho=rho, phi=phi, u=u)

    def reduce(self, kind: int) -> float:
        return lbm_reduce(self.h, kind, self.stream())

    def get_populations(self):
        t = self.torch
        out = t.empty((2, self.q) + self.shape, dtype=t.float32,
                      device=self.device)
        lbm_get_populations(self.h, out, self.stream())
        return out

    def set_populations(self, f):
        t = self.torch
        src = t.as_tensor(f).to(self.device, t.float32).contiguous()
        assert src.numel() == 2 * self.q * self.N
        lbm_set_populations(self.h, src, self.stream())

    def swap_inlet(self, colour: int):
        """Eqs. (37)-(38): the inlet plane's nodes become pure colour
        `colour` (0 = r, 1 = b)."""
        lbm_swap_inlet(self.h, colour, self.stream())

    def geometry(self):
        t = self.torch
        cls = t.empty(self.shape, dtype=t.uint8, device=self.device)
        nw = t.empty((3,) + self.shape, dtype=t.float32, device=self.device)
        lbm_get_geometry(self.h, cls, nw, self.stream())
        return cls, nw


def session_for(case, storage: str = "fp32") -> Session:
    """A Session set up from a :class:`workloads.Case` (geometry, params,
    initial state)."""
    s = Session(case.lattice, case.solid, case.periodic, storage)
    s.set_params(**case.params)
    s.init_state(case.phi0.astype(np.float32))
    return s


# ------------------------------------------------------------------ batches
def _bcheck(st: int, b=None, what: str = ""):
    if st != LBM_OK:
        msg = load_library().lbm_batch_last_error(b).decode() if b else ""
        raise LbmError(f"{what}: {STATUS.get(st, st)} {msg}")


def lbm_batch_workspace_bytes(ncases: int) -> int:
    return int(load_library().lbm_batch_workspace_bytes(int(ncases)))


def lbm_batch_create(handles, workspace, stream):
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p)
                                        else h for h in handles])
    out = C.c_void_p()
    _bcheck(load_library().lbm_batch_create(
        C.byref(out), arr, len(handles), C.c_void_p(workspace.data_ptr()),
        workspace.numel() * workspace.element_size(), stream),
        None, "lbm_batch_create")
    return out


def lbm_batch_set_config(b, mode: int, threads: int, chunk: int, stream):
    _bcheck(load_library().lbm_batch_set_config(b, int(mode), int(threads),
                                                int(chunk), stream),
            b, "lbm_batch_set_config")


def lbm_batch_step(b, nsteps: int, stream):
    _bcheck(load_library().lbm_batch_step(b, int(nsteps), stream), b,
            "lbm_batch_step")


def lbm_batch_status(b, stream) -> int:
    """The status code (LBM_OK or LBM_ERR_TIMEOUT), without raising."""
    return int(load_library().lbm_batch_status(b, stream))


def lbm_batch_check_wait(b, limit_ms: float, stream) -> float:
    waited = C.c_double()
    _bcheck(load_library().lbm_batch_check_wait(b, float(limit_ms),
                                                C.byref(waited), stream),
            b, "lbm_batch_check_wait")
    return waited.value


def lbm_batch_last_error(b) -> str:
    return load_library().lbm_batch_last_error(b).decode()


def lbm_batch_destroy(b):
    load_library().lbm_batch_destroy(b)


class Batch:
    """Many Sessions stepped together (``lbm_batch_*``). Keeps the Sessions
    alive; their results equal stepping each Session on its own."""

    def __init__(self, sessions):
        if not sessions:
            raise LbmError("empty batch")
        self.sessions = list(sessions)
        torch = self.sessions[0].torch
        self.torch = torch
        dev = self.sessions[0].device
        ws = lbm_batch_workspace_bytes(len(self.sessions))
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=dev)
        self.b = lbm_batch_create([s.h for s in self.sessions],
                                  self.workspace, self.stream())
        self.config = (0, 256, 4)

    def stream(self):
        return _stream(self.torch)

    def __del__(self):
        b = getattr(self, "b", None)
        if b:
            lbm_batch_destroy(b)
            self.b = None

    @property
    def n_fluid(self) -> int:
        return sum(s.n_fluid for s in self.sessions)

    def set_config(self, mode: int, threads: int = 256, chunk: int = 4):
        lbm_batch_set_config(self.b, mode, threads, chunk, self.stream())
        self.config = (int(mode), int(threads), int(chunk))

    def step(self, n: int = 1):
        lbm_batch_step(self.b, n, self.stream())

    def status(self) -> int:
        return lbm_batch_status(self.b, self.stream())

    def check_wait(self, limit_ms: float) -> float:
        return lbm_batch_check_wait(self.b, limit_ms, self.stream())


# ------------------------------------------------------ checkpoints, adjoint
def lbm_state_bytes(h) -> int:
    return int(load_library().lbm_state_bytes(h))


def lbm_save_state(h, dst, stream):
    _check(load_library().lbm_save_state(h, C.c_void_p(dst.data_ptr()), stream),
           h, "lbm_save_state")


def lbm_load_state(h, src, stream):
    _check(load_library().lbm_load_state(h, C.c_void_p(src.data_ptr()), stream),
           h, "lbm_load_state")


def _acheck(st: int, a=None, what: str = ""):
    if st != LBM_OK:
        msg = load_library().lbm_adj_last_error(a).decode() if a else ""
        raise LbmError(f"{what}: {STATUS.get(st, st)} {msg}")


def lbm_adj_workspace_bytes(h) -> int:
    return int(load_library().lbm_adj_workspace_bytes(h))


def lbm_adj_create(h, workspace):
    out = C.c_void_p()
    _acheck(load_library().lbm_adj_create(
        C.byref(out), h, C.c_void_p(workspace.data_ptr()),
        workspace.numel() * workspace.element_size()), None, "lbm_adj_create")
    return out


def lbm_adj_seed_sw(a, stream):
    _acheck(load_library().lbm_adj_seed_sw(a, stream), a, "lbm_adj_seed_sw")


def lbm_adj_step(a, stream):
    _acheck(load_library().lbm_adj_step(a, stream), a, "lbm_adj_step")


def lbm_adj_gradients(a, stream):
    out = (C.c_double * 4)()
    _acheck(load_library().lbm_adj_gradients(a, out, stream), a,
            "lbm_adj_gradients")
    return list(out)


def lbm_adj_get_lambda(a, lt, ls, stream):
    _acheck(load_library().lbm_adj_get_lambda(
        a, C.c_void_p(lt.data_ptr()), C.c_void_p(ls.data_ptr()), stream), a,
        "lbm_adj_get_lambda")


def lbm_adj_set_freeze(a, freeze_sin: float):
    _acheck(load_library().lbm_adj_set_freeze(a, float(freeze_sin)), a,
            "lbm_adj_set_freeze")


def lbm_adj_set_cmin(a, c_min: float):
    _acheck(load_library().lbm_adj_set_cmin(a, float(c_min)), a,
            "lbm_adj_set_cmin")


def lbm_adj_last_error(a) -> str:
    return load_library().lbm_adj_last_error(a).decode()


def lbm_adj_destroy(a):
    load_library().lbm_adj_destroy(a)
