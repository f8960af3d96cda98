"""Python handle on the FP64 CPU oracle (``lbm_oracle.cpp``).

Test infrastructure only: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product path never does.

Arrays follow the project's layout: a field has numpy shape ``(nz, ny, nx)``
(x fastest), populations ``(2, Q, nz, ny, nx)`` with colour 0 = red, 1 = blue,
vector fields ``(3, nz, ny, nx)``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.cpp")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

MASS_R, MASS_B, SW_COUNT, SW_SMOOTH, DP, CA_R, CA_B = range(7)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, OpenMP) next to its source."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                    _SRC, "-o", tmp], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("tau_r", C.c_double), ("tau_b", C.c_double),
                ("gamma", C.c_double), ("beta", C.c_double),
                ("rho0", C.c_double), ("theta_deg", C.c_double),
                ("wetting", C.c_int), ("zou_he", C.c_int),
                ("flow_axis", C.c_int),
                ("rho_in", C.c_double), ("rho_out", C.c_double),
                ("zeta_r", C.c_double), ("g", C.c_double * 3),
                ("collision", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.c_void_p, C.c_uint]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_params.restype = C.c_int
        L.orc_set_params.argtypes = [C.c_void_p, C.POINTER(_Params)]
        L.orc_collide_mrt.argtypes = [C.c_void_p, C.c_void_p, C.c_double,
                                      C.c_double, C.c_double, C.c_double,
                                      C.c_void_p, C.c_void_p]
        L.orc_moment_matrix.argtypes = [C.c_void_p]
        L.orc_init_state.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_set_pops.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_get_pops.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_swap_inlet.argtypes = [C.c_void_p, C.c_int]
        L.orc_swap_inlet.restype = C.c_long
        L.orc_stream_only.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_extrapolate.argtypes = [C.c_void_p] + [C.c_void_p] * 4
        L.orc_stencils.argtypes = [C.c_void_p] + [C.c_void_p] * 5
        L.orc_collide_recolour.argtypes = [C.c_void_p] + [C.c_void_p] * 7
        L.orc_geometry.argtypes = [C.c_void_p] + [C.c_void_p] * 3
        L.orc_fields.argtypes = [C.c_void_p] + [C.c_void_p] * 6
        L.orc_reduce.restype = C.c_double
        L.orc_reduce.argtypes = [C.c_void_p, C.c_int]
        L.orc_lattice.restype = C.c_int
        L.orc_lattice.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_scheme1.argtypes = [dp, dp, C.c_double, dp]
        L.orc_scheme2.argtypes = [dp, dp, C.c_double, dp]
        L.orc_collide.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_double,
                                  C.c_double, C.c_void_p, C.c_void_p]
        L.orc_max_threads.restype = C.c_int
        L.orc_tlm_create.restype = C.c_void_p
        L.orc_tlm_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_void_p, C.c_uint]
        L.orc_tlm_destroy.argtypes = [C.c_void_p]
        L.orc_tlm_set_params.restype = C.c_int
        L.orc_tlm_set_params.argtypes = [C.c_void_p, C.POINTER(_Params),
                                         C.c_int]
        L.orc_tlm_init_state.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_tlm_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_tlm_sw.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_tlm_set_freeze.argtypes = [C.c_void_p, C.c_double]
        L.orc_tlm_set_cmin.argtypes = [C.c_void_p, C.c_double]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _vec(v):
    return (C.c_double * 3)(*[float(x) for x in v])


def lattice(q: int):
    """Velocities (Q, 3), weights (Q,), opposite index (Q,)."""
    e = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    o = np.zeros(19, np.int32)
    n = lib().orc_lattice(q, _ptr(e), _ptr(w), _ptr(o))
    return e[:n].copy(), w[:n].copy(), o[:n].copy()


def scheme1(n_c, n_w, theta_rad):
    out = (C.c_double * 3)()
    lib().orc_scheme1(_vec(n_c), _vec(n_w), float(theta_rad), out)
    return np.array(out[:])


def scheme2(n_c, n_w, theta_rad):
    out = (C.c_double * 3)()
    lib().orc_scheme2(_vec(n_c), _vec(n_w), float(theta_rad), out)
    return np.array(out[:])


def collide(q, ft, F, S, rho0=1.0):
    ft = np.ascontiguousarray(ft, np.float64)
    Fv = np.ascontiguousarray(F, np.float64)
    out = np.zeros(q)
    u = np.zeros(3)
    lib().orc_collide(q, _ptr(ft), _ptr(Fv), float(S), float(rho0),
                      _ptr(out), _ptr(u))
    return out, u


def collide_mrt(ft, F, S, rho0=1.0, Sq=None, Sm=None):
    """MRT collision of one D3Q19 node (Eq. 2 in moment space); S_q and S_m
    default to Eq. (16)."""
    ft = np.ascontiguousarray(ft, np.float64)
    Fv = np.ascontiguousarray(F, np.float64)
    if Sq is None:
        Sq = mrt_rate(S)
    if Sm is None:
        Sm = mrt_rate(S)
    out = np.zeros(19)
    u = np.zeros(3)
    lib().orc_collide_mrt(_ptr(ft), _ptr(Fv), float(S), float(Sq), float(Sm),
                          float(rho0), _ptr(out), _ptr(u))
    return out, u


def mrt_rate(S):
    """Eq. (16): S_q = S_m = 8 (2 - S_nu) / (8 - S_nu)."""
    return 8.0 * (2.0 - S) / (8.0 - S)


def moment_matrix():
    """The oracle's M (Eq. A.3), built from the moment polynomials."""
    M = np.zeros(19 * 19)
    lib().orc_moment_matrix(_ptr(M))
    return M.reshape(19, 19)


PARAM_DEFAULTS = dict(tau_r=1.0, tau_b=1.0, gamma=0.01, beta=0.7, rho0=1.0,
                      theta_deg=90.0, wetting=0, zou_he=0, flow_axis=0,
                      rho_in=1.0, rho_out=1.0, zeta_r=1.0, g=(0.0, 0.0, 0.0),
                      collision=0)


class Oracle:
    """One oracle domain: geometry, state and parameters."""

    def __init__(self, lattice_q: int, solid: np.ndarray,
                 periodic=(True, True, True)):
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        if solid.ndim == 2:
            solid = solid[None]
        self.q = lattice_q
        self.shape = solid.shape  # (nz, ny, nx)
        nz, ny, nx = self.shape
        self.N = nx * ny * nz
        self.solid = solid
        mask = sum((1 << a) for a in range(3) if periodic[a])
        self._h = lib().orc_create(lattice_q, nx, ny, nz, _ptr(solid), mask)
        if not self._h:
            raise ValueError("oracle: bad lattice/shape")
        self.params = dict(PARAM_DEFAULTS)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    def set_params(self, **kw):
        for k in kw:
            if k not in PARAM_DEFAULTS:
                raise KeyError(k)
        self.params.update(kw)
        p = self.params
        st = _Params(p["tau_r"], p["tau_b"], p["gamma"], p["beta"], p["rho0"],
                     p["theta_deg"], int(p["wetting"]), int(p["zou_he"]),
                     int(p["flow_axis"]), p["rho_in"], p["rho_out"],
                     p["zeta_r"], (C.c_double * 3)(*p["g"]),
                     int(p["collision"]))
        if lib().orc_set_params(self._h, C.byref(st)) != 0:
            raise ValueError("collision must be 0 or 1 (MRT: D3Q19 only)")

    def init_state(self, phi0: np.ndarray):
        a = np.ascontiguousarray(np.broadcast_to(phi0, self.shape), np.float64)
        lib().orc_init_state(self._h, _ptr(a))

    @property
    def pops(self) -> np.ndarray:
        out = np.zeros((2, self.q) + self.shape)
        lib().orc_get_pops(self._h, _ptr(out))
        return out

    @pops.setter
    def pops(self, f: np.ndarray):
        a = np.ascontiguousarray(f, np.float64).reshape((2, self.q) + self.shape)
        lib().orc_set_pops(self._h, _ptr(a))

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def swap_inlet(self, colour: int) -> int:
        """Eqs. (37)-(38) on the inlet plane of the flow axis: the nodes
        become pure colour `colour` (0 = r, 1 = b). Returns the number of
        nodes changed."""
        n = lib().orc_swap_inlet(self._h, int(colour))
        if n < 0:
            raise ValueError("colour must be 0 (r) or 1 (b)")
        return int(n)

    def stream_only(self) -> np.ndarray:
        """Streamed (and Zou-He rebuilt) populations of the next step,
        without changing the stored state."""
        out = np.zeros((2, self.q) + self.shape)
        lib().orc_stream_only(self._h, _ptr(out))
        return out

    def extrapolate(self, phi: np.ndarray, nc: np.ndarray):
        """Eqs. (34)-(35) alone on a prescribed phase field (nz, ny, nx) and
        n_c (3, nz, ny, nx) of the fluid nodes: returns both fields with the
        solid-boundary nodes filled. The stored state is not changed."""
        pi = np.ascontiguousarray(phi, np.float64)
        ni = np.ascontiguousarray(nc, np.float64)
        po = np.zeros(self.shape)
        no = np.zeros((3,) + self.shape)
        lib().orc_extrapolate(self._h, _ptr(pi), _ptr(ni), _ptr(po), _ptr(no))
        return po, no

    def stencils(self, phi: np.ndarray, nc: np.ndarray):
        """Eqs. (6), (11) on a prescribed phase field (nz, ny, nx) and Eq.
        (12) on a prescribed n_c (3, nz, ny, nx): returns C, n_c and kappa.
        The stored state is not changed."""
        pi = np.ascontiguousarray(phi, np.float64)
        ni = np.ascontiguousarray(nc, np.float64)
        Co = np.zeros((3,) + self.shape)
        no = np.zeros((3,) + self.shape)
        ko = np.zeros(self.shape)
        lib().orc_stencils(self._h, _ptr(pi), _ptr(ni), _ptr(Co), _ptr(no),
                           _ptr(ko))
        return Co, no, ko

    def collide_recolour(self, ft, rho_r, rho_b, phi, nc, F):
        """Eq. (2) and Eqs. (20)-(21) alone on a prescribed state: ft
        (2, Q, nz, ny, nx) the streamed populations, rho_r, rho_b and phi
        (nz, ny, nx), nc and F (3, nz, ny, nx). Returns the post-recolouring
        populations (2, Q, nz, ny, nx); the stored populations are not
        changed."""
        q = ft.shape[1]
        a = [np.ascontiguousarray(x, np.float64)
             for x in (ft, rho_r, rho_b, phi, nc, F)]
        out = np.zeros((2, q) + self.shape)
        lib().orc_collide_recolour(self._h, *[_ptr(x) for x in a], _ptr(out))
        return out

    def geometry(self):
        cls = np.zeros(self.shape, np.uint8)
        gsm = np.zeros(self.shape)
        nw = np.zeros((3,) + self.shape)
        lib().orc_geometry(self._h, _ptr(cls), _ptr(gsm), _ptr(nw))
        return cls, gsm, nw

    def fields(self):
        rho = np.zeros(self.shape)
        phi = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        nc = np.zeros((3,) + self.shape)
        kap = np.zeros(self.shape)
        F = np.zeros((3,) + self.shape)
        lib().orc_fields(self._h, _ptr(rho), _ptr(phi), _ptr(u), _ptr(nc),
                         _ptr(kap), _ptr(F))
        return dict(rho=rho, phi=phi, u=u, nc=nc, kappa=kap, F=F)

    def reduce(self, kind: int) -> float:
        return lib().orc_reduce(self._h, int(kind))


class TangentLinear:
    """The oracle's step on forward-mode dual numbers (FP64): the smooth
    saturation after n steps and its derivatives with respect to the
    contact angle (per radian) and the component g_axis of the body
    acceleration."""

    def __init__(self, lattice_q: int, solid: np.ndarray,
                 periodic=(True, True, True), g_axis: int = 0):
        self.g_axis = int(g_axis)
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        if solid.ndim == 2:
            solid = solid[None]
        self.shape = solid.shape
        nz, ny, nx = self.shape
        mask = sum((1 << a) for a in range(3) if periodic[a])
        self._h = lib().orc_tlm_create(lattice_q, nx, ny, nz, _ptr(solid),
                                       mask)
        if not self._h:
            raise ValueError("oracle: bad lattice/shape")
        self.params = dict(PARAM_DEFAULTS)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_tlm_destroy(h)
            self._h = None

    def set_params(self, **kw):
        for k in kw:
            if k not in PARAM_DEFAULTS:
                raise KeyError(k)
        self.params.update(kw)
        p = self.params
        st = _Params(p["tau_r"], p["tau_b"], p["gamma"], p["beta"], p["rho0"],
                     p["theta_deg"], int(p["wetting"]), int(p["zou_he"]),
                     int(p["flow_axis"]), p["rho_in"], p["rho_out"],
                     p["zeta_r"], (C.c_double * 3)(*p["g"]),
                     int(p["collision"]))
        if lib().orc_tlm_set_params(self._h, C.byref(st), self.g_axis) != 0:
            raise ValueError("collision must be 0 or 1 (MRT: D3Q19 only)")

    def init_state(self, phi0: np.ndarray):
        a = np.ascontiguousarray(np.broadcast_to(phi0, self.shape), np.float64)
        lib().orc_tlm_init_state(self._h, _ptr(a))

    def set_freeze(self, freeze_sin: float):
        """Hold Scheme-II's direction around n_w constant in the
        linearisation where sin(theta') < freeze_sin (0: exact)."""
        lib().orc_tlm_set_freeze(self._h, float(freeze_sin))

    def set_cmin(self, c_min: float):
        """Hold the direction of n_c constant in the linearisation where
        |C| < c_min (0: exact)."""
        lib().orc_tlm_set_cmin(self._h, float(c_min))

    def step(self, n: int = 1):
        lib().orc_tlm_step(self._h, int(n))

    def sw(self):
        """(S_w smooth, dS_w/dtheta per radian, dS_w/dg[g_axis])."""
        out = np.zeros(3)
        lib().orc_tlm_sw(self._h, _ptr(out))
        return float(out[0]), float(out[1]), float(out[2])


def max_threads() -> int:
    return lib().orc_max_threads()
