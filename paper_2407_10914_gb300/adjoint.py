"""Gradients of the final smooth saturation with respect to the contact
angle and the body force, by the hand-written adjoint of the time step
(``lbm_adj_*``) with checkpoints and recomputation.

J(theta, g) = LBM_SW_SMOOTH after T steps from a given initial phase field:
the mean over fluid nodes of (1 - phi)/2 (the wetting-phase saturation in
its smooth form), phi taken from the last step's streamed populations, so J
depends on x_{T-1}. The forward run keeps x_0, x_K, x_2K, ... (K about
sqrt(T)); the reverse sweep rebuilds each segment of K states from its
checkpoint and reverses the steps one by one, so memory holds about 2
sqrt(T) states and the work is about 3T steps. Every step runs in the CUDA
library; this module only schedules the calls.

freeze_sin (default 0.05) and c_min (default 1e-3) regularise the
linearisation (lbm_adj_set_freeze, lbm_adj_set_cmin): over long runs the
exact derivative of the discrete step grows without bound through wetting
nodes where n_c is almost along n_w (Jacobian ~ 1/sin(theta')) and through
the interface tails (Jacobian of n_c = C/|C| ~ 1/|C|). Zeros give the exact
derivative, right for short runs.

``SwGradient`` wraps it as a torch.autograd.Function of (theta in degrees,
g as a 3-vector): J.backward() fills their .grad.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

from . import lbm


class Run:
    """One checkpointed forward run of a Session and its reverse sweep."""

    def __init__(self, session, phi0, steps: int, every: Optional[int] = None,
                 freeze_sin: float = 0.05, c_min: float = 1e-3):
        if steps < 1:
            raise ValueError("steps must be >= 1")
        self.s = session
        self.phi0 = np.asarray(phi0, np.float32)
        self.T = int(steps)
        self.K = int(every) if every else max(1, int(round(math.sqrt(steps))))
        torch = session.torch
        self.nb = lbm.lbm_state_bytes(session.h)
        self._new = lambda: torch.empty(self.nb, dtype=torch.uint8,
                                        device=session.device)
        self.freeze_sin = float(freeze_sin)
        self.c_min = float(c_min)
        self.checkpoints = {}
        self.last = None  # x_{T-1}
        self.J = None

    def forward(self) -> float:
        s, st = self.s, self.s.stream()
        s.init_state(self.phi0)
        for t in range(self.T - 1):
            if t % self.K == 0:
                buf = self._new()
                lbm.lbm_save_state(s.h, buf, st)
                self.checkpoints[t] = buf
            s.step(1)
        self.last = self._new()
        lbm.lbm_save_state(s.h, self.last, st)
        s.step(1)
        self.J = s.reduce(lbm.LBM_SW_SMOOTH)
        return self.J

    def backward(self):
        """dJ/dtheta (per radian) and dJ/dg (3) by the reverse sweep."""
        s, st = self.s, self.s.stream()
        torch = s.torch
        ws = torch.empty(lbm.lbm_adj_workspace_bytes(s.h), dtype=torch.uint8,
                         device=s.device)
        a = lbm.lbm_adj_create(s.h, ws)
        try:
            lbm.lbm_adj_set_freeze(a, self.freeze_sin)
            lbm.lbm_adj_set_cmin(a, self.c_min)
            lbm.lbm_load_state(s.h, self.last, st)
            lbm.lbm_adj_seed_sw(a, st)
            n_states = self.T - 1  # x_0 .. x_{T-2} are reversed
            seg = [None] * self.K
            for t0 in reversed(range(0, n_states, self.K)):
                t1 = min(t0 + self.K, n_states)
                lbm.lbm_load_state(s.h, self.checkpoints[t0], st)
                for t in range(t0, t1):
                    if seg[t - t0] is None:
                        seg[t - t0] = self._new()
                    lbm.lbm_save_state(s.h, seg[t - t0], st)
                    if t + 1 < t1:
                        s.step(1)
                for t in reversed(range(t0, t1)):
                    lbm.lbm_load_state(s.h, seg[t - t0], st)
                    lbm.lbm_adj_step(a, st)
            g = lbm.lbm_adj_gradients(a, st)
        finally:
            lbm.lbm_adj_destroy(a)
        return g[0], np.array(g[1:4])


class SwGradient:
    """torch.autograd.Function: J = SwGradient.apply(theta_deg, g, session,
    case_params, phi0, steps) with theta_deg a 0-d tensor (degrees) and g a
    3-tensor; the other arguments are fixed. Built lazily so that importing
    this module needs no torch."""

    _fn = None

    @classmethod
    def apply(cls, theta_deg, g, session, params: dict, phi0, steps: int,
              every: Optional[int] = None):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, th, gg, sess, prm, p0, n, k):
                    p = dict(prm)
                    p["theta_deg"] = float(th)
                    p["g"] = tuple(float(v) for v in gg.tolist())
                    sess.set_params(**p)
                    run = Run(sess, p0, n, k)
                    J = run.forward()
                    ctx.run = run
                    ctx.dev = th.device
                    return torch.tensor(J, dtype=torch.float64, device=th.device)

                @staticmethod
                def backward(ctx, gJ):
                    dth, dg = ctx.run.backward()
                    scale = float(gJ)
                    d_theta = torch.tensor(scale * dth * math.pi / 180.0,
                                           dtype=torch.float64, device=ctx.dev)
                    d_g = torch.tensor(scale * dg, dtype=torch.float64,
                                       device=ctx.dev)
                    return d_theta, d_g, None, None, None, None, None

            cls._fn = _F
        return cls._fn.apply(theta_deg, g, session, params, phi0, steps, every)
