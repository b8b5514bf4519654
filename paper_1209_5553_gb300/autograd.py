"""Temperature misfit of an EREM run as a torch.autograd.Function.

Forward: the steady pressure for ln K (the library's Jacobi CG), the state of
the heat problem, ``steps`` EREM steps (eq. ``EERM`` with real Leja phi_1,
§4.2) from T0, and L = sum_o (T^N_o - data_o)^2 over the observation cells.
Backward: the library's adjoint entry points (erem_adjoint_*), one step at a
time from T^N back to T^0 with every step's Leja schedule frozen at its
forward value; the states T^n are recomputed from checkpoints kept every
``checkpoint`` steps by replaying those schedules, so at most ``checkpoint``
states are held at once.  With ``tape`` (default "segment") the replay of a
segment records its Newton vectors on the device (erem_adjoint_tape) and the
adjoint steps use them instead of computing them a second time.  With
``tape="full"`` the forward run itself records them and keeps every state
(60 steps at 128^3 in FP32-bulk fill about 12 GB), so the backward pass
replays nothing.
Gradients with respect to ln K and T0.

The adjoint differentiates the run with the interval of every step held at
its forward value; ``interval=`` holds it (``MisfitModel.interval`` of a
forward run) so that perturbed forwards evaluate that same map.

Argument marshalling and step sequencing only: every step runs in the
library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Context, Physics, leja_opts


class MisfitModel:
    """Grid, physics and run length of the misfit (one library context).

    physics: the heat-model constants and heads (fluid_model 0);
    phi, lam: porosity and conductivity fields [N] (CUDA FP64 tensors);
    obs: observation cells (CUDA int64), data: observed values (CUDA FP64)."""

    def __init__(self, dim, nx, ny, nz, physics: Physics, phi, lam, dt, steps, obs, data,
                 precision="fp32_bulk", checkpoint=10, tol=1e-6, pressure_tol=1e-12,
                 replay=None, interval=None, tape=True):
        if physics.fluid_model != 0:
            raise ValueError("the adjoint needs fluid_model 0")
        self.ctx = Context(dim, nx, ny, nz, physics=physics, precision=precision)
        self.n = nx * ny * nz
        self.nx = nx
        self.n_padded = (nx + 3) // 4 * 4 * ny * nz
        self.qbytes = 4 if precision == "fp32_bulk" else 8
        self.tape = {True: "segment", False: None, None: None}.get(tape, tape)
        if self.tape not in (None, "segment", "full"):
            raise ValueError("tape must be 'segment', 'full' or False")
        self.physics = physics
        self.phi, self.lam = phi, lam
        self.dt, self.steps = float(dt), int(steps)
        self.obs, self.data = obs, data
        self.checkpoint = max(1, int(checkpoint))
        self.tol, self.pressure_tol = tol, pressure_tol
        self.replay = replay          # forced schedules (one per step), or None
        self.schedules = []           # schedules of the last forward run
        self.interval = None          # Gershgorin interval of J of the last forward run
        if interval is not None:      # held: the map the adjoint differentiates
            self.ctx.hold_interval(interval)

    def head_guess(self, like):
        x = (torch.arange(self.nx, dtype=torch.float64, device=like.device) + 0.5) / self.nx
        ramp = self.physics.head_left + (self.physics.head_right - self.physics.head_left) * x
        return ramp.repeat(self.n // self.nx).contiguous()

    def full_tape_reserve(self):
        """Arena for a whole run: room for 64 Newton vectors a step (plus one
        interpolation's look-ahead), at most half the free device memory.  A run
        that outgrows it is not taped at all: the adjoint then recomputes every
        step from the kept states."""
        free, _ = torch.cuda.mem_get_info()
        want = (self.steps + 1) * 64 * self.qbytes * self.n_padded
        return int(min(want, 0.5 * free))

    def tape_bytes(self, scheds):
        """Device bytes the adjoint tape needs for these steps."""
        total = 0
        for sc in scheds:
            s = sc[0]
            total += (s - 1) * 8 * self.n_padded
            total += sum(m + 1 for m in sc[1:]) * self.qbytes * self.n_padded
        return total

    def close(self):
        self.ctx.close()


class EremMisfit(torch.autograd.Function):
    @staticmethod
    def forward(fctx, lnk, T0, model: MisfitModel):
        m = model
        lnk = lnk.detach().contiguous()
        p = m.head_guess(lnk)
        m.ctx.pressure_solve(lnk, None, p, tol=m.pressure_tol, maxit=1000000)
        T = T0.detach().clone().contiguous()
        m.ctx.set_state(T, p, lnk, m.phi, m.lam, m.dt)
        full = m.tape == "full"
        if full:   # record the forward run itself
            m.ctx.adjoint_tape(m.full_tape_reserve(), True)
        ckpts = {0: T.clone()}
        scheds = []
        for n in range(m.steps):
            opts = leja_opts(tol=m.tol) if m.replay is None else leja_opts(tol=m.tol, replay=m.replay[n])
            st = m.ctx.erem_step(T, m.dt, opts=opts)
            scheds.append(st.schedule)
            if n == 0:
                m.interval = (st.alpha / m.dt, st.beta / m.dt)
            if n + 1 < m.steps and (full or (n + 1) % m.checkpoint == 0):
                ckpts[n + 1] = T.clone()
        m.schedules = scheds
        fctx.model, fctx.ckpts, fctx.scheds = m, ckpts, scheds
        fctx.save_for_backward(lnk, T)
        r = T[m.obs] - m.data
        return (r * r).sum()

    @staticmethod
    def backward(fctx, gL):
        m, ckpts, scheds = fctx.model, fctx.ckpts, fctx.scheds
        lnk, TN = fctx.saved_tensors
        lam = torch.zeros_like(TN)
        lam[m.obs] = 2.0 * (TN[m.obs] - m.data) * gL
        m.ctx.adjoint_begin()
        if m.tape == "full":  # every state kept and every step taped by the forward run
            for n in range(m.steps - 1, -1, -1):
                m.ctx.adjoint_step(ckpts[n], lam, scheds[n])
            m.ctx.adjoint_tape(0, False)
            glnk = torch.zeros_like(lnk)
            m.ctx.adjoint_lnk(lnk, glnk, tol=m.pressure_tol)
            return glnk, lam, None
        starts = sorted(ckpts)
        for a, s0 in reversed(list(enumerate(starts))):
            s1 = starts[a + 1] if a + 1 < len(starts) else m.steps
            if m.tape:  # every step of the segment recorded once, consumed backwards
                m.ctx.adjoint_tape(m.tape_bytes(scheds[s0:s1]), True)
            states = [ckpts[s0].clone()]
            T = states[0].clone()
            last = s1 if m.tape else s1 - 1
            for n in range(s0, last):
                m.ctx.erem_step(T, m.dt, opts=leja_opts(tol=m.tol, replay=scheds[n]))
                if n + 1 < s1:
                    states.append(T.clone())
            for n in range(s1 - 1, s0 - 1, -1):
                m.ctx.adjoint_step(states[n - s0], lam, scheds[n])
            if m.tape:
                m.ctx.adjoint_tape(0, False)
        glnk = torch.zeros_like(lnk)
        m.ctx.adjoint_lnk(lnk, glnk, tol=m.pressure_tol)
        return glnk, lam, None


def misfit(lnk, T0, model: MisfitModel):
    """L(lnK, T0) with gradients through the adjoint (see EremMisfit)."""
    return EremMisfit.apply(lnk, T0, model)
