"""Gradients of a final-state loss with respect to the initial fields, through
the hand-written discrete-adjoint kernel (amr_hydro_step_adjoint) behind a
torch.autograd.Function, with sqrt(N) step checkpointing and recompute.

The time steps of the base forward run are recorded and frozen: the forward,
the adjoint and any finite-difference run use the same dt sequence.
Marshalling only: every step and every adjoint step runs in libamr_hydro.so.
"""
import math

import torch

from . import amr_hydro as A
from .uniform import UniformGrid


class CheckpointedRun:
    """N FP64 steps of a periodic box with a frozen dt sequence; the backward
    pass stores a checkpoint every ceil(sqrt(N)) steps and recomputes each
    segment's states before reversing it."""

    def __init__(self, shape, gamma=5.0 / 3.0, cfl=0.5, stream=None):
        self.grid = UniformGrid(shape, gamma=gamma, cfl=cfl, prec=A.AMR_FP64, stream=stream)
        self.shape = shape

    def close(self):
        self.grid.close()

    def record_dts(self, U0, n_steps):
        """Base forward run: dt of every step from Eq. (CFL2)."""
        g = self.grid
        g.upload(U0)
        dts = []
        for _ in range(n_steps):
            dt = g.min_dt()
            dts.append(dt)
            g.step(dt)
        return dts

    def forward(self, U0, dts):
        """U0: dense [5][nz][ny][nx] cuda tensor -> final dense state; keeps
        the checkpoints for backward."""
        g = self.grid
        g.upload(U0)
        n = len(dts)
        self.K = max(1, math.ceil(math.sqrt(n)))
        self.dts = list(dts)
        self.ckpt = {}
        for k, dt in enumerate(self.dts):
            if k % self.K == 0:
                self.ckpt[k] = g.state().clone()
            g.step(dt)
        return self.grid.download(out=torch.empty_like(U0))

    def backward(self, lam_dense):
        """dL/dU0 from dL/dU_N (dense cuda tensors)."""
        g = self.grid
        nx, ny, nz = self.shape
        lam = torch.empty_like(g.state())
        A.amr_hydro_pack_uniform(lam_dense.contiguous(), nx, ny, nz, lam, g.stream)
        tmp = torch.empty_like(lam)
        n = len(self.dts)
        starts = sorted(self.ckpt)
        for s0 in reversed(starts):
            s1 = min(s0 + self.K, n)
            # recompute the segment's states from its checkpoint
            states = [self.ckpt[s0]]
            g.state().copy_(self.ckpt[s0])
            A.amr_hydro_touch_level(g.ctx, 0)
            for k in range(s0, s1 - 1):
                g.step(self.dts[k])
                states.append(g.state().clone())
            for k in range(s1 - 1, s0 - 1, -1):
                A.amr_hydro_step_adjoint(g.ctx, 0, self.dts[k], states[k - s0], lam, tmp)
                lam, tmp = tmp, lam
        out = torch.empty_like(lam_dense)
        A.amr_hydro_unpack_uniform(lam, nx, ny, nz, out, g.stream)
        return out


class HydroRun(torch.autograd.Function):
    """U_N = S_{N-1} o ... o S_0 (U_0) with frozen time steps; backward runs
    the discrete adjoint."""

    @staticmethod
    def forward(ctx, U0, runner, dts):
        ctx.runner = runner
        return runner.forward(U0.detach(), dts)

    @staticmethod
    def backward(ctx, grad):
        return ctx.runner.backward(grad), None, None


def density_loss(U_final, rho_target, dV):
    """L = 1/2 sum_cells (rho - rho*)^2 dV."""
    return 0.5 * ((U_final[0] - rho_target) ** 2).sum() * dV
