"""torch.autograd.Function over the GPU step: gradient of the final-time
perturbation energy with respect to the initial perturbation's coefficients.

Forward: tc_init_perturbation from the psi (and T') coefficients, nsteps
steps of fixed dt, J = E_pert = (1/2) int |u - u_base|^2 dV.  Every
``checkpoint`` steps the state is copied to a device tensor.
Backward: lambda = dJ/dX^N (tc_objective); for each segment, last first, the
segment is stepped again from its checkpoint with tc_step_record (each step's
state, predictor state and physical-grid fields kept in one device buffer)
and tc_adjoint_steps runs back through the records.  When a segment's
records would exceed ``record_budget`` bytes, its states alone are kept and
tc_adjoint_step recomputes each step's forward stages instead.
tc_init_perturbation_adjoint maps lambda^0 to the coefficients (the amplitude
scales of the initial condition are held fixed).
Marshalling only: all arithmetic runs in libtc.
"""
from __future__ import annotations

import numpy as np
import torch

from . import tc


class PerturbationEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, tcoef, run, nsteps, dt, amp, amp_T, checkpoint, record_budget):
        psi_np = psi.detach().cpu().numpy().astype(np.complex128)
        t_np = tcoef.detach().cpu().numpy().astype(np.complex128) if tcoef is not None else None
        run.init_perturbation(psi_np, amp, t_np, amp_T)
        shape = run.shape
        ckpts = []
        for n0 in range(0, nsteps, checkpoint):
            buf = torch.empty(shape, dtype=torch.complex128, device="cuda")
            tc.tc_get_state(run.ctx, buf)
            ckpts.append(buf)
            tc.tc_step(run.ctx, min(checkpoint, nsteps - n0), dt)
        J = tc.tc_objective(run.ctx)
        ctx.run, ctx.nsteps, ctx.dt, ctx.checkpoint = run, nsteps, dt, checkpoint
        ctx.record_budget = record_budget
        ctx.ckpts = ckpts
        ctx.mp, ctx.kp = psi.shape[1] - 1, (psi.shape[2] - 1) // 2
        ctx.with_T = tcoef is not None
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        run = ctx.run
        lam = torch.empty(run.shape, dtype=torch.complex128, device="cuda")
        tc.tc_objective(run.ctx, lam)
        lam *= float(gJ)
        nseg = len(ctx.ckpts)
        per_step = tc.tc_record_bytes_per_step(run.ctx)
        record = None
        if ctx.checkpoint * per_step <= ctx.record_budget:
            record = torch.empty(ctx.checkpoint * per_step, dtype=torch.uint8, device="cuda")
        for seg in range(nseg - 1, -1, -1):
            n0 = seg * ctx.checkpoint
            n1 = min(ctx.nsteps, n0 + ctx.checkpoint)
            tc.tc_set_state(run.ctx, ctx.ckpts[seg])
            if record is not None:
                tc.tc_step_record(run.ctx, n1 - n0, ctx.dt, record)
                tc.tc_adjoint_steps(run.ctx, n1 - n0, record, ctx.dt, lam)
                continue
            states = []
            for n in range(n0, n1):
                buf = torch.empty(run.shape, dtype=torch.complex128, device="cuda")
                tc.tc_get_state(run.ctx, buf)
                states.append(buf)
                if n + 1 < n1:
                    tc.tc_step(run.ctx, 1, ctx.dt)
            for buf in reversed(states):
                tc.tc_adjoint_step(run.ctx, buf, ctx.dt, lam)
        pb, tb = tc.tc_init_perturbation_adjoint(run.ctx, lam, ctx.mp, ctx.kp, ctx.with_T)
        g_psi = torch.from_numpy(pb)
        g_t = torch.from_numpy(tb) if tb is not None else None
        return g_psi, g_t, None, None, None, None, None, None, None


def perturbation_energy(run, psi, nsteps, dt, amp, tcoef=None, amp_T=0.0, checkpoint=20,
                        record_budget=4 << 30):
    """J(psi) = E_pert after nsteps; differentiable in psi (and tcoef).

    record_budget: device bytes one checkpoint segment's records may take
    (0: always recompute each step's forward stages in the adjoint)."""
    return PerturbationEnergy.apply(psi, tcoef, run, nsteps, dt, amp, amp_T, checkpoint,
                                    record_budget)
