"""torch.autograd bridge to the CUDA discrete adjoint (lbm_adjoint_run): the loss of an N-step
D2Q9 run as a differentiable function of the initial velocity field and of the relaxation
rates.  Argument marshalling only; the forward run, the checkpointing and the adjoint sweep all
execute in liblbm.so."""

import torch

from . import lbm


class LBMRun(torch.autograd.Function):
    """loss = LBMRun.apply(ux0, uy0, rates, rho0, nsteps, model, storage, loss_kind,
    ux_target, uy_target, checkpoint_every)

    ux0, uy0, rho0: float64 CUDA tensors [ny][nx] (initial equilibrium state, Sec. 5a);
    rates: float64 tensor (omega_nu, omega3, omega4); loss_kind 0 = misfit to the targets,
    1 = kinetic energy.  Gradients flow to ux0, uy0 and rates."""

    @staticmethod
    def forward(ctx, ux0, uy0, rates, rho0, nsteps, model, storage, loss_kind, ux_target, uy_target,
                checkpoint_every=0):
        ny, nx = ux0.shape
        r = [float(v) for v in rates.detach().cpu()]
        lat = lbm.Lattice(nx, ny, model, r, storage=storage)
        try:
            lat.init_equilibrium(rho0.contiguous(), ux0.detach().contiguous(), uy0.detach().contiguous())
            gx = torch.empty_like(ux0, dtype=torch.float64)
            gy = torch.empty_like(uy0, dtype=torch.float64)
            tx = ux_target.contiguous() if ux_target is not None else None
            ty = uy_target.contiguous() if uy_target is not None else None
            loss, grates, _ = lbm.lbm_adjoint_run(lat.ctx, nsteps, loss_kind, tx, ty, gx, gy, checkpoint_every)
        finally:
            lat.close()
        ctx.save_for_backward(gx, gy, torch.tensor(grates, dtype=rates.dtype, device=rates.device))
        return torch.tensor(loss, dtype=torch.float64, device=ux0.device)

    @staticmethod
    def backward(ctx, g):
        gx, gy, gr = ctx.saved_tensors
        return g * gx, g * gy, g.to(gr.device) * gr, None, None, None, None, None, None, None, None
