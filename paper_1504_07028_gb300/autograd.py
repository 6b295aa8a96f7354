"""torch.autograd.Function around the differentiable solver (segsalsa_str_backward).

z = UnrolledSegSalsa.apply(log_p, lam, omega, solver, iters, checkpoint_every) returns z^T of
`iters` SALSA iterations from p = exp(log p) (class-major (K, H, W) device tensor in the
solver's precision), with lambda `lam` and shift weights `omega` (L values); backward gives the
gradients with respect to log p, lam and omega. Argument marshalling only: the forward and the
reverse pass run in the library's kernels. `solver` is a binding.Solver whose H, W, K, M, mu
and Schatten p fix the rest of the problem.
"""
from __future__ import annotations

import numpy as np
import torch


class UnrolledSegSalsa(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_p, lam, omega, solver, iters, checkpoint_every=10):
        lam_v = float(lam)
        om_v = omega.detach().to(torch.float64).cpu().numpy()
        lp = log_p.detach().contiguous()
        solver.set_lambda(lam_v)
        solver.set_weights(om_v)
        solver.set_log_probs(lp)
        solver.solve(int(iters))
        z = torch.empty_like(lp)
        solver.get_z(z)
        ctx.solver, ctx.iters, ctx.every = solver, int(iters), int(checkpoint_every)
        ctx.lam, ctx.om = lam_v, om_v
        ctx.save_for_backward(lp)
        ctx.lam_like, ctx.om_like = (lam if torch.is_tensor(lam) else None), omega
        return z

    @staticmethod
    def backward(ctx, zbar):
        (lp,) = ctx.saved_tensors
        s = ctx.solver
        s.set_lambda(ctx.lam)            # the solver may have been used since the forward
        s.set_weights(ctx.om)
        s.set_log_probs(lp)
        g, glam, gom = s.backward(ctx.iters, zbar.contiguous().to(lp.dtype), ctx.every)
        dev_l = ctx.lam_like.device if ctx.lam_like is not None else lp.device
        glam_t = torch.tensor(glam, dtype=torch.float64, device=dev_l)
        gom_t = torch.from_numpy(np.asarray(gom)).to(ctx.om_like.device, ctx.om_like.dtype)
        return g, glam_t, gom_t, None, None, None
