"""torch.autograd.Function over the discrete adjoint of the coupled step.

``deformation(factory, E_ext, G, Q, nsteps, ckpt_every, dn0_dQ)`` returns the
drop deformation D after ``nsteps`` steps of the system that ``factory(E_ext,
G, Q)`` builds and loads, as a tensor differentiable in E_ext (3,), G and Q.
The forward call runs lbeh_step_adjoint once (forward sweep with checkpoints,
then the reverse sweep); backward scales the stored derivatives by the
incoming gradient.  Marshalling only: all arithmetic runs in the library.
"""
import numpy as np
import torch


class _Deformation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E_ext, G, Q, factory, nsteps, ckpt_every, dn0_dQ):
        e = [float(v) for v in E_ext.detach().cpu().reshape(3)]
        s = factory(e, float(G), float(Q))
        try:
            g = s.step_adjoint(int(nsteps), int(ckpt_every), d_deformation=1.0, dn0_dQ=dn0_dQ)
        finally:
            s.close()
        ctx.save_for_backward(torch.tensor(g["dE_ext"], dtype=torch.float64),
                              torch.tensor(g["dG"], dtype=torch.float64),
                              torch.tensor(g["dQ"], dtype=torch.float64))
        ctx.status = g["status"]
        return torch.tensor(g["deformation"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad):
        dE, dG, dQ = ctx.saved_tensors
        return grad * dE, grad * dG, grad * dQ, None, None, None, None


def deformation(factory, E_ext, G, Q, nsteps, ckpt_every, dn0_dQ=None):
    """D(t_end) as a differentiable function of (E_ext, G, Q) (float64 tensors)."""
    if dn0_dQ is not None:
        dn0_dQ = np.ascontiguousarray(dn0_dQ, dtype=np.float64)
    return _Deformation.apply(E_ext, G, Q, factory, nsteps, ckpt_every, dn0_dQ)
