"""Differentiable compliance f(rho, u) = u^T K(rho) u on a device-resident mesh.

Forward: the sensitivity kernels' c = sum_e E(rho_e) u_e^T K_e^0 u_e (Sec. 2.2).
Backward: the hand-written adjoint soptx_compliance_vjp -- the rho-gradient
g E'(rho_e) u_e^T K_e^0 u_e and the u-gradient 2 g K(rho) u.  With u an
independent input the rho-gradient is +E' s_e, i.e. minus the compliance
sensitivity dc_e that Appendix D writes for the displacement solving K u = F.
"""
import torch


class Compliance(torch.autograd.Function):
    """c = Compliance.apply(rho, u, mesh) -> 0-d float64 tensor."""

    @staticmethod
    def forward(ctx, rho, u, mesh):
        rho = rho.detach().contiguous()
        u = u.detach().contiguous()
        _, c = mesh.sensitivity(rho, u)
        ctx.mesh = mesh
        ctx.save_for_backward(rho, u)
        return c.reshape(())

    @staticmethod
    def backward(ctx, gout):
        rho, u = ctx.saved_tensors
        g = gout.detach().to(torch.float64).reshape(1).contiguous()
        grad_rho, grad_u = ctx.mesh.compliance_vjp(rho, u, g, want_u=ctx.needs_input_grad[1])
        return (grad_rho if ctx.needs_input_grad[0] else None), grad_u, None


def compliance(rho, u, mesh):
    return Compliance.apply(rho, u, mesh)
