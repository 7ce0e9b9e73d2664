"""Differentiable cavity solves: a torch.autograd.Function whose backward is the adjoint solve.

The forward solves K(nu) x = f_lid(theta, nu) + f_body(coef) with the context's preconditioned
Krylov solver. K is symmetric, so the backward solves K lambda = dL/dx through the same path and
returns
  dL/dtheta_k = lambda^T phi_k,   phi_k = Nitsche lid load of the k-th lid B-spline (unit theta),
  dL/dcoef_cm = lambda^T psi_cm,  psi_cm = load of the (c, m) sine mode with unit coefficient,
  dL/dnu      = (lambda^T f_lid - lambda_u^T A x_u) / nu     (A and f_lid are linear in nu).
Objectives must depend on the velocity only (dL/dq = 0): then the adjoint right-hand side is
orthogonal to the constant-pressure null vector of K and the zero-mean pressure shift of the
forward solution does not enter the gradient.
Every load, solve, operator apply and inner product runs in the CUDA library; torch holds the
tensors. nu is a property of the context, so its gradient is reported, not applied.
"""
import numpy as np
import torch


class CavitySolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, coef, nu, G, waves, tol):
        th = theta.detach().cpu().double().numpy()
        cf = coef.detach().cpu().double().numpy()
        if abs(float(nu) - G.nu) > 1e-15 * max(1.0, G.nu):
            raise ValueError("nu must equal the context's viscosity")
        f_lid = G.rhs_lid_profile(th)
        f = f_lid.clone()
        if cf.size:
            G.rhs_body(cf, waves, accumulate=True, out=f)
        x, it, rr, _ = G.solve(f, tol)
        ctx.G, ctx.waves, ctx.tol = G, np.asarray(waves), tol
        ctx.shapes = (th.shape, cf.shape)
        ctx.devices = (theta.device, coef.device,
                       nu.device if isinstance(nu, torch.Tensor) else torch.device("cpu"))
        ctx.save_for_backward(x, f_lid)
        return x

    @staticmethod
    def backward(ctx, gx):
        G = ctx.G
        x, f_lid = ctx.saved_tensors
        g = gx.detach().double().contiguous().clone()
        if bool(g[G.n_vel:].abs().max() > 0):
            raise NotImplementedError("objectives must not depend on the pressure")
        lam, it, rr, _ = G.solve(g, ctx.tol)
        (th_shape, cf_shape) = ctx.shapes
        # lambda against the unit loads, contracted on the device without forming the loads
        grad_theta = G.lid_profile_dots(int(np.prod(th_shape)), lam).reshape(th_shape)
        grad_coef = np.zeros(cf_shape)
        if grad_coef.size:
            grad_coef = G.body_load_dots(ctx.waves, lam).reshape(cf_shape)
        Ax = G.apply_A(x[:G.n_vel].contiguous())
        grad_nu = (G.dot(lam, f_lid) - G.dot(lam[:G.n_vel].contiguous(), Ax)) / G.nu
        d_th, d_cf, d_nu = ctx.devices
        return (torch.from_numpy(grad_theta).to(d_th), torch.from_numpy(grad_coef).to(d_cf),
                torch.tensor(grad_nu, dtype=torch.float64, device=d_nu), None, None, None)


class MassMisfit(torch.autograd.Function):
    """J = 1/2 (u - u_t)^T M_V (u - u_t) on the velocity part of x (M_V: velocity mass)."""

    @staticmethod
    def forward(ctx, x, u_target, G):
        e = (x[:G.n_vel] - u_target).contiguous()
        Me = G.apply_mass(e)
        ctx.G, ctx.size = G, x.numel()
        ctx.save_for_backward(Me)
        return torch.tensor(0.5 * G.dot(e, Me), dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, gJ):
        (Me,) = ctx.saved_tensors
        G = ctx.G
        gx = torch.zeros(ctx.size, dtype=torch.float64, device=Me.device)
        gx[:G.n_vel] = gJ * Me
        return gx, -gJ * Me, None


def cavity_solve(G, theta, coef, nu, waves, tol=1e-10):
    """Differentiable x(theta, coef, nu) (see CavitySolve)."""
    return CavitySolve.apply(theta, coef, nu, G, waves, tol)


def mass_misfit(G, x, u_target):
    return MassMisfit.apply(x, u_target, G)
