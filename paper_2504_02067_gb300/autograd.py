"""The entropic OT value as a differentiable torch function.

Forward: eot_solve (Alg. 1) to the potentials (u, v) at gamma_f, then eot_value,
which returns on the device
    F* = (<r, u> + <c, v> - sum P + 1) / gamma_f,
the dual value at (u, v). At the optimum it equals the primal value
<P*, C> - H(P*) / gamma_f with H(P) = -sum P log P (strong duality, Sec. 2.1),
and it is stationary in (u, v), so potentials solved to a marginal tolerance
give it to second order in that tolerance.

Backward: eot_backward at the saved potentials (envelope theorem on the
Lagrangian, Appx. A; s_C held constant):
    dC = P,   dx_i = 2 s_C sum_j P_ij (x_i - y_j),   dy_j = 2 s_C sum_i P_ij (y_j - x_i),
    dr = u / gamma_f,   dc = v / gamma_f,
each scaled by the incoming gradient, which eot_backward reads on the device
(no host synchronisation). The gradients with respect to r and c are defined up
to a constant vector (only simplex-tangent directions are admissible).

All arithmetic runs in libeot.so; this module only marshals tensors.
"""
import torch

from .binding import Problem, default_params


class EOTFunction(torch.autograd.Function):
    """value = EOTFunction.apply(handle, C, X, Y, r, c, params, precision, cost_scale)

    Dense problems pass C (FP32 for "mixed" / "plain_fp32", FP64 for "fp64") and
    X = Y = None; point problems pass C = None and FP32 X [n, d], Y [m, d].
    r, c: FP64 marginals. params: an EotParams (gamma_f is the temperature of the
    value). cost_scale: s_C for point costs (<= 0: computed by the library, and
    still held constant in the backward)."""

    @staticmethod
    def forward(ctx, handle, C, X, Y, r, c, params, precision, cost_scale):
        prob = Problem(C=C, X=X, Y=Y, r=r, c=c, precision=precision, cost_scale=cost_scale)
        u, v, stats = handle.solve(prob, params)
        gamma = float(params.gamma_f)
        value = torch.empty((), dtype=torch.float64, device=u.device)
        handle.eot_value(prob, u, v, gamma, value)
        ctx.handle, ctx.prob, ctx.gamma, ctx.stats = handle, prob, gamma, stats
        ctx.save_for_backward(u, v)
        ctx.mark_non_differentiable(u, v)
        return value, u, v

    @staticmethod
    def backward(ctx, g_value, g_u, g_v):
        u, v = ctx.saved_tensors
        need = ctx.needs_input_grad
        prob = ctx.prob
        dev = u.device
        dC = dX = dY = dr = dc = None
        if need[1] and prob.C is not None:
            dC = torch.empty(prob.n, prob.m, dtype=torch.float32, device=dev)
        if need[2] and prob.X is not None:
            dX = torch.empty(prob.n, prob.d, dtype=torch.float32, device=dev)
        if need[3] and prob.Y is not None:
            dY = torch.empty(prob.m, prob.d, dtype=torch.float32, device=dev)
        if need[4]:
            dr = torch.empty(prob.n, dtype=torch.float64, device=dev)
        if need[5]:
            dc = torch.empty(prob.m, dtype=torch.float64, device=dev)
        if g_value is None:
            g_value = torch.zeros((), dtype=torch.float64, device=dev)
        g = g_value.detach().to(device=dev, dtype=torch.float64).contiguous()
        ctx.handle.eot_backward(prob, u, v, ctx.gamma, 1.0, dC=dC, dX=dX, dY=dY, dr=dr, dc=dc,
                                grad_scale_dev=g)
        if dC is not None and prob.C is not None and prob.C.dtype != torch.float32:
            dC = dC.to(prob.C.dtype)
        return None, dC, dX, dY, dr, dc, None, None, None


def eot_value(handle, r, c, C=None, X=None, Y=None, precision="mixed", cost_scale=0.0,
              params=None, **overrides):
    """F* at gamma_f with autograd support; returns (value, u, v)."""
    if params is None:
        params = default_params(**overrides)
    return EOTFunction.apply(handle, C, X, Y, r, c, params, precision, cost_scale)
