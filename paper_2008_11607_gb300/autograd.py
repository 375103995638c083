"""torch.autograd bindings of the REXII step: gradients with respect to the
state (the adjoint step, rexi_step_adjoint) and to the depth field
(rexi_step_grad_depth), and a multi-step rollout that stores only every
`every`-th state and recomputes the others during the backward pass.

Argument marshalling only: the forward, adjoint and depth-gradient work all
runs in librexi.  PyTorch's gradient of a real loss with respect to a complex
tensor is dL/dRe + i dL/dIm, the convention the library's adjoint uses.
"""
import torch


class RexiStep(torch.autograd.Function):
    """out = r(dt A(H)) state.  `depth` must be the tensor the plan was built on
    (variable-depth plans) or None; its gradient is returned when required."""

    @staticmethod
    def forward(ctx, state, depth, plan, dt, tol, real_input):
        out = plan.step(state.contiguous(), dt, tol=tol, real_input=real_input)
        ctx.save_for_backward(state)
        ctx.plan, ctx.dt, ctx.tol, ctx.real_input = plan, dt, tol, real_input
        ctx.has_depth = depth is not None
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (state,) = ctx.saved_tensors
        plan, dt, tol, real = ctx.plan, ctx.dt, ctx.tol, ctx.real_input
        g = grad_out.contiguous()
        grad_state = plan.step_adjoint(g, dt, tol=tol, real_input=real) if ctx.needs_input_grad[0] else None
        grad_depth = None
        if ctx.has_depth and ctx.needs_input_grad[1]:
            grad_depth = plan.grad_depth(state.contiguous(), g, dt, tol=tol, real_input=real)
        return grad_state, grad_depth, None, None, None, None


def rexi_step(state, plan, dt, depth=None, tol=1e-10, real_input=True):
    return RexiStep.apply(state, depth, plan, dt, tol, real_input)


class RexiRollout(torch.autograd.Function):
    """`nsteps` REXII steps.  Keeps the states at steps 0, every, 2 every, ... and
    recomputes the states inside each segment in the backward pass, then runs
    the adjoint (and depth-gradient) steps backwards through the segment."""

    @staticmethod
    def forward(ctx, state0, depth, plan, dt, nsteps, every, tol, real_input):
        s = state0.contiguous()
        ckpts = [s]
        for k in range(1, nsteps + 1):
            s = plan.step(s, dt, tol=tol, real_input=real_input)
            if k % every == 0 and k < nsteps:
                ckpts.append(s)
        ctx.save_for_backward(*ckpts)
        ctx.plan, ctx.dt, ctx.nsteps, ctx.every, ctx.tol, ctx.real_input = plan, dt, nsteps, every, tol, real_input
        ctx.has_depth = depth is not None
        return s

    @staticmethod
    def backward(ctx, grad_T):
        ckpts = ctx.saved_tensors
        plan, dt, tol, real = ctx.plan, ctx.dt, ctx.tol, ctx.real_input
        want_depth = ctx.has_depth and ctx.needs_input_grad[1]
        g = grad_T.contiguous()
        grad_depth = None
        if want_depth:
            grad_depth = torch.zeros((plan.ny, plan.nx), dtype=torch.float64, device=g.device)
        ws = None
        for seg in reversed(range(len(ckpts))):
            first = seg * ctx.every
            last = min(first + ctx.every, ctx.nsteps)
            states = [ckpts[seg]]
            for _ in range(first, last - 1):  # recompute the states inside the segment
                states.append(plan.step(states[-1], dt, tol=tol, real_input=real))
            for j in reversed(range(last - first)):
                if want_depth:
                    plan.grad_depth(states[j], g, dt, tol=tol, real_input=real, grad=grad_depth, workspace=ws)
                g = plan.step_adjoint(g, dt, tol=tol, real_input=real)
        return g, grad_depth, None, None, None, None, None, None


def rexi_rollout(state0, plan, dt, nsteps, every=2, depth=None, tol=1e-10, real_input=True):
    return RexiRollout.apply(state0, depth, plan, dt, nsteps, every, tol, real_input)
