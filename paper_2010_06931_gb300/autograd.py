"""torch.autograd over the registration objective (Eq. 1-10).

``objective(problem, level, disp)`` returns f as a 0-d float64 tensor on the
displacement's device; ``f.backward()`` yields df/dD in ``disp.grad``.  Both
directions run the library's kernels (``octmc_eval_objective_grad``):

* ``mode="save"`` evaluates f and the gradient in the forward pass and keeps
  the gradient (6 w h float64) for the backward pass;
* ``mode="recompute"`` keeps only the displacement and evaluates again in
  the backward pass (the interpolation weights are recomputed, nothing of
  size w h d or w h is stored between the passes).

``batch_objective`` sums several independent pairs with one batched
evaluation (``octmc_eval_batch``) per pass.

The objective is not differentiable twice through this function (the
backward pass is not itself tracked).
"""
import torch

__all__ = ["ObjectiveFunction", "BatchObjectiveFunction", "objective", "batch_objective"]


class ObjectiveFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, disp, problem, level, mode):
        disp = disp.detach()
        if mode == "save":
            g = torch.empty_like(disp)
            f = problem.eval_objective_grad(level, disp, g)
            ctx.save_for_backward(g)
        elif mode == "recompute":
            f = problem.eval_objective_grad(level, disp, None)
            ctx.save_for_backward(disp)
        else:
            raise ValueError("mode must be 'save' or 'recompute'")
        ctx.problem, ctx.level, ctx.mode = problem, level, mode
        return torch.tensor(f, dtype=torch.float64, device=disp.device)

    @staticmethod
    def backward(ctx, grad_out):
        (saved,) = ctx.saved_tensors
        if ctx.mode == "save":
            g = saved
        else:
            g = torch.empty_like(saved)
            ctx.problem.eval_objective_grad(ctx.level, saved, g)
        return grad_out.to(g.dtype) * g, None, None, None


def objective(problem, level, disp, mode="save"):
    """f(D) of ``problem`` at pyramid ``level`` as a differentiable tensor."""
    return ObjectiveFunction.apply(disp, problem, level, mode)


class BatchObjectiveFunction(torch.autograd.Function):
    """Sum of the objectives of several independent pairs, each pass one
    batched evaluation of all of them (``octmc_eval_batch``: one launch per
    kernel for the whole batch)."""

    @staticmethod
    def forward(ctx, problems, level, mode, *disps):
        from . import eval_batch
        disps = [D.detach() for D in disps]
        levels = [level] * len(disps)
        if mode == "save":
            grads = [torch.empty_like(D) for D in disps]
            fs = eval_batch(problems, levels, disps, grads)
            ctx.save_for_backward(*grads)
        elif mode == "recompute":
            fs = eval_batch(problems, levels, disps, None)
            ctx.save_for_backward(*disps)
        else:
            raise ValueError("mode must be 'save' or 'recompute'")
        ctx.problems, ctx.level, ctx.mode = problems, level, mode
        return torch.tensor(sum(fs), dtype=torch.float64, device=disps[0].device)

    @staticmethod
    def backward(ctx, grad_out):
        from . import eval_batch
        saved = ctx.saved_tensors
        if ctx.mode == "save":
            grads = list(saved)
        else:
            grads = [torch.empty_like(D) for D in saved]
            eval_batch(ctx.problems, [ctx.level] * len(saved), list(saved), grads)
        return (None, None, None) + tuple(grad_out.to(g.dtype) * g for g in grads)


def batch_objective(problems, level, disps, mode="recompute"):
    """Sum of the objectives of several independent pairs (one displacement
    tensor per problem) from one batched evaluation per pass; its backward
    fills each tensor's ``grad``."""
    return BatchObjectiveFunction.apply(list(problems), level, mode, *disps)
