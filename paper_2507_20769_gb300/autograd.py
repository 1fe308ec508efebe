"""torch.autograd.Function for the point value and gradient at c.

forward(x) launches the library's point-gradient kernel (round-to-nearest value
and reverse-mode gradient of every output, same local partials as the interval
rules) on the current stream and keeps the gradient; backward multiplies it by
the incoming gradient. Section 3.2: derivative information of the objective and
constraints feeds the Mean Value Form; this exposes the point form to torch.
"""
from __future__ import annotations

import torch

from .ivb import Problem


class IvbPointGrad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, problem: Problem):
        if x.dtype != torch.float64 or not x.is_cuda:
            raise TypeError("x must be a float64 CUDA tensor [n_points, n_vars]")
        f, g = problem.ivb_point_grad(x.detach().contiguous())
        ctx.save_for_backward(g)
        return f

    @staticmethod
    def backward(ctx, grad_f: torch.Tensor):
        (g,) = ctx.saved_tensors
        # d/dx sum_o grad_f[p, o] f_o(x_p) = sum_o grad_f[p, o] * g[p, o, :]
        return torch.einsum("po,poi->pi", grad_f.to(g.dtype), g), None


def point_values(problem: Problem, x: torch.Tensor) -> torch.Tensor:
    """f(x) for every output, differentiable with respect to x"""
    return IvbPointGrad.apply(x, problem)
