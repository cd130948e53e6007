"""The misfit as a differentiable function of eps_r (Section 5).

``MisfitGrad.apply(eps, problem, tx, rx, S_meas, w)`` returns J (Eq. defJ) as a
float64 tensor.  Forward: re-assemble and re-factorise for eps, solve the
state problems, take the misfit.  Backward: the adjoint solve with the same
operator and factors and the per-tet gradient kernel; the gradient of a real
loss with respect to a complex eps follows PyTorch's convention,
dJ/dRe(eps) + i dJ/dIm(eps).

``lbfgs_invert`` runs the paper's quasi-Newton reconstruction loop (L-BFGS,
Section 5 and Section 6.3) over (Re eps, Im eps).
"""

import numpy as np
import torch


class MisfitGrad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, problem, tx, rx, S_meas, w=None):
        e = eps.detach().to(torch.complex128).contiguous()
        if e.is_cuda:
            problem.update_eps(e)
        else:
            problem.update_eps(e.numpy())
        S = problem.forward_solve(tx, rx)
        J = problem.misfit(S_meas, w)
        ctx.problem = problem
        ctx.S_meas = S_meas
        ctx.w = w
        ctx.device = eps.device
        ctx.S = S
        return torch.tensor(J, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_out):
        J, grad = ctx.problem.misfit_and_gradient(ctx.S_meas, ctx.w)
        g = torch.from_numpy(grad).to(ctx.device)
        return grad_out.to(torch.complex128) * g, None, None, None, None, None


def lbfgs_invert(problem, eps0, tx, rx, S_meas, w=None, iters=10, lr=1.0, history=10, callback=None):
    """Minimise J over eps with torch.optim.LBFGS (strong-Wolfe line search).

    Returns the reconstructed eps (complex128 numpy) and the list of J values
    of every function evaluation.  A problem created with recycle=1 starts every
    evaluation's forward and adjoint solves from the span of the previous
    evaluation's solutions (fewer iterations, same tolerance).
    """
    x = torch.from_numpy(np.stack([np.real(eps0), np.imag(eps0)]).astype(np.float64)).requires_grad_(True)
    opt = torch.optim.LBFGS([x], lr=lr, max_iter=iters, history_size=history, line_search_fn="strong_wolfe",
                            tolerance_grad=0.0, tolerance_change=0.0)
    values = []

    def closure():
        opt.zero_grad()
        eps = torch.complex(x[0], x[1])
        J = MisfitGrad.apply(eps, problem, tx, rx, S_meas, w)
        J.backward()
        values.append(float(J.detach()))
        if callback:
            callback(len(values), values[-1])
        return J

    opt.step(closure)
    out = x.detach().numpy()
    return out[0] + 1j * out[1], values


def normalised_weights(problem, eps_empty, tx, rx):
    """Weights w_ij = 1 / |S^empty_ij|^2 of the normalised misfit (Eq. defJ2),
    from one forward solve of the empty (gel-filled) chamber eps_empty [nt];
    the library forms them (mwi_normalised_weights)."""
    from . import mwi
    problem.update_eps(eps_empty)
    return mwi.normalised_weights(problem.forward_solve(tx, rx))


def p1_objective(problem, kappa, tx, rx, S_meas, w=None, alpha=0.0):
    """Phi(kappa) = J(kappa) + (alpha/2) integral |grad kappa|^2 (Eq. defJ2) for a
    per-vertex permittivity kappa (device tensor [nv]; the piecewise-linear
    parameter of Section 6.3, varying inside every tet in the mass term), with
    its gradient dPhi/dRe kappa + i dPhi/dIm kappa as a device tensor [nv]."""
    problem.update_kappa(kappa)
    problem.forward_solve(tx, rx)
    J, R, g = problem.misfit_and_gradient_kappa(S_meas, w, alpha)
    return J + R, g
