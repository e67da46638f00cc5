"""Differentiable likelihood and the maximum-likelihood loop (eq. 1, Sec. III).

``TlrLogLik`` is a ``torch.autograd.Function`` whose forward runs one TLR
likelihood evaluation on the GPU (generation, compression, Cholesky, solve)
and whose backward returns the adjoint gradient computed by the CUDA library
(TLR inverse and the fused regenerate-and-reduce pass).  It is
differentiable in theta only; locations and z are constants.

``fit`` maximises l(theta) with L-BFGS-B over (sigma2, beta, nu) inside
bounds, using the exact (TLR) gradient; a non-positive-definite evaluation
is answered with a large value so that the line search backs off.
"""
from __future__ import annotations

import numpy as np
import torch

from . import tlr as T

DEFAULT_BOUNDS = ((1e-3, 10.0), (1e-3, 5.0), (0.1, 3.0))


class TlrLogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, handle: "T.Handle", z: torch.Tensor):
        th = [float(v) for v in theta.detach().cpu().tolist()]
        handle.factor(th)
        ll, g = handle.loglik_grad(z)
        ctx.save_for_backward(g.to(theta.device, theta.dtype))
        return ll.reshape(()).to(theta.device, theta.dtype)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return gout * g, None, None


def loglik(theta: torch.Tensor, handle: "T.Handle", z: torch.Tensor) -> torch.Tensor:
    """l(theta), differentiable in theta (a float64 tensor of 3)."""
    return TlrLogLik.apply(theta, handle, z)


def fit(handle: "T.Handle", z: torch.Tensor, theta0, bounds=DEFAULT_BOUNDS, maxiter: int = 100,
        ftol: float = 1e-9, gtol: float = 1e-6, history: list | None = None):
    """Maximum-likelihood estimate of theta by L-BFGS-B; returns (theta_hat, l_hat, info)."""
    from scipy.optimize import minimize

    evals = {"n": 0}

    def fg(th):
        evals["n"] += 1
        handle.factor(th)
        ll, g = handle.loglik_grad(z)
        rc, _ = handle.status()
        llv = float(ll.cpu().item())
        gv = g.cpu().numpy().astype(np.float64)
        if rc != T.TLR_OK or not np.isfinite(llv):
            return 1e30, np.zeros(3)
        if history is not None:
            history.append((list(map(float, th)), llv))
        return -llv, -gv

    res = minimize(fg, np.asarray(theta0, dtype=np.float64), jac=True, method="L-BFGS-B", bounds=bounds,
                   options={"maxiter": maxiter, "ftol": ftol, "gtol": gtol, "maxfun": 2 * maxiter})
    return res.x, -res.fun, {"evals": evals["n"], "success": bool(res.success), "message": str(res.message)}
