"""torch.autograd.Function over the C ABI: the smoothed dual evaluation and its adjoint.

``SmoothedDual.apply(solver, terms, nu)`` evaluates, on the GPU, Q_beta per instance and the
gradient g (message layout) at the multipliers ``nu`` (Sec. 4.1.2 soft-min dual, Sec. 4.2),
for the term matrices ``terms``; its backward runs the adjoint kernel (lrh_vjp), which
recomputes the eigenbasis of every region and propagates the cotangents of Q_beta and g to
the multipliers and the term matrices.  Derivatives with respect to couplings follow by
building ``terms`` from them with torch operations; unrolled iterations follow by composing
the function with torch arithmetic for the message update.

Shapes: terms complex128 (n_instances, term_total) (any device), nu complex64
(n_instances, msg_elems) on the solver's device.  Returns q float64 (n_instances,) and g
complex64 (n_instances, msg_elems).
"""
from __future__ import annotations

import numpy as np
import torch


class SmoothedDual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, terms, nu):
        _set_point(solver, terms, nu)
        solver.evaluate()
        q = torch.from_numpy(solver.bound("last")).to(nu.device)
        g = torch.empty_like(nu)
        solver.messages("grad", out=g)
        ctx.solver = solver
        ctx.save_for_backward(terms, nu)
        return q, g

    @staticmethod
    def backward(ctx, q_bar, g_bar):
        terms, nu = ctx.saved_tensors
        s = ctx.solver
        _set_point(s, terms, nu)
        gb = g_bar.to(torch.complex64).contiguous() if g_bar is not None else None
        qb = q_bar if q_bar is not None else torch.zeros(s.n_instances, dtype=torch.float64)
        nu_bar, term_bar = s.vjp_device(qb, gb)
        return None, term_bar.to(terms.dtype).to(terms.device), nu_bar.to(nu.dtype)


def _set_point(solver, terms, nu):
    flat = torch.view_as_real(terms.detach().to(torch.complex128).cpu().contiguous()).numpy().reshape(-1)
    solver.set_terms(np.ascontiguousarray(flat))
    solver.set_messages("nu", nu.detach().to(torch.complex64).contiguous())
    solver.restart()      # theta = 1, zeta = nu: the evaluation point eta is nu itself


def smoothed_dual(solver, terms, nu):
    return SmoothedDual.apply(solver, terms, nu)
