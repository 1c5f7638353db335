"""Differentiable actions: torch.autograd.Function wrappers over the C ABI.

Each action of Sec. I / Sec. II is a scalar function of the links U (a
complex128 tensor [V, 4, 3, 3] on the device, canonical order: lexicographic
site, direction mu, row-major 3x3).  Its backward pass is the action's force
kernel (for S_PF: solve, then the outer products projected onto su(3)),
turned into a link gradient by ``hmc_link_gradient``:

    G = 2 F U,   F = sum_a F_a T_a,   (omega, F) = d/d eps S(exp(eps omega) U)

which is the gradient of S in the complex-autograd convention
(dS = Re sum conj(G) dU) restricted to the tangent space of SU(3) at U.  A
finite difference of S along exp(eps omega) U therefore equals
Re sum conj(G) (omega U) to O(eps^2), for any antihermitian traceless omega,
and F = G U^dag / 2 recovers the force.

* ``gauge_action(hctx, L, U, beta, kappa=0, k=0)``: S_G + T_k (Sec. I, the
  Wilson plaquette action, plus the hopping-expansion term of Sec. II for
  k = 1, 2); ``hopexp_action`` is T_k alone (beta = 0).
* ``pf_action(hctx, L, U, phi, kappa, b=None, alpha=0)``: the pseudo-fermion
  action, plain (b None) or filtered |(alpha Mhat^-1 + sum_n b_n K^n) phi|^2
  with the same truncation in the action and its force.  phi (complex
  [Vh, 4, 3], even sites) is not differentiated.

``force_prec`` selects the precision of the backward kernels (F64, or F32
links with FP64 accumulation); the forward action is always FP64.
"""
import torch

from . import hmc as H


def _links(U):
    if not (torch.is_tensor(U) and U.is_complex() and U.dim() == 4 and U.shape[1:] == (4, 3, 3)):
        raise ValueError("U must be a complex tensor [V, 4, 3, 3]")
    return U.detach().to(torch.complex128).contiguous()


def _grad_input(ctx_needs, G):
    return G if ctx_needs else None


class _GaugeAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, hctx, L, beta, kappa, k, force_prec):
        Uc = _links(U)
        U64 = hctx.pack_gauge(L, Uc, H.F64, H.LINK18)
        S = hctx.force_hopexp(L, U64, beta, kappa, k)
        ctx.save_for_backward(Uc)
        ctx.args = (hctx, L, beta, kappa, k, force_prec, U64)
        return torch.tensor(S, dtype=torch.float64, device=Uc.device)

    @staticmethod
    def backward(ctx, g):
        (Uc,) = ctx.saved_tensors
        hctx, L, beta, kappa, k, fp, U64 = ctx.args
        Uf = U64 if fp == H.F64 else hctx.pack_gauge(L, Uc, H.F32, H.LINK12)
        F = hctx.new_algebra(L)
        hctx.force_hopexp(L, Uf, beta, kappa, k, F=F, want_action=False)
        G = hctx.link_gradient(L, Uc, F, float(g))
        return _grad_input(ctx.needs_input_grad[0], G), None, None, None, None, None, None


class _PFAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, phi, hctx, L, kappa, b, alpha, tol, inner_prec, force_prec):
        Uc = _links(U)
        U64 = hctx.pack_gauge(L, Uc, H.F64, H.LINK18)
        Ulo = hctx.pack_gauge(L, Uc, inner_prec, H.LINK12) if inner_prec != H.F64 else None
        ph = hctx.pack_spinor(L, phi.detach() if torch.is_tensor(phi) else phi)
        S = hctx.action_pf(L, U64, ph, kappa, tol=tol, U_lo=Ulo, inner_prec=inner_prec, b=b,
                           alpha=alpha)
        ctx.save_for_backward(Uc)
        ctx.args = (hctx, L, kappa, b, alpha, tol, inner_prec, force_prec, U64, Ulo, ph)
        return torch.tensor(S, dtype=torch.float64, device=Uc.device)

    @staticmethod
    def backward(ctx, g):
        (Uc,) = ctx.saved_tensors
        hctx, L, kappa, b, alpha, tol, inner_prec, fp, U64, Ulo, ph = ctx.args
        F = hctx.new_algebra(L)
        hctx.force_pf(L, U64, ph, kappa, F, coeff=1.0, tol=tol, U_lo=Ulo, inner_prec=inner_prec,
                      b=b, alpha=alpha, force_prec=fp)
        G = hctx.link_gradient(L, Uc, F, float(g))
        return (_grad_input(ctx.needs_input_grad[0], G),) + (None,) * 9


def gauge_action(hctx, L, U, beta, kappa=0.0, k=0, force_prec=H.F64):
    """S_G + T_k as a differentiable scalar (FP64 value on U's device)."""
    return _GaugeAction.apply(U, hctx, tuple(L), float(beta), float(kappa), int(k), force_prec)


def hopexp_action(hctx, L, U, kappa, k, force_prec=H.F64):
    """The hopping-expansion term T_k = 2 sum_{n<=k} (1/n) Tr_e K^n alone."""
    return gauge_action(hctx, L, U, 0.0, kappa, k, force_prec)


def pf_action(hctx, L, U, phi, kappa, b=None, alpha=0.0, tol=1e-12, inner_prec=H.F64,
              force_prec=H.F64):
    """S_PF (plain, or filtered with coefficients b and alpha) as a
    differentiable function of U."""
    return _PFAction.apply(U, phi, hctx, tuple(L), float(kappa), b, float(alpha), float(tol),
                           inner_prec, force_prec)
