"""The fermion force as the adjoint of the pseudofermion action in torch.autograd.

Section 2 of the paper: the HMC force of S_F = phi^dag (M^dag M)^-1 phi is
dS_F/dU = -phi^dag K^-1 (dK/dU) K^-1 phi.  Here S is a function of the link
algebra: w = (w_a(x, mu)) moves every link as U_mu(x) -> exp(i w_a T_a) U_mu(x),
and dS/dw at w = 0 is the force in the library's convention.  `PFAction`
evaluates S at the current links (forward, one solve through the C ABI,
keeping only X = A^-1 psi and Y = M_hat X) and returns dS/dw by the
hand-written outer-product kernel (backward, no solve; the polynomial-term
vectors are recomputed).  Argument marshalling only: every step runs in the
CUDA library.

Usage:
    w = torch.zeros(lat.algebra_field().numel(), dtype=torch.float64,
                    device="cuda", requires_grad=True)
    S = pf_action(w, lat, term, phi, params)      # scalar tensor
    S.backward()                                  # w.grad = dS/dw = the force
"""
import torch

from . import wdhmc as wd


class PFAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, lat, term, phi, params, force_prec):
        if w.numel() != 64 * lat.Vh:
            raise ValueError("w must be an algebra field of the lattice (64 * Vh reals)")
        if bool(torch.count_nonzero(w)):
            raise ValueError("w is the tangent at the current links: evaluate at w = 0")
        X, Y = lat.half_spinor(zero=False), lat.half_spinor(zero=False)
        S = lat.pf_action_xy(term, phi, params, X, Y)
        ctx.save_for_backward(X, Y)
        ctx.lat, ctx.term, ctx.phi, ctx.force_prec = lat, term, phi, force_prec
        return torch.tensor(S, dtype=torch.float64, device=w.device)

    @staticmethod
    def backward(ctx, gS):
        X, Y = ctx.saved_tensors
        lat = ctx.lat
        F = lat.algebra_field()
        kind = ctx.term.kind
        lat.fermion_force_xy(ctx.term, ctx.phi, None if kind in (wd.POLY, wd.RATIO) else X,
                             Y if kind in (wd.PLAIN, wd.HASENBUSCH) else None, ctx.force_prec,
                             float(gS), F)
        return F, None, None, None, None, None


def pf_action(w, lat, term, phi, params, force_prec=wd.F64):
    """S(exp(i w . T) U) at w = 0, differentiable in w through the force kernel."""
    return PFAction.apply(w, lat, term, phi, params, force_prec)
