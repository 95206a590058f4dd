"""torch.autograd.Function around the ladder energy.

E_L(B, tau, t2) = sum_ijab R_ij^ab (2 t2_ij^ab - t2_ij^ba) with R the ladder
term of (B, tau).  Forward: ladder_apply + ladder_energy.  Backward, with
W = 2 t2 - t2^T (ladder_pair_combine):
    dE/dtau = transposed ladder of W           (ladder_backward)
    dE/dB   = 2 sum Gamma B, Gamma = W^T tau    (ladder_backward)
    dE/dt2  = 2 R - R^T                         (ladder_pair_combine)
Both ladder_backward terms run in the mode of the plan that serves the
backward: the forward plan itself (FP64, BF16X3 or BF16X6), or a separate
`grad_ladder`.  The error-free mode has no dE/dB of its own, so an
error-free forward plan (E_L and R to FP64 class) takes a BF16X6 or FP64
grad_ladder created with backward=True for dE/dB; when that forward plan
has sym_b (B symmetric in a <-> c), the transposed ladder is the ladder
itself and dE/dtau comes from the forward plan, error-free, instead.
dE/dt2 comes from the forward's R.
All arithmetic runs in the library's kernels; the incoming gradient (a
scalar) is applied with an in-place multiply.
"""
from __future__ import annotations

import torch

from . import LADDER_OZAKI, Ladder, ladder_get_tuning, ladder_pair_combine


def _error_free_symmetric(L: Ladder) -> bool:
    return L.mode == LADDER_OZAKI and ladder_get_tuning(L.plan).sym_b == 1


class LadderEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, B, tau, t2, ladder: Ladder, grad_ladder=None):
        R = ladder.apply(B, tau)
        E = ladder.energy(R, t2)
        ctx.save_for_backward(B, tau, t2, R)
        ctx.ladder = ladder if grad_ladder is None else grad_ladder
        # an error-free forward with symmetric B serves dE/dtau itself
        ctx.tau_ladder = ladder if _error_free_symmetric(ladder) else ctx.ladder
        return E

    @staticmethod
    def backward(ctx, gE):
        B, tau, t2, R = ctx.saved_tensors
        L, Lt = ctx.ladder, ctx.tau_ladder
        need_B, need_tau, need_t2 = ctx.needs_input_grad[:3]
        dB = dtau = dt2 = None
        if need_B or need_tau:
            W = L.weights(t2)
            if Lt is L:
                dtau, dB = L.backward(B, tau, W, dtau=bool(need_tau), dB=bool(need_B))
            else:
                if need_tau:
                    dtau, _ = Lt.backward(B, tau, W, dtau=True, dB=False)
                if need_B:
                    _, dB = L.backward(B, tau, W, dtau=False, dB=True)
        if need_t2:
            dt2 = torch.empty_like(t2)
            ladder_pair_combine(L.o, L.v, 2.0, -1.0, R, dt2)
        g = gE.to(torch.float64)
        for t in (dB, dtau, dt2):
            if t is not None:
                t.mul_(g)
        return dB, dtau, dt2, None, None


def ladder_energy(B, tau, t2, ladder: Ladder, grad_ladder: Ladder = None):
    """Differentiable E_L(B, tau, t2) computed by `ladder` (a Ladder plan;
    create it with backward=True when it serves the backward too).
    grad_ladder: a plan of the same shape with backward=True that serves the
    backward instead, e.g. BF16X6 behind an error-free forward."""
    if grad_ladder is not None and (grad_ladder.o, grad_ladder.v, grad_ladder.naux) != (
            ladder.o, ladder.v, ladder.naux):
        raise ValueError("grad_ladder has another shape than ladder")
    return LadderEnergy.apply(B, tau, t2, ladder, grad_ladder)
