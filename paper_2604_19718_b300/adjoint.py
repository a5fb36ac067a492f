"""log Z as a differentiable function of the soft codon constraints.

The library's outside pass is the hand-written adjoint of its inside pass, so
one cf_outside after one cf_inside gives the whole gradient of log Z:

* d log Z / d lw[r][s] = p_r(s), the marginal probability that residue r uses
  its s-th codon (paper Eq. marginal-codon; a weight enters as e^{+lw});
* d log Z / d pb[c][c'] = expected number of adjacent residue pairs coded
  (c, c') (the codon-pair factors of Eq. pair-tt enter the same way).

``LogZ`` wraps the two calls in a ``torch.autograd.Function``.
``weight_ascent`` is a gradient form of frequency matching (paper Section "A
simple iterative approach to frequency matching", Algorithm "Naive iterative
algorithm for frequency matching", which instead rescales the multiplicative
bonuses by a ratio of achieved and desired frequencies): ascent on the concave
objective
L(lw) = sum_{r,s} f*[r][s] lw[r][s] - log Z(lw), whose gradient f* - p vanishes
exactly when the codon marginals equal the targets f*.
"""
from __future__ import annotations

import numpy as np
import torch

from . import AMINO_ACIDS, CF_FP32_SCALED, CodonFold

# sense codons per amino acid under the standard genetic code, in the order
# ARNDCQEGHILKMFPSTWYV
CODONS_PER_AA = dict(zip(AMINO_ACIDS, (4, 6, 2, 2, 2, 2, 2, 4, 2, 3, 6, 2, 1, 2, 4, 6, 4, 1, 2, 4)))


def slot_mask(aa: str) -> np.ndarray:
    """(m, 6) bool: slot s of residue r is one of its codons."""
    M = np.array([CODONS_PER_AA[a] for a in aa])
    return np.arange(6)[None, :] < M[:, None]


def frequency_targets(aa: str, logits) -> np.ndarray:
    """Per-residue softmax of ``logits`` over the residue's own codon slots
    (zero on unused slots): target codon frequencies f*."""
    mask = slot_mask(aa)
    z = np.where(mask, np.asarray(logits, dtype=np.float64), -np.inf)
    z = np.exp(z - z.max(axis=1, keepdims=True))
    return z / z.sum(axis=1, keepdims=True)


class LogZ(torch.autograd.Function):
    """logz = LogZ.apply(lw, pb, fold, precision).

    lw: (m, 6) float64 tensor of codon log-weights; pb: (61, 61) float64 tensor
    of codon-pair log-bonuses, or None (= 0).  ``fold`` is a CodonFold holding
    the protein.  Forward: cf_set_weights + cf_inside.  Backward: cf_outside,
    whose codon marginals and pair counts are the gradients.  The fold keeps
    only its latest inside pass, so each forward must be followed by its
    backward before the fold is evaluated again (checked).
    """

    @staticmethod
    def forward(ctx, lw, pb, fold: CodonFold, precision: int = CF_FP32_SCALED):
        lw_h = lw.detach().to("cpu", torch.float64).numpy()
        pb_h = None if pb is None else pb.detach().to("cpu", torch.float64).numpy()
        fold.set_weights(lw_h, pb_h)
        logz = fold.inside(precision)
        fold._evals = getattr(fold, "_evals", 0) + 1
        ctx.fold, ctx.eval_id, ctx.has_pb = fold, fold._evals, pb is not None
        ctx.device = lw.device
        return torch.tensor(logz, dtype=torch.float64, device=lw.device)

    @staticmethod
    def backward(ctx, g):
        fold = ctx.fold
        if fold._evals != ctx.eval_id:
            raise RuntimeError("LogZ.backward: the fold was evaluated again after this forward")
        dev = ctx.device
        cm = torch.zeros((fold.m, 6), dtype=torch.float64, device=dev)
        pg = torch.zeros((61, 61), dtype=torch.float64, device=dev) if ctx.has_pb else None
        fold.outside(pair_prob=False, codon=cm, pair_grad=False if pg is None else pg)
        return g * cm, (g * pg if pg is not None else None), None, None


def log_partition(fold: CodonFold, lw, pb=None, precision: int = CF_FP32_SCALED):
    return LogZ.apply(lw, pb, fold, precision)


def weight_ascent(fold: CodonFold, aa: str, targets, steps: int = 50, lr: float = 1.0, lw0=None, pb=None,
                  precision: int = CF_FP32_SCALED, device="cpu"):
    """``steps`` ascent steps on L(lw) = <f*, lw> - log Z(lw) from lw0 (default 0).

    Each step is one inside and one outside pass.  Returns (lw, history); the
    history holds per step the objective, log Z and the largest
    |f* - p| over valid slots, measured at the weights before the step.
    """
    f_star = torch.as_tensor(np.asarray(targets, dtype=np.float64), device=device)
    mask = torch.as_tensor(slot_mask(aa), device=device)
    lw = torch.zeros((len(aa), 6), dtype=torch.float64, device=device) if lw0 is None else \
        torch.as_tensor(np.asarray(lw0, dtype=np.float64), device=device).clone()
    lw.requires_grad_(True)
    pb_t = None if pb is None else torch.as_tensor(np.asarray(pb, dtype=np.float64), device=device)
    hist = []
    for step in range(steps):
        logz = LogZ.apply(lw, pb_t, fold, precision)
        obj = (f_star * lw).sum() - logz
        (grad,) = torch.autograd.grad(obj, lw)
        gap = float(grad[mask].abs().max())
        hist.append({"step": step, "objective": float(obj.detach()), "logZ": float(logz.detach()), "max_gap": gap})
        with torch.no_grad():
            lw += lr * torch.where(mask, grad, torch.zeros_like(grad))
    return lw.detach(), hist
