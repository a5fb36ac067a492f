"""Frequency matching: per-codon multiplicative bonuses f for which the
expected codon counts of the design distribution equal target counts (paper
Section "A simple iterative approach to frequency matching", Algorithm
"Naive iterative algorithm for frequency matching"), with the fixed-point
iteration accelerated by Anderson mixing (type II, depth ``depth``).

Counts rather than normalised frequencies: for a codon c,
  b(c)  = sum over residues r of p_r(c), the codon marginals of the current
          bonuses (cf_outside), and
  b*(c) = sum over residues r coding c's amino acid of f*(c) / sum_{c' in
          C(psi_r)} f*(c'), the counts of independent per-residue draws
          weighted by the target bonuses f* (the algorithm's b*).
Both sum to the protein length.  The iteration works on x = log f (one entry
per sense codon of the protein, bonus e^{x} on every slot holding that codon,
starting from x = log f*) and the residual F(x) = log b*(c) - log b(c): the
naive step is x <- x + F(x), i.e. the bonus is multiplied by desired /
achieved (the printed algorithm writes the ratio the other way round; only
this direction moves b towards b*), and it stops when max |F| < r_tol.

Each evaluation of b is one inside and one outside pass through the library;
the marginals come from a callable so that the same driver runs against the
oracle in the tests.
"""
from __future__ import annotations

from typing import Callable

import numpy as np

from . import AMINO_ACIDS, CF_FP32_SCALED, CodonFold

# the standard genetic code over codons in lexicographic order of the bases
# A, C, G, U (64 entries, '*' = stop); sense codon ids skip the stops
STANDARD_CODE = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF"
N_SENSE = 61


def _sense_ids_by_aa() -> dict:
    out, sid = {a: [] for a in AMINO_ACIDS}, 0
    for c in range(64):
        if STANDARD_CODE[c] == "*":
            continue
        out[STANDARD_CODE[c]].append(sid)
        sid += 1
    return out


_SENSE_BY_AA = _sense_ids_by_aa()


def slot_codon_ids(aa: str) -> np.ndarray:
    """(m, 6) sense codon id of each residue's codon slot (slots in codon-id
    order, as in the library's codon_logw), -1 for unused slots."""
    out = -np.ones((len(aa), 6), dtype=np.int64)
    for r, a in enumerate(aa):
        ids = _SENSE_BY_AA[a]
        out[r, :len(ids)] = ids
    return out


def target_counts(aa: str, fstar) -> np.ndarray:
    """b*: expected count of each sense codon when every residue draws its
    codon independently with probability proportional to f* (61 bonuses)."""
    f = np.asarray(fstar, dtype=np.float64)
    ids = slot_codon_ids(aa)
    b = np.zeros(N_SENSE)
    for r in range(len(aa)):
        row = ids[r][ids[r] >= 0]
        w = f[row]
        b[row] += w / w.sum()
    return b


def codon_counts(aa: str, codon_marg) -> np.ndarray:
    """b: expected count of each sense codon from the codon marginals (m, 6)."""
    ids = slot_codon_ids(aa)
    cm = np.asarray(codon_marg, dtype=np.float64)
    b = np.zeros(N_SENSE)
    mask = ids >= 0
    np.add.at(b, ids[mask], cm[mask])
    return b


def slot_weights(aa: str, x) -> np.ndarray:
    """codon_logw (m, 6) carrying the per-codon log-bonus x (61) on every slot."""
    ids = slot_codon_ids(aa)
    xv = np.asarray(x, dtype=np.float64)
    return np.where(ids >= 0, xv[np.maximum(ids, 0)], 0.0)


def fold_marginals(fold: CodonFold, pair_bonus=None, precision: int = CF_FP32_SCALED) -> Callable:
    """Marginal provider for ``match_frequencies``: new weights, one inside and
    one outside pass of the library, the codon marginals (m, 6)."""

    def marginals(codon_logw):
        fold.set_weights(codon_logw, pair_bonus)
        fold.inside(precision)
        return fold.outside(pair_prob=False, codon=True, pair_grad=False)[1]

    return marginals


def match_frequencies(marginals: Callable, aa: str, fstar, rtol: float = 0.002, max_iter: int = 100,
                      depth: int = 5):
    """Bonuses matching the target counts of ``fstar``.  Returns (x, history):
    x the per-codon log-bonuses (61; codons absent from the protein keep
    log f*), history per evaluation the largest |log(b*/b)| over the codons of
    the protein.  depth = 0 is the naive iteration."""
    bstar = target_counts(aa, fstar)
    act = np.flatnonzero(bstar > 0)
    x = np.log(np.asarray(fstar, dtype=np.float64))
    xs, fs, hist = [], [], []
    for _ in range(max_iter):
        b = codon_counts(aa, marginals(slot_weights(aa, x)))
        F = np.log(bstar[act]) - np.log(b[act])
        hist.append(float(np.abs(F).max()))
        if hist[-1] < rtol:
            break
        xa = x[act].copy()
        xs.append(xa)
        fs.append(F)
        if depth > 0 and len(fs) > 1:
            k = min(depth, len(fs) - 1)
            dF = np.stack([fs[-i] - fs[-i - 1] for i in range(1, k + 1)], axis=1)
            dX = np.stack([xs[-i] - xs[-i - 1] for i in range(1, k + 1)], axis=1)
            gamma = np.linalg.lstsq(dF, F, rcond=None)[0]
            xa = xa + F - (dX + dF) @ gamma
        else:
            xa = xa + F
        x = x.copy()
        x[act] = xa
        if len(xs) > depth + 1:
            xs.pop(0)
            fs.pop(0)
    return x, hist
