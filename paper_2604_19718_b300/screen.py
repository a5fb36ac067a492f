"""Window labelling, surrogate training and surrogate pre-screening.

* ``Windows`` scores windows exactly: G = -RT ln Z from cf_window_logz (the
  structure-only partition function of a fixed sequence).
* ``train`` fits the surrogate (cf_surrogate_train_step) to exact labels.
* ``prescreen`` designs one window: it draws candidate codon choices for the
  window's residues, ranks them by the surrogate's predicted G and re-scores
  the best ``top`` exactly; ``dp_only`` is the method without the surrogate
  (random candidates, all scored exactly).  Lower G = more stable, the
  objective of the design step.

Candidates come either uniformly per residue or from the exact sampler of the
codon-constrained ensemble (paper Section "Sequence sampling"), restricted to
the window's residues.
"""
from __future__ import annotations

import time

import numpy as np

from . import (AMINO_ACIDS, CodonFold, cf_load_model, cf_model_free, cf_problem_create, cf_problem_free,
               cf_window_last_ms, cf_window_logz)

# Standard genetic code over codons in lexicographic A, C, G, U order.
_CODE = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF"
CODONS = [[(c >> 4 & 3, c >> 2 & 3, c & 3) for c in range(64) if _CODE[c] == a] for a in AMINO_ACIDS]


_TABLE = np.zeros((20, 6, 3), dtype=np.uint8)
for _r, _cods in enumerate(CODONS):
    for _s, _trip in enumerate(_cods):
        _TABLE[_r, _s] = _trip


def gas_constant_kT(params) -> float:
    """RT in kcal/mol at the model's temperature (parameter 180, Celsius)."""
    return 1.98717e-3 * (float(params[180]) + 273.15)


def bases_of(residues, slots) -> np.ndarray:
    """Bases (uint8) of a codon choice: slot s of residue r is CODONS[r][s]."""
    return _TABLE[np.asarray(residues), np.asarray(slots)].ravel()


class Windows:
    """Exact window free energies on one device."""

    def __init__(self, params, device: int = 0, stream: int = 0):
        self.kT = gas_constant_kT(params)
        self.model = cf_load_model(params)
        self.prob = cf_problem_create(self.model, device, stream)

    def logz(self, bases, offsets) -> np.ndarray:
        out = np.zeros(len(offsets) - 1)
        cf_window_logz(self.prob, np.ascontiguousarray(bases, dtype=np.uint8),
                       np.ascontiguousarray(offsets, dtype=np.int64), out)
        return out

    def free_energy(self, bases, offsets) -> np.ndarray:
        return -self.kT * self.logz(bases, offsets)

    def last_ms(self) -> float:
        return cf_window_last_ms(self.prob)

    def close(self):
        if self.prob:
            cf_problem_free(self.prob)
            self.prob = None
        if self.model:
            cf_model_free(self.model)
            self.model = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batches(offsets, batch: int, rng):
    """Window indices in shuffled batches."""
    idx = rng.permutation(len(offsets) - 1)
    for i in range(0, len(idx), batch):
        yield idx[i:i + batch]


def gather(bases, offsets, idx):
    """Concatenate the windows ``idx`` into (bases, offsets)."""
    lens = offsets[idx + 1] - offsets[idx]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    out = np.concatenate([bases[offsets[i]:offsets[i + 1]] for i in idx]) if len(idx) else np.zeros(0, np.uint8)
    return out.astype(np.uint8), off


def train(sur, bases, offsets, G, epochs: int = 4, batch: int = 512, lr: float = 2e-3, seed: int = 0,
          log=None):
    """Adam on the surrogate over ``epochs`` passes; returns per-epoch mean loss."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        tot, cnt = 0.0, 0
        lr_ep = lr * (0.5 ** ep)
        for idx in batches(offsets, batch, rng):
            b, o = gather(bases, offsets, idx)
            tot += sur.train_step(b, o, G[idx], lr_ep) * len(idx)
            cnt += len(idx)
        hist.append(tot / cnt)
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.5f}")
    return hist


def uniform_candidates(residues, ncand: int, rng) -> np.ndarray:
    """ncand codon-slot choices, uniform per residue."""
    M = np.array([len(CODONS[int(r)]) for r in residues])
    return np.minimum((rng.random((ncand, len(residues))) * M).astype(np.int64), M - 1)


def sampler_candidates(params, residues, ncand: int, seed: int) -> np.ndarray:
    """ncand codon-slot choices drawn by the exact sampler of the window's
    residues as a protein (FP32 scaled inside pass)."""
    f = CodonFold(params)
    f.set_protein(residues)
    f.inside(1)
    cod, _ = f.sample(ncand, seed)
    f.close()
    # cf_sample returns sense-codon ids; map each to its slot within the residue
    sense = [c for c in range(64) if _CODE[c] != "*"]
    slot_of = {}
    for r in range(20):
        for s, trip in enumerate(CODONS[r]):
            slot_of[sense.index(trip[0] * 16 + trip[1] * 4 + trip[2])] = s
    return np.vectorize(slot_of.__getitem__)(cod)


def _pack(residues, cands):
    """Bases of every candidate (rows of codon slots) as one window batch."""
    cands = np.asarray(cands)
    seqs = _TABLE[np.asarray(residues)[None, :], cands].reshape(len(cands), -1)
    off = np.arange(len(cands) + 1, dtype=np.int64) * seqs.shape[1]
    return seqs.ravel(), off


def prescreen(sur, exact: Windows, residues, cands, top: int = 32):
    """Rank candidates by predicted G, re-score the ``top`` best exactly."""
    t0 = time.perf_counter()
    b, o = _pack(residues, cands)
    pred = sur.predict(b, o)
    keep = np.argsort(pred, kind="stable")[:top]
    bk, ok = _pack(residues, cands[keep])
    G = exact.free_energy(bk, ok)
    dt = time.perf_counter() - t0
    j = int(np.argmin(G))
    return {"best_G": float(G[j]), "best": cands[keep[j]], "exact_evals": len(keep), "screened": len(cands),
            "seconds": dt, "pred": pred}


def dp_only(exact: Windows, residues, cands):
    """Score every candidate exactly and keep the best (no surrogate)."""
    t0 = time.perf_counter()
    b, o = _pack(residues, cands)
    G = exact.free_energy(b, o)
    dt = time.perf_counter() - t0
    j = int(np.argmin(G))
    return {"best_G": float(G[j]), "best": cands[j], "exact_evals": len(cands), "seconds": dt, "G": G}
