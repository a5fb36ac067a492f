"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds random draws only: no part of the partition-function
arithmetic lives here, so that the oracle and the CUDA library stay
independent of each other while reading identical inputs.

Every artefact uses its own ``numpy.random.default_rng(seed)`` and draws in the
order written below.  The paper's workloads are real proteins and a trained
tensor model (Section "Example proteins and free energy models"), neither of
which exists here; these generators stand in for them with the shapes the
nearest-neighbour model uses.

Parameter vector layout (float64, ``NPARAMS`` entries), energies in kcal/mol:

====================  =====  ==============================================
slice                 size   meaning
====================  =====  ==============================================
``[0:36]``            6x6    stack[outer pair type][inner pair type]
``[36:67]``           31     hairpin length term H[L], L = 0..30
``[67:98]``           31     bulge length term Bu[L]
``[98:129]``          31     interior length term In[L]
``[129:145]``         4x4    terminal mismatch tm[x][y]
``[145:161]``         4x4    5' dangle d5[paired base][dangling base]
``[161:177]``         4x4    3' dangle d3[paired base][dangling base]
``[177:180]``         3      multiloop a (closing), b (per unpaired), c (per branch)
``[180]``             1      temperature in degrees Celsius
====================  =====  ==============================================

Bases are indexed A, C, G, U = 0..3 and pair types AU, CG, GC, UA, GU, UG = 0..5.
Amino acids are indexed in the order ``ARNDCQEGHILKMFPSTWYV``.
"""
from __future__ import annotations

import numpy as np

AMINO_ACIDS = "ARNDCQEGHILKMFPSTWYV"
NPARAMS = 181
MAXLOOP = 30
N_SENSE = 61


def nn_params(seed: int = 0) -> np.ndarray:
    """Synthetic nearest-neighbour parameter vector (layout in the module docstring)."""
    rng = np.random.default_rng(seed)
    stack = rng.uniform(-3.5, -0.5, (6, 6))
    hairpin = rng.uniform(1.0, 6.0, MAXLOOP + 1)
    bulge = rng.uniform(1.0, 6.0, MAXLOOP + 1)
    interior = rng.uniform(1.0, 6.0, MAXLOOP + 1)
    tm = rng.uniform(-1.5, 0.0, (4, 4))
    d5 = rng.uniform(-1.5, 0.0, (4, 4))
    d3 = rng.uniform(-1.5, 0.0, (4, 4))
    out = np.concatenate([
        stack.ravel(), hairpin, bulge, interior, tm.ravel(), d5.ravel(), d3.ravel(),
        np.array([3.4, 0.0, 0.4, 37.0]),
    ])
    assert out.size == NPARAMS
    return out


def residues_uniform(m: int, seed: int) -> np.ndarray:
    """Residues drawn uniformly over the 20 amino acids (int32 indices)."""
    return np.random.default_rng(seed).integers(0, 20, m).astype(np.int32)


def residues_dirichlet(m: int, seed: int) -> np.ndarray:
    """Composition ~ Dirichlet(1), then residues i.i.d. from it (same generator)."""
    rng = np.random.default_rng(seed)
    freqs = rng.dirichlet(np.ones(20))
    return rng.choice(20, m, p=freqs).astype(np.int32)


def to_string(res: np.ndarray) -> str:
    return "".join(AMINO_ACIDS[int(r)] for r in res)


def soft_weights(m: int, seed: int, sigma_codon: float = 0.5, sigma_pair: float = 0.2,
                 pair: bool = True):
    """Per-(residue, codon slot) log-weights ~ N(0, sigma_codon), all 6 slots drawn
    (slots beyond an amino acid's codon count are ignored), then the 61x61
    codon-pair log-bonus ~ N(0, sigma_pair) from the same generator."""
    rng = np.random.default_rng(seed)
    lw = rng.normal(0.0, sigma_codon, (m, 6))
    pb = rng.normal(0.0, sigma_pair, (N_SENSE, N_SENSE)) if pair else np.zeros((N_SENSE, N_SENSE))
    return lw, pb


def workload(name: str):
    """The named synthetic workloads (residues, lw, pb); lw/pb None means all-zero."""
    if name == "p8_uniform":          # 8 aa, uniform residues, seed 0
        return residues_uniform(8, 0), None, None
    if name == "p300_dirichlet":      # 300 aa, Dirichlet(1) composition, seed 1
        return residues_dirichlet(300, 1), None, None
    if name == "p300_weighted":       # the 300-aa protein with soft weights, seed 2
        lw, pb = soft_weights(300, 2)
        return residues_dirichlet(300, 1), lw, pb
    if name == "p1000_weighted":      # 1000 aa, Dirichlet(1) seed 4, codon weights only
        rng = np.random.default_rng(4)
        freqs = rng.dirichlet(np.ones(20))
        res = rng.choice(20, 1000, p=freqs).astype(np.int32)
        lw = rng.normal(0.0, 0.5, (1000, 6))
        return res, lw, None
    if name == "p200_bent":           # 100 lysines, then 100 aa of Dirichlet(1) composition, seed 5
        # Lysine codons (AAA, AAG) cannot pair with each other, so the best
        # interval of each length lies in the second half until the length
        # passes 300 nt: the per-diagonal exponents bend there.
        res = np.concatenate([np.full(100, AMINO_ACIDS.index("K")), residues_dirichlet(100, 5)])
        return res.astype(np.int32), None, None
    raise KeyError(name)


def batch_p8(count: int = 4096):
    """The small-protein throughput batch: `count` proteins of 8 residues,
    protein k drawn uniformly over the 20 amino acids with seed k (protein 0
    is p8_uniform)."""
    return [residues_uniform(8, k) for k in range(count)]


# Standard genetic code, codons in lexicographic order over A, C, G, U
# (AAA, AAC, ..., UUU); '*' marks the three stop codons.
GENETIC_CODE = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF"


def codon_table():
    """Per amino acid (ARNDCQEGHILKMFPSTWYV order), its sense codons as base
    triples (0..3), in codon order."""
    out = []
    for a in AMINO_ACIDS:
        out.append([(c >> 4 & 3, c >> 2 & 3, c & 3) for c in range(64) if GENETIC_CODE[c] == a])
    return out


def windows(nwin: int, seed: int = 3):
    """Windows of designed sequences: per window a random protein of
    U{100..400} residues with Dirichlet(1) composition, codons uniform per
    residue, a window length U{60..240} nt rounded down to whole codons and a
    start codon uniform over the protein.  Only the window's own residues are
    drawn (residues are i.i.d. given the composition, so the distribution is
    that of cutting the full protein).

    Returns (residues, slots, bases, offsets): per window the amino-acid
    indices and codon slots (index into the residue's codon list), and all
    windows' bases concatenated (uint8) with int64 offsets."""
    rng = np.random.default_rng(seed)
    plen = rng.integers(100, 401, nwin)
    freqs = rng.dirichlet(np.ones(20), nwin)
    wcod = rng.integers(60, 241, nwin) // 3
    start = (rng.random(nwin) * (plen - wcod + 1)).astype(np.int64)
    u_res = rng.random((nwin, 80))
    u_cod = rng.random((nwin, 80))
    table = codon_table()
    ncod = np.array([len(c) for c in table])
    cum = np.cumsum(freqs, axis=1)
    res = np.minimum((u_res[:, :, None] > cum[:, None, :]).sum(axis=2), 19)
    slots = np.minimum((u_cod * ncod[res]).astype(np.int64), ncod[res] - 1)
    flat = np.array([b for cods in table for c in cods for b in c], dtype=np.uint8).reshape(-1, 3)
    first = np.concatenate([[0], np.cumsum(ncod)[:-1]])
    offsets = np.concatenate([[0], np.cumsum(3 * wcod)]).astype(np.int64)
    bases = np.empty(offsets[-1], dtype=np.uint8)
    rl, sl = [], []
    for w in range(nwin):
        r, s_ = res[w, :wcod[w]], slots[w, :wcod[w]]
        bases[offsets[w]:offsets[w + 1]] = flat[first[r] + s_].ravel()
        rl.append(r.astype(np.int32))
        sl.append(s_.astype(np.int32))
    del start  # the start fixes where the window sits in its protein, not its content
    return rl, sl, bases, offsets


SURROGATE_SHAPES = [(64, 4, 5), (64,), (64, 64, 5), (64,), (64, 64, 5), (64,), (64, 64, 5), (64,), (64,), (1,)]


def surrogate_init(seed: int = 0) -> np.ndarray:
    """Initial surrogate parameters in flat order (W1, b1, .., W4, b4, wh, bh):
    conv weights ~ N(0, 2 / fan_in), head weights ~ N(0, 1/64), biases 0."""
    rng = np.random.default_rng(seed)
    out = []
    for s in SURROGATE_SHAPES:
        if len(s) == 3:
            out.append(rng.normal(0.0, np.sqrt(2.0 / (s[1] * s[2])), s).ravel())
        elif s == (64,) and len(out) == 8:
            out.append(rng.normal(0.0, 1.0 / 8.0, s))
        else:
            out.append(np.zeros(s))
    return np.concatenate(out)


def ascent_targets(m: int, seed: int = 3) -> np.ndarray:
    """Independent N(0,1) logits per (residue, slot) for frequency targets."""
    return np.random.default_rng(seed).normal(0.0, 1.0, (m, 6))


# canonical and wobble pairs (A, C, G, U = 0..3): AU, CG, GC, UA, GU, UG
_PAIRS = ((0, 3), (1, 2), (2, 1), (3, 0), (2, 3), (3, 2))


def tm_params(seed: int = 0, gamma: int = 4, nrho: int = 2, pair_scale: float = 2.0):
    """A synthetic tensor-based model (the paper's trained tensors are not
    available): V[4][g][g] ~ U(0.2, 1.0); B[rho][x][y][g][g] ~ pair_scale *
    U(0, 1) for the six canonical and wobble pairs (x, y), zero for every
    other base pair; S[g][g] ~ U(0.1, 1.0); drawn in that order from
    default_rng(seed)."""
    rng = np.random.default_rng(seed)
    V = rng.uniform(0.2, 1.0, (4, gamma, gamma))
    Braw = pair_scale * rng.uniform(0.0, 1.0, (nrho, 4, 4, gamma, gamma))
    mask = np.zeros((4, 4))
    for x, y in _PAIRS:
        mask[x, y] = 1.0
    B = Braw * mask[None, :, :, None, None]
    S = rng.uniform(0.1, 1.0, (gamma, gamma))
    return V, B, S
