"""Brute-force enumeration of every codon sequence and every secondary structure.

Independent of the oracle: its own genetic-code table (built from the NCBI
translation-table string in TCAG order), its own structure enumerator and its
own loop-decomposition energy evaluator, written from the model definition:

  * ensemble: pseudoknot-free structures with canonical pairs (AU, CG, GU),
    hairpins of >= 3 unpaired bases, interior/bulge loops of <= 30 unpaired
    (paper, Section "Sequence and structural ensembles"; hairpin minimum from
    Section "Dynamic programming algorithms for fixed RNA sequences");
  * sequence weight prod_r e^{lw[r][c_r]} prod_r e^{pb[c_r][c_{r+1}]}
    (Section "Incorporating soft constraints");
  * structure weight e^{-E/RT} with the nearest-neighbour loop energies.

Only usable for a handful of residues.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

AA = "ARNDCQEGHILKMFPSTWYV"
_NCBI = "FFLLSSSSYY**CC*WLLLLPPPPHHQQRRRRIIIMTTTTNNKKSSRRVVVVAAAADDEEGGGG"
_TCAG = "UCAG"
_IDX = {"A": 0, "C": 1, "G": 2, "U": 3}


def _code():
    table = {}
    for k, aa in enumerate(_NCBI):
        cod = _TCAG[k // 16] + _TCAG[(k // 4) % 4] + _TCAG[k % 4]
        table[cod] = aa
    return table


CODE = _code()
SENSE = sorted([c for c, a in CODE.items() if a != "*"], key=lambda s: [_IDX[x] for x in s])
SENSE_ID = {c: i for i, c in enumerate(SENSE)}


def codons_for(aa_index: int) -> list[str]:
    return [c for c in SENSE if CODE[c] == AA[aa_index]]


PAIRS = {(0, 3): 0, (1, 2): 1, (2, 1): 2, (3, 0): 3, (2, 3): 4, (3, 2): 5}


class Params:
    def __init__(self, vec):
        v = np.asarray(vec, dtype=np.float64)
        self.stack = v[0:36].reshape(6, 6)
        self.H = v[36:67]
        self.Bu = v[67:98]
        self.In = v[98:129]
        self.tm = v[129:145].reshape(4, 4)
        self.d5 = v[145:161].reshape(4, 4)
        self.d3 = v[161:177].reshape(4, 4)
        self.a, self.b, self.c = v[177], v[178], v[179]
        self.kT = 1.98717e-3 * (v[180] + 273.15)


def hairpin_len(p: Params, L: int) -> float:
    if L <= 30:
        return p.H[L]
    return p.H[30] + 1.07856 * math.log(L / 30.0)


def structures(seq, any_pair=False, allow=None):
    """All pseudoknot-free structures as partner lists (-1 = unpaired)."""
    n = len(seq)
    memo = {}

    def ok(i, j):
        if j - i < 4:
            return False
        if allow is not None and not allow[i][j]:
            return False
        return any_pair or (seq[i], seq[j]) in PAIRS

    def rec(i, j):  # structures on [i, j] as tuples of pairs
        if i > j:
            return [()]
        key = (i, j)
        if key in memo:
            return memo[key]
        out = [s for s in rec(i + 1, j)]
        for k in range(i + 4, j + 1):
            if ok(i, k):
                for a in rec(i + 1, k - 1):
                    for b in rec(k + 1, j):
                        out.append(((i, k),) + a + b)
        memo[key] = out
        return out

    res = []
    for pairs in rec(0, n - 1):
        pt = [-1] * n
        for i, j in pairs:
            pt[i], pt[j] = j, i
        res.append(pt)
    return res


def energy(p: Params, seq, pt, any_pair=False):
    """Free energy (kcal/mol) by loop decomposition; None if a loop is outside
    the ensemble (interior/bulge loop longer than 30)."""
    n = len(seq)
    E = 0.0
    # exterior loop
    q = 0
    while q < n:
        if pt[q] > q:
            k, l = q, pt[q]
            if k > 0:
                E += p.d5[seq[k], seq[k - 1]]
            if l < n - 1:
                E += p.d3[seq[l], seq[l + 1]]
            q = l + 1
        else:
            q += 1
    for i in range(n):
        j = pt[i]
        if j <= i:
            continue
        branches = []
        unp = 0
        q = i + 1
        while q < j:
            if pt[q] > q:
                branches.append((q, pt[q]))
                q = pt[q] + 1
            else:
                unp += 1
                q += 1
        if not branches:
            L = j - i - 1
            E += hairpin_len(p, L) + (p.tm[0, 0] if any_pair else p.tm[seq[i + 1], seq[j - 1]])
        elif len(branches) == 1:
            k, l = branches[0]
            l1, l2 = k - i - 1, j - l - 1
            if l1 == 0 and l2 == 0:
                if any_pair:
                    E += p.stack[0, 0]
                else:
                    E += p.stack[PAIRS[(seq[i], seq[j])], PAIRS[(seq[k], seq[l])]]
            elif l1 + l2 > 30:
                return None
            elif l1 == 0 or l2 == 0:
                E += p.Bu[l1 + l2]
            else:
                if any_pair:
                    E += p.In[l1 + l2] + 2 * p.tm[0, 0]
                else:
                    E += p.In[l1 + l2] + p.tm[seq[i + 1], seq[j - 1]] + p.tm[seq[l + 1], seq[k - 1]]
        else:
            E += p.a + p.c * (len(branches) + 1) + p.b * unp
            E += p.d5[seq[j], seq[j - 1]] + p.d3[seq[i], seq[i + 1]]
            for k, l in branches:
                E += p.d5[seq[k], seq[k - 1]] + p.d3[seq[l], seq[l + 1]]
    return E


def enumerate_ensemble(params, residues, lw=None, pb=None, any_pair=False, allow=None):
    """Every (codon tuple, partner list, Boltzmann weight) of the joint ensemble."""
    p = Params(params)
    res = [int(r) for r in residues]
    m = len(res)
    opts = [codons_for(r) for r in res]
    out = []
    struct_cache = {}
    for combo in itertools.product(*[range(len(o)) for o in opts]):
        cods = [opts[r][combo[r]] for r in range(m)]
        seq = tuple(_IDX[b] for c in cods for b in c)
        logw = 0.0
        for r in range(m):
            if lw is not None:
                logw += lw[r][combo[r]]
            if pb is not None and r + 1 < m:
                logw += pb[SENSE_ID[cods[r]]][SENSE_ID[cods[r + 1]]]
        key = seq
        if key not in struct_cache:
            struct_cache[key] = structures(seq, any_pair=any_pair, allow=allow)
        for pt in struct_cache[key]:
            E = energy(p, seq, pt, any_pair=any_pair)
            if E is None:
                continue
            w = math.exp(logw - E / p.kT)
            out.append((tuple(combo), tuple(SENSE_ID[c] for c in cods), tuple(pt), w))
    return out


def summary(params, residues, lw=None, pb=None, any_pair=False, allow=None):
    """log Z, P, codon marginals (by slot), pair-bonus gradient, base marginals."""
    ens = enumerate_ensemble(params, residues, lw, pb, any_pair, allow)
    m = len(residues)
    n = 3 * m
    Z = sum(e[3] for e in ens)
    P = np.zeros((n, n))
    pc = np.zeros((m, 6))
    pg = np.zeros((61, 61))
    pbase = np.zeros((n, 4))
    for slots, cids, pt, w in ens:
        pr = w / Z
        for i in range(n):
            j = pt[i]
            P[i, i if j < 0 else j] += pr
        for r in range(m):
            pc[r, slots[r]] += pr
            if r + 1 < m:
                pg[cids[r], cids[r + 1]] += pr
            cod = SENSE[cids[r]]
            for off in range(3):
                pbase[3 * r + off, _IDX[cod[off]]] += pr
    return {"logZ": math.log(Z), "P": P, "codon": pc, "pair_grad": pg, "base": pbase,
            "ensemble": ens, "Z": Z}


# ---------------------------------------------------------------- exact integer costs (MFE)
# The minimum free energy form works on integer costs: every elementary energy
# term, and every codon log-weight and pair bonus converted to kcal/mol as
# -kT w, is rounded once to the nearest multiple of 2^-32 kcal/mol (half away
# from zero); a configuration's cost is the sum of its terms.

Q_SCALE = 2.0 ** 32


def qcost(e: float) -> int:
    v = e * Q_SCALE
    return int(math.floor(v + 0.5)) if v >= 0 else -int(math.floor(-v + 0.5))


def energy_q(p: Params, seq, pt):
    """Integer cost of a structure by loop decomposition (same loops as
    energy()); None outside the ensemble."""
    n = len(seq)
    E = 0
    q = 0
    while q < n:
        if pt[q] > q:
            k, l = q, pt[q]
            if k > 0:
                E += qcost(p.d5[seq[k], seq[k - 1]])
            if l < n - 1:
                E += qcost(p.d3[seq[l], seq[l + 1]])
            q = l + 1
        else:
            q += 1
    for i in range(n):
        j = pt[i]
        if j <= i:
            continue
        branches, unp, q = [], 0, i + 1
        while q < j:
            if pt[q] > q:
                branches.append((q, pt[q]))
                q = pt[q] + 1
            else:
                unp += 1
                q += 1
        if not branches:
            E += qcost(hairpin_len(p, j - i - 1)) + qcost(p.tm[seq[i + 1], seq[j - 1]])
        elif len(branches) == 1:
            k, l = branches[0]
            l1, l2 = k - i - 1, j - l - 1
            if l1 == 0 and l2 == 0:
                E += qcost(p.stack[PAIRS[(seq[i], seq[j])], PAIRS[(seq[k], seq[l])]])
            elif l1 + l2 > 30:
                return None
            elif l1 == 0 or l2 == 0:
                E += qcost(p.Bu[l1 + l2])
            else:
                E += qcost(p.In[l1 + l2]) + qcost(p.tm[seq[i + 1], seq[j - 1]]) + qcost(p.tm[seq[l + 1], seq[k - 1]])
        else:
            E += qcost(p.a) + qcost(p.c) * (len(branches) + 1) + qcost(p.b) * unp
            E += qcost(p.d5[seq[j], seq[j - 1]]) + qcost(p.d3[seq[i], seq[i + 1]])
            for k, l in branches:
                E += qcost(p.d5[seq[k], seq[k - 1]]) + qcost(p.d3[seq[l], seq[l + 1]])
    return E


def weight_cost(p: Params, slots, cids, lw=None, pb=None) -> int:
    """Integer cost of the soft constraints of a codon choice: -kT w per
    codon log-weight and per adjacent codon-pair bonus, each rounded."""
    tot = 0
    m = len(slots)
    for r in range(m):
        tot += qcost(-(p.kT * (lw[r][slots[r]] if lw is not None else 0.0)))
        if r + 1 < m:
            tot += qcost(-(p.kT * (pb[cids[r]][cids[r + 1]] if pb is not None else 0.0)))
    return tot


def config_cost(params, residues, cids, partner, lw=None, pb=None):
    """Cost of one (codon sequence, structure) given as sense codon ids and
    a partner list; None if the structure is outside the ensemble."""
    p = Params(params)
    res = [int(r) for r in residues]
    slots = []
    for r, cid in zip(res, cids):
        cods = codons_for(r)
        c = SENSE[int(cid)]
        if c not in cods:
            return None
        slots.append(cods.index(c))
    seq = tuple(_IDX[b] for cid in cids for b in SENSE[int(cid)])
    pt = [int(x) for x in partner]
    for i, j in enumerate(pt):
        if j >= 0 and (pt[j] != i or abs(j - i) < 4 or (seq[min(i, j)], seq[max(i, j)]) not in PAIRS):
            return None
    for i in range(len(pt)):  # no crossing pairs
        j = pt[i]
        if j > i and any(pt[k] > j or (0 <= pt[k] < i) for k in range(i + 1, j)):
            return None
    e = energy_q(p, seq, pt)
    return None if e is None else e + weight_cost(p, slots, [int(c) for c in cids], lw, pb)


def mfe_bruteforce(params, residues, lw=None, pb=None):
    """Minimum integer cost over every codon sequence and structure."""
    p = Params(params)
    res = [int(r) for r in residues]
    opts = [codons_for(r) for r in res]
    best = None
    for combo in itertools.product(*[range(len(o)) for o in opts]):
        cods = [opts[r][combo[r]] for r in range(len(res))]
        cids = [SENSE_ID[c] for c in cods]
        seq = tuple(_IDX[b] for c in cods for b in c)
        wc = weight_cost(p, combo, cids, lw, pb)
        for pt in structures(seq):
            e = energy_q(p, seq, pt)
            if e is not None and (best is None or e + wc < best):
                best = e + wc
    return best
