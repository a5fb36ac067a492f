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
