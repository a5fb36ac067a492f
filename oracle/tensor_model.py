"""Oracle for the tensor-based free energy model under codon constraints --
TEST INFRASTRUCTURE ONLY (imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the library).

Model (paper SI "Tensor-based free energy models", Eq. general-model): a
gamma x gamma matrix V_x for an unpaired base x, matrices B^rho_{x,y}
(rho = 0..nrho-1) for the two sides of a base pair, and S for the weighted
trace Tr_S[X] = tr(S X).  The Boltzmann weight of a structure of a fixed
sequence is the sum over one rho per base pair of the product over loops of
Tr_S[the loop's matrices in backbone order]: V for an unpaired base, B^rho of
the pair for a base whose next base in the loop is its partner, and the
identity for a paired base whose next base continues along the backbone.
Pairs closer than 4 positions have no weight (hairpins of >= 3 bases).  The
exterior loop is closed by the same weighted trace (the strand break matrix
folded into V and B, as the paper does).

Sequences (Eq. amino-q, codon-pair tensor train Eq. pair-tt): every codon
sequence c encoding the protein weighs e^{lw[r][c_r]} per residue and
e^{pb[c_r][c_{r+1}]} per residue boundary; Z sums weight x structure weight
over all codon sequences and structures, log Z is its natural log.

Two independent computations:
  * ``logz`` -- the recursion of Eq. complicated-pf with the fold of Eq. fold
    generalised to sequence states by DesignFold (Eq. design-fold), over
    intervals [i, j) whose matrices carry (codon state, structural index) at
    both ends; float64, plain loops, no rescaling;
  * ``brute_force_logz`` -- Eq. general-model written out: every codon
    sequence, every structure, every assignment of rho, every loop's traced
    product (tiny inputs only).
``normalize`` is the spectral-radius renormalisation of SI "Free energy model
renormalization": V'_x = V_x / r_x, B'_{x,y} = B_{x,y} / sqrt(r_x r_y),
r_x the spectral radius of V_x.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

MIN_SPAN = 4  # a pair (k, l) needs l - k >= 4 (hairpin loops of >= 3 bases)

# standard genetic code over bases A, C, G, U (codons in lexicographic order)
_CODE = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF"
_AA = "ARNDCQEGHILKMFPSTWYV"


def codon_states(aa: int) -> list[tuple[int, int, int, int]]:
    """Sense codons of amino acid ``aa`` (ARNDCQEGHILKMFPSTWYV order) in codon
    order, each as (sense id 0..60, base 1, base 2, base 3) with A, C, G, U = 0..3."""
    out, sid = [], 0
    for c in range(64):
        if _CODE[c] == "*":
            continue
        if _CODE[c] == _AA[aa]:
            out.append((sid, c >> 4 & 3, c >> 2 & 3, c & 3))
        sid += 1
    return out


def spectral_radius(A) -> float:
    """Largest |eigenvalue| of a square matrix (library eigenvalue routine)."""
    return float(np.max(np.abs(np.linalg.eigvals(np.asarray(A, dtype=np.float64)))))


def normalize(V, B):
    """SI "Free energy model renormalization": V_x / r_x and B_{x,y} / sqrt(r_x r_y)."""
    V = np.asarray(V, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    r = np.array([spectral_radius(V[x]) for x in range(4)])
    Vn = V / r[:, None, None]
    Bn = B / np.sqrt(r[None, :, None, None, None] * r[None, None, :, None, None])
    return Vn, Bn


def _sequence_side(residues, lw, pb):
    """Per position: codon states (their bases), and the transfer weights."""
    res = [int(r) for r in residues]
    m = len(res)
    lw = np.zeros((m, 6)) if lw is None else np.asarray(lw, dtype=np.float64).reshape(m, 6)
    pb = np.zeros((61, 61)) if pb is None else np.asarray(pb, dtype=np.float64).reshape(61, 61)
    cods = [codon_states(r) for r in res]
    n = 3 * m
    states = [cods[p // 3] for p in range(n)]
    base = [[c[1 + p % 3] for c in states[p]] for p in range(n)]
    # T_p (states at p -> states at p+1): identity inside a residue,
    # e^{lw[r+1][b] + pb[c_a][c_b]} across the boundary r -> r+1
    T = []
    for p in range(n - 1):
        A, Bs = states[p], states[p + 1]
        t = np.zeros((len(A), len(Bs)))
        if p % 3 != 2:
            t[:] = np.eye(len(A))
        else:
            r1 = (p + 1) // 3
            for a, ca in enumerate(A):
                for b, cb in enumerate(Bs):
                    t[a, b] = math.exp(lw[r1, b] + pb[ca[0], cb[0]])
        T.append(t)
    u0 = np.array([math.exp(lw[0, a]) for a in range(len(states[0]))])
    return n, base, T, u0


def logz(V, B, S, residues, lw=None, pb=None) -> float:
    """log Z by the recursion (Eq. complicated-pf, Eq. fold, Eq. design-fold).

    Q[(i, j)] for the interval [i, j): a matrix over (state at i, zeta) x
    (state at j-1, zeta'), flattened state-major.  Q[(i, i+1)] = delta_ab V;
      Q[(i, j+1)] = Q[(i, j)] X_j + sum_{k=i}^{j-4} L_{i,k} F_{k,j}
    where X_j = T_{j-1} (x) V_j (base j unpaired), L_{i,i} = identity and
    L_{i,k} = Q[(i, k)] (T_{k-1} (x) I) (the bases before k, bonded to k),
    and F_{k,j} (k paired to j) = sum_rho B^rho_{k,j} Tr_S[B^rho_{j,k} Y_{k,j}]
    per pair of end states, Y_{k,j} = (T_k (x) I) Q[(k+1, j)] (T_{j-1} (x) I)
    (the closed loop: j -> k across the pair, then along k+1 .. j-1 back to
    j).  Z = sum_{a, c} u0[a] Tr_S[Q[(0, n)]_{a c}] (the exterior loop)."""
    V = np.asarray(V, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    g = V.shape[1]
    nrho = B.shape[0]
    n, base, T, u0 = _sequence_side(residues, lw, pb)
    M = [len(b) for b in base]
    I = np.eye(g)

    def kron_state(t):  # a state-to-state matrix acting on (state, zeta)
        return np.kron(t, I)

    Q, L = {}, {}
    for i in range(n):
        Q[(i, i + 1)] = np.zeros((M[i] * g, M[i] * g))
        for a in range(M[i]):
            Q[(i, i + 1)][a * g:(a + 1) * g, a * g:(a + 1) * g] = V[base[i][a]]
        if i + 1 < n:
            L[(i, i + 1)] = Q[(i, i + 1)] @ kron_state(T[i])
    F = {}
    for length in range(2, n + 1):
        # folds of the pairs (k, j) at distance length - 1, from Q[(k+1, j)]
        D = length - 1
        if D >= MIN_SPAN:
            for k in range(0, n - D):
                j = k + D
                Y = kron_state(T[k]) @ Q[(k + 1, j)] @ kron_state(T[j - 1])
                f = np.zeros((M[k] * g, M[j] * g))
                for a in range(M[k]):
                    for c in range(M[j]):
                        blk = Y[a * g:(a + 1) * g, c * g:(c + 1) * g]
                        xa, xc = base[k][a], base[j][c]
                        for rho in range(nrho):
                            t = np.trace(S @ B[rho, xc, xa] @ blk)
                            f[a * g:(a + 1) * g, c * g:(c + 1) * g] += B[rho, xa, xc] * t
                F[(k, j)] = f
        for i in range(0, n - length + 1):
            j1 = i + length  # new interval [i, j1), new last base j = j1 - 1
            j = j1 - 1
            X = np.zeros((M[j - 1] * g, M[j] * g))
            for b in range(M[j - 1]):
                for c in range(M[j]):
                    X[b * g:(b + 1) * g, c * g:(c + 1) * g] = T[j - 1][b, c] * V[base[j][c]]
            q = Q[(i, j)] @ X
            for k in range(i, j - MIN_SPAN + 1):
                Lik = np.eye(M[i] * g) if k == i else L[(i, k)]
                q = q + Lik @ F[(k, j)]
            Q[(i, j1)] = q
            if j1 < n:
                L[(i, j1)] = q @ kron_state(T[j1 - 1])
    QN = Q[(0, n)]
    Z = 0.0
    for a in range(M[0]):
        for c in range(M[n - 1]):
            Z += u0[a] * np.trace(S @ QN[a * g:(a + 1) * g, c * g:(c + 1) * g])
    return math.log(Z)


def _structures(n):
    """Every pseudoknot-free pairing of 0..n-1 with l - k >= MIN_SPAN (partner list)."""
    def rec(i, j):  # structures of [i, j)
        if j - i <= 0:
            yield []
            return
        for s in rec(i + 1, j):  # i unpaired
            yield s
        for l in range(i + MIN_SPAN, j):
            for inner in rec(i + 1, l):
                for rest in rec(l + 1, j):
                    yield [(i, l)] + inner + rest
    for pairs in rec(0, n):
        part = [-1] * n
        for k, l in pairs:
            part[k], part[l] = l, k
        yield part


def _loop_weight(part, seq, V, B, S, rho_of, start, stop, closing):
    """Tr_S of the loop whose bases are start..stop-1 at this level, closed by
    the pair ``closing`` = (k, l) (None: the exterior loop): the traversal
    begins at l with B_{l,k}, then k (identity), then the loop's bases."""
    g = V.shape[1]
    Mx = np.eye(g)
    if closing is not None:
        k, l = closing
        Mx = Mx @ B[rho_of[(k, l)], seq[l], seq[k]]
    p = start
    while p < stop:
        q = part[p]
        if q < 0:
            Mx = Mx @ V[seq[p]]
            p += 1
        else:  # p pairs with q > p: B_{p,q} (next in this loop is q), q itself identity
            Mx = Mx @ B[rho_of[(p, q)], seq[p], seq[q]]
            p = q + 1
    return float(np.trace(S @ Mx))


def brute_force_logz(V, B, S, residues, lw=None, pb=None) -> float:
    """Eq. general-model summed over every codon sequence, structure and rho
    assignment, with the codon weights of Eq. amino-q (tiny inputs only)."""
    V = np.asarray(V, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    nrho = B.shape[0]
    res = [int(r) for r in residues]
    m = len(res)
    lw = np.zeros((m, 6)) if lw is None else np.asarray(lw, dtype=np.float64).reshape(m, 6)
    pb = np.zeros((61, 61)) if pb is None else np.asarray(pb, dtype=np.float64).reshape(61, 61)
    n = 3 * m
    structs = list(_structures(n))
    Z = 0.0
    for choice in itertools.product(*[list(enumerate(codon_states(r))) for r in res]):
        w = 1.0
        for r, (slot, c) in enumerate(choice):
            w *= math.exp(lw[r, slot])
            if r + 1 < m:
                w *= math.exp(pb[c[0], choice[r + 1][1][0]])
        seq = [c[1 + p % 3] for (_, c) in choice for p in range(3)]
        for part in structs:
            pairs = [(k, l) for k, l in enumerate(part) if l > k]
            for rhos in itertools.product(range(nrho), repeat=len(pairs)):
                rho_of = dict(zip(pairs, rhos))
                wt = _loop_weight(part, seq, V, B, S, rho_of, 0, n, None)
                for (k, l) in pairs:
                    wt *= _loop_weight(part, seq, V, B, S, rho_of, k + 1, l, (k, l))
                Z += w * wt
    return math.log(Z)
