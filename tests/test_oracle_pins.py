"""Pins of the CPU oracle against things other than itself.

* brute-force enumeration of every codon sequence and every structure
  (2-5 residues, and sparse pair masks at 36-60 nt so that long hairpins,
  long bulges and the 30-nt interior-loop cap are reached);
* closed forms: the structure-free tensor-train count (paper, Section
  "Incorporating hard constraints": e^{-q_seq} = |Phi(psi)|), a single
  allowed pair, and the scalar counting recursion (Eq. scalar-pf) with all
  pairs allowed and all energies zero;
* invariants of the pair-probability matrix (symmetric, doubly stochastic;
  Section "Dynamic programming algorithms for fixed RNA sequences") and of
  the marginals;
* definitions: codon marginals by clamping the codon (Eq. marginal-codon),
  pair probabilities by forbidding the pair, derivatives by central finite
  differences.
"""
import math

import numpy as np
import pytest

import bruteforce as bf
import oracle
import synth

P0 = synth.nn_params(0)


def _cmp(b, o, tol=1e-11):
    assert abs(b["logZ"] - o["logZ"]) < tol * max(1.0, abs(b["logZ"]))
    assert np.abs(b["P"] - o["P"]).max() < tol
    assert np.abs(b["codon"] - o["codon"]).max() < tol
    assert np.abs(b["pair_grad"] - o["pair_grad"]).max() < tol


def test_codon_tables_agree():
    for aa in range(20):
        assert oracle.codons_of(aa) == [bf.SENSE_ID[c] for c in bf.codons_for(aa)]
    assert len(bf.SENSE) == 61
    assert sum(len(oracle.codons_of(a)) for a in range(20)) == 61


@pytest.mark.parametrize("res", [[0, 1], [10, 15], [0, 1, 2], [12, 17, 3], [0, 1, 2, 3], [5, 7, 2, 14]])
def test_bruteforce_plain(res):
    _cmp(bf.summary(P0, res), oracle.outside(P0, res))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bruteforce_soft_weights(seed):
    rng = np.random.default_rng(seed)
    res = list(rng.integers(0, 20, 4))
    lw = rng.normal(0, 0.5, (4, 6))
    pb = rng.normal(0, 0.3, (61, 61))
    b = bf.summary(P0, res, lw, pb)
    o = oracle.outside(P0, res, lw, pb)
    _cmp(b, o)
    assert np.abs(b["base"] - oracle.base_marginals(res, o["codon"])).max() < 1e-11


@pytest.mark.parametrize("res", [[12, 17, 12, 17], [12, 17, 12, 17, 12], [3, 12, 17, 12, 17]])
def test_bruteforce_multiloops(res):
    # every base pairs with every base: multiloops with 2-3 branches appear at 12-15 nt
    rng = np.random.default_rng(len(res))
    lw = rng.normal(0, 0.5, (len(res), 6))
    b = bf.summary(P0, res, lw, None, any_pair=True)
    ens_ml = 0
    for _, _, pt, _ in b["ensemble"]:
        for i, j in enumerate(pt):
            if j > i:
                br, q = 0, i + 1
                while q < j:
                    if pt[q] > q:
                        br, q = br + 1, pt[q] + 1
                    else:
                        q += 1
                ens_ml += br >= 2
    assert ens_ml > 0
    _cmp(b, oracle.outside(P0, res, lw, None, any_pair=True))


def _sparse_mask(res, npairs, seed, forced=()):
    """Random subset of canonical pairs over the sequences the protein allows."""
    rng = np.random.default_rng(seed)
    m = len(res)
    n = 3 * m
    opts = [bf.codons_for(r) for r in res]
    allow = np.zeros((n, n), dtype=np.uint8)
    cand = []
    for i in range(n):
        for j in range(i + 4, n):
            bi = {bf._IDX[c[i % 3]] for c in opts[i // 3]}
            bj = {bf._IDX[c[j % 3]] for c in opts[j // 3]}
            if any((x, y) in bf.PAIRS for x in bi for y in bj):
                cand.append((i, j))
    for k in rng.choice(len(cand), min(npairs, len(cand)), replace=False):
        allow[cand[k]] = 1
    for i, j in forced:
        allow[i, j] = 1
    return allow


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_bruteforce_long_loops(seed):
    """36-54 nt with mostly single-codon residues and a sparse pair mask: long
    hairpins (> 30, log extrapolation), long bulges/interior loops and the cap."""
    rng = np.random.default_rng(100 + seed)
    m = 12 + 3 * seed
    res = [int(x) for x in rng.choice([12, 17], m)]  # M, W
    for r in rng.choice(m, 2, replace=False):
        res[r] = int(rng.choice([1, 9, 3]))
    n = 3 * m
    allow = _sparse_mask(res, 14, seed)
    lw = rng.normal(0, 0.5, (m, 6))
    b = bf.summary(P0, res, lw, None, allow=allow)
    _cmp(b, oracle.outside(P0, res, lw, None, allow=allow))
    assert n > 33


def test_interior_cap_closed_form():
    """Outer pair (i,j) around inner (k,l): an interior loop of 30 unpaired
    counts, one of 31 does not (l1 + l2 <= 30)."""
    res = [12, 17] * 14  # AUG UGG ... fixed sequence, 84 nt
    m = len(res)
    n = 3 * m
    seq = [bf._IDX[ch] for r in res for ch in bf.codons_for(r)[0]]
    p = bf.Params(P0)

    def find(L):
        for i in range(0, 20):
            for l1 in range(1, L):
                l2 = L - l1
                k = i + 1 + l1
                for l in range(k + 4, k + 12):
                    j = l + 1 + l2
                    if j >= n:
                        continue
                    if (seq[i], seq[j]) in bf.PAIRS and (seq[k], seq[l]) in bf.PAIRS:
                        return i, j, k, l
        raise AssertionError("no geometry")

    for L, counts in [(30, True), (31, False)]:
        i, j, k, l = find(L)
        allow = np.zeros((n, n), dtype=np.uint8)
        allow[i, j] = allow[k, l] = 1
        lz = oracle.inside(P0, res, allow=allow)
        # closed form: empty + hairpin(k,l) + hairpin(i,j) + (interior if L <= 30)
        def ext(a, b):
            e = 0.0
            if a > 0:
                e += p.d5[seq[a], seq[a - 1]]
            if b < n - 1:
                e += p.d3[seq[b], seq[b + 1]]
            return e
        hk = bf.hairpin_len(p, l - k - 1) + p.tm[seq[k + 1], seq[l - 1]]
        hi = bf.hairpin_len(p, j - i - 1) + p.tm[seq[i + 1], seq[j - 1]]
        Z = 1.0 + math.exp(-(hk + ext(k, l)) / p.kT) + math.exp(-(hi + ext(i, j)) / p.kT)
        if counts:
            e_int = p.In[L] + p.tm[seq[i + 1], seq[j - 1]] + p.tm[seq[l + 1], seq[k - 1]]
            Z += math.exp(-(e_int + hk + ext(i, j)) / p.kT)
        assert abs(lz - math.log(Z)) < 1e-12


def _tensor_train_logZ(res, lw, pb):
    """Structure-free partition function u0^T T_0 ... T_{n-2} 1 from the
    brute-force module's codon table (independent of the oracle)."""
    m = len(res)
    cods = [bf.codons_for(r) for r in res]
    v = np.array([math.exp(lw[0][a]) if lw is not None else 1.0 for a in range(len(cods[0]))])
    for r in range(1, m):
        T = np.zeros((len(cods[r - 1]), len(cods[r])))
        for a, ca in enumerate(cods[r - 1]):
            for b, cb in enumerate(cods[r]):
                w = lw[r][b] if lw is not None else 0.0
                if pb is not None:
                    w += pb[bf.SENSE_ID[ca]][bf.SENSE_ID[cb]]
                T[a, b] = math.exp(w)
        v = v @ T
    return math.log(v.sum())


def test_no_pairs_is_tensor_train_count():
    res, lw, pb = synth.workload("p300_weighted")
    res, lw = res[:60], lw[:60]
    n = 3 * len(res)
    allow = np.zeros((n, n), dtype=np.uint8)
    assert abs(oracle.inside(P0, res, lw, pb, allow=allow) - _tensor_train_logZ(res, lw, pb)) < 1e-10
    # unweighted: |Phi(psi)| = prod of codon counts
    count = sum(math.log(len(bf.codons_for(r))) for r in res)
    assert abs(oracle.inside(P0, res, allow=allow) - count) < 1e-10


def test_single_pair_hairpin_any_length():
    """Only the pair (0, n-1) allowed: Z = sum_c w(c) (1 + [pair ok] e^{-(H(L)+tm)/RT}),
    L = n-2 up to 58 (the logarithmic extrapolation beyond 30)."""
    p = bf.Params(P0)
    for m in (3, 9, 11, 20):
        rng = np.random.default_rng(m)
        res = [int(x) for x in rng.integers(0, 20, m)]
        lw = rng.normal(0, 0.5, (m, 6))
        n = 3 * m
        allow = np.zeros((n, n), dtype=np.uint8)
        allow[0, n - 1] = 1
        cods = [bf.codons_for(r) for r in res]
        # transfer chain from the first to the last residue, tracking end codons
        chain = np.diag([math.exp(lw[0][a]) for a in range(len(cods[0]))])
        for r in range(1, m):
            T = np.array([[math.exp(lw[r][b]) for b in range(len(cods[r]))] for _ in cods[r - 1]])
            chain = chain @ T
        Z = chain.sum()
        L = n - 2
        for a, ca in enumerate(cods[0]):
            for b, cb in enumerate(cods[-1]):
                x, y = bf._IDX[ca[0]], bf._IDX[cb[2]]
                if (x, y) in bf.PAIRS:
                    e = bf.hairpin_len(p, L) + p.tm[bf._IDX[ca[1]], bf._IDX[cb[1]]]
                    Z += chain[a, b] * math.exp(-e / p.kT)
        assert abs(oracle.inside(P0, res, lw, allow=allow) - math.log(Z)) < 1e-12


def _count_structures(n):
    """Eq. scalar-pf with the hairpin minimum: structures on n bases when any two pair."""
    N = {}

    def q(i, j):
        if i > j:
            return 1
        if (i, j) in N:
            return N[(i, j)]
        v = q(i + 1, j) + sum(q(i + 1, k - 1) * q(k + 1, j) for k in range(i + 4, j + 1))
        N[(i, j)] = v
        return v

    return q(0, n - 1)


def test_scalar_counting_recursion():
    zero = P0.copy()
    zero[:180] = 0.0
    for m in (2, 5, 12):  # n <= 36: the 30-nt loop cap cannot bind
        res = list(np.random.default_rng(m).integers(0, 20, m))
        n = 3 * m
        expect = sum(math.log(len(bf.codons_for(r))) for r in res) + math.log(_count_structures(n))
        assert abs(oracle.inside(zero, res, any_pair=True) - expect) < 1e-10


@pytest.fixture(scope="module")
def mid():
    res, lw, pb = synth.workload("p300_weighted")
    res, lw = res[:25], lw[:25]
    return res, lw, pb, oracle.outside(P0, res, lw, pb)


def test_invariants(mid):
    res, lw, pb, o = mid
    P = o["P"]
    assert np.allclose(P, P.T, atol=1e-14)
    assert P.min() > -1e-14 and P.max() < 1 + 1e-14
    assert np.abs(P.sum(1) - 1).max() < 1e-12
    assert np.abs(o["codon"].sum(1) - 1).max() < 1e-12
    for r in range(len(res)):
        k = len(bf.codons_for(res[r]))
        assert np.all(o["codon"][r, k:] == 0)
    # joint marginals of adjacent residues reduce to the single-residue ones
    T = o["trans"]
    assert np.abs(T.sum(2) - o["codon"][:-1]).max() < 1e-12
    assert np.abs(T.sum(1) - o["codon"][1:]).max() < 1e-12
    assert abs(o["pair_grad"].sum() - (len(res) - 1)) < 1e-10
    bm = oracle.base_marginals(res, o["codon"])
    assert np.abs(bm.sum(1) - 1).max() < 1e-12


def test_codon_marginal_by_clamping(mid):
    res, lw, pb, o = mid
    lz = o["logZ"]
    rng = np.random.default_rng(7)
    for r in rng.choice(len(res), 5, replace=False):
        k = len(bf.codons_for(res[r]))
        for c in range(k):
            lwc = lw.copy()
            lwc[r, [x for x in range(6) if x != c]] = -np.inf
            pc = math.exp(oracle.inside(P0, res, lwc, pb) - lz)
            assert abs(pc - o["codon"][r, c]) < 1e-12


def test_pair_probability_by_forbidding(mid):
    res, lw, pb, o = mid
    P, lz = o["P"], o["logZ"]
    n = 3 * len(res)
    iu = np.argwhere(np.triu(P, 4) > 1e-3)
    rng = np.random.default_rng(8)
    for i, j in iu[rng.choice(len(iu), min(8, len(iu)), replace=False)]:
        allow = np.ones((n, n), dtype=np.uint8)
        allow[i, j] = 0
        pij = 1 - math.exp(oracle.inside(P0, res, lw, pb, allow=allow) - lz)
        assert abs(pij - P[i, j]) < 1e-11


def test_finite_differences(mid):
    res, lw, pb, o = mid
    h = 1e-4
    rng = np.random.default_rng(9)
    for _ in range(6):
        r = int(rng.integers(len(res)))
        c = int(rng.integers(len(bf.codons_for(res[r]))))
        lp, lm = lw.copy(), lw.copy()
        lp[r, c] += h
        lm[r, c] -= h
        fd = (oracle.inside(P0, res, lp, pb) - oracle.inside(P0, res, lm, pb)) / (2 * h)
        assert abs(fd - o["codon"][r, c]) < 1e-7
    g = o["pair_grad"]
    for c1, c2 in np.argwhere(g > 0.05)[:4]:
        pp, pm = pb.copy(), pb.copy()
        pp[c1, c2] += h
        pm[c1, c2] -= h
        fd = (oracle.inside(P0, res, lw, pp) - oracle.inside(P0, res, lw, pm)) / (2 * h)
        assert abs(fd - g[c1, c2]) < 1e-7


def test_sampler_exact_distribution():
    res = [1, 9, 10]
    rng = np.random.default_rng(1)
    lw = rng.normal(0, 0.5, (3, 6))
    pb = rng.normal(0, 0.3, (61, 61))
    b = bf.summary(P0, res, lw, pb)
    probs = {}
    for _, cids, pt, w in b["ensemble"]:
        probs[(cids, pt)] = probs.get((cids, pt), 0.0) + w / b["Z"]
    N = 100000
    cod, par = oracle.sample(P0, res, N, 2024, lw, pb)
    cnt = {}
    for c, x in zip(map(tuple, cod), map(tuple, par)):
        cnt[(c, x)] = cnt.get((c, x), 0) + 1
    assert all(k in probs for k in cnt)
    chi, dof = 0.0, 0
    for k, pr in probs.items():
        e = N * pr
        if e >= 5:
            chi += (cnt.get(k, 0) - e) ** 2 / e
            dof += 1
    # chi-square upper tail ~ 1e-4 via Wilson-Hilferty
    z = ((chi / dof) ** (1 / 3) - (1 - 2 / (9 * dof))) / math.sqrt(2 / (9 * dof))
    assert z < 3.8, (chi, dof)


def test_sampler_marginals(mid):
    res, lw, pb, o = mid
    N = 4000
    cod, par = oracle.sample(P0, res, N, 77, lw, pb)
    n = 3 * len(res)
    for r in range(len(res)):
        ids = oracle.codons_of(res[r])
        for s, cid in enumerate(ids):
            p = o["codon"][r, s]
            f = np.mean(cod[:, r] == cid)
            assert abs(f - p) <= 4.5 * math.sqrt(p * (1 - p) / N) + 1e-9
    emp = np.zeros((n, n))
    for x in par:
        for i, j in enumerate(x):
            emp[i, i if j < 0 else j] += 1
    emp /= N
    sd = np.sqrt(o["P"] * (1 - o["P"]) / N)
    assert np.all(np.abs(emp - o["P"]) <= 4.5 * sd + 2.0 / N)
    assert np.all((par >= -1) & (par < n))
