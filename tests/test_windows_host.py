"""Host side of the window workload: the generator's codon table and window
layout (no GPU)."""
import numpy as np

import bruteforce as bf
import synth

BASES = "ACGU"


def test_codon_table_is_the_standard_code():
    table = synth.codon_table()
    assert sum(len(c) for c in table) == 61
    for k in range(20):
        got = ["".join(BASES[b] for b in c) for c in table[k]]
        assert got == bf.codons_for(k)


def test_windows_layout():
    res, slots, bases, off = synth.windows(500, seed=3)
    lens = np.diff(off)
    assert off[0] == 0 and off[-1] == len(bases)
    assert lens.min() >= 60 and lens.max() <= 240 and np.all(lens % 3 == 0)
    table = synth.codon_table()
    for w in (0, 17, 499):
        seq = bases[off[w]:off[w + 1]].reshape(-1, 3)
        for r, s, c in zip(res[w], slots[w], seq):
            assert tuple(c) == table[r][s]
    assert np.array_equal(synth.windows(500, seed=3)[2], bases)  # seeded


def test_screen_packing_matches_generator():
    from paper_2604_19718_b300 import screen
    res, slots, bases, off = synth.windows(20, seed=8)
    for w in range(20):
        assert np.array_equal(screen.bases_of(res[w], slots[w]), bases[off[w]:off[w + 1]])
    c = np.stack([slots[3], slots[3], slots[3]])
    b, o = screen._pack(res[3], c)
    assert np.array_equal(o, np.arange(4) * len(slots[3]) * 3)
    assert np.array_equal(b[o[2]:o[3]], bases[off[3]:off[4]])
    rng = np.random.default_rng(0)
    u = screen.uniform_candidates(res[3], 500, rng)
    M = np.array([len(screen.CODONS[r]) for r in res[3]])
    assert u.shape == (500, len(res[3])) and np.all(u >= 0) and np.all(u < M)
    assert screen.CODONS == [list(c) for c in synth.codon_table()]
