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
