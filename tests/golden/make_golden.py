"""Write the oracle's expected values for the full-size workloads.

Calls only ``oracle`` and ``synth``; nothing here touches the CUDA library.
Each output ``<workload>.npz`` holds: logZ, codon marginals (m x 6 by slot),
the codon-pair gradient (61 x 61), the unpaired probabilities (n), the whole
pair-probability matrix (n x n, stored as binary32: its rounding, at most
6e-8, is below every tolerance the tests apply to P) and the oracle's wall
time.  Run:  python tests/golden/make_golden.py [name ...]
"""
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = Path(__file__).resolve().parent

JOBS = {
    # 300 aa, Dirichlet(1) composition, no soft weights
    "p300_dirichlet": lambda: synth.workload("p300_dirichlet"),
    # the same protein with codon log-weights and codon-pair bonuses
    "p300_weighted": lambda: synth.workload("p300_weighted"),
    # 150-aa prefix of the 1000-aa protein with codon log-weights
    "p1000_weighted_prefix150": lambda: tuple(
        None if x is None else x[:150] for x in synth.workload("p1000_weighted")[:2]) + (None,),
}


def main(names):
    params = synth.nn_params(0)
    for name in names:
        res, lw, pb = JOBS[name]()
        t = time.time()
        o = oracle.outside(params, res, lw, pb)
        dt = time.time() - t
        n = 3 * len(res)
        np.savez_compressed(OUT / f"{name}.npz", logZ=o["logZ"], codon=o["codon"],
                            pair_grad=o["pair_grad"], unpaired=np.diag(o["P"]).copy(),
                            P=o["P"].astype(np.float32), n=n, seconds=dt)
        print(f"{name}: logZ={o['logZ']:.12f}  ({dt:.1f} s)", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(JOBS))
