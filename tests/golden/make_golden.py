"""Write the oracle's expected values for the full-size workloads.

Calls only ``oracle`` and ``synth``; nothing here touches the CUDA library.
Each output ``<workload>.npz`` holds: logZ, codon marginals (m x 6 by slot),
the codon-pair gradient (61 x 61), the unpaired probabilities (n), the whole
pair-probability matrix (n x n, stored as binary32: its rounding, at most
6e-8, is below every tolerance the tests apply to P) and the oracle's wall
time.  ``mfe_<workload>.npz`` holds the oracle's minimum free energy (integer
cost in 2^-32 kcal/mol and kcal/mol) and its minimiser.
Run:  python tests/golden/make_golden.py [name ...]
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
    # 100 lysines then 100 aa: beyond the binary32 range (binary64 only)
    "p200_bent": lambda: synth.workload("p200_bent"),
    # 150-aa prefix of the 1000-aa protein with codon log-weights
    "p1000_weighted_prefix150": lambda: tuple(
        None if x is None else x[:150] for x in synth.workload("p1000_weighted")[:2]) + (None,),
}


def mfe_job(name):
    """Minimum free energy (integer cost in 2^-32 kcal/mol) of a workload."""
    params = synth.nn_params(0)
    res, lw, pb = synth.workload(name[len("mfe_"):])
    t = time.time()
    q, kc, cod, par = oracle.mfe(params, res, lw, pb)
    dt = time.time() - t
    np.savez_compressed(OUT / f"{name}.npz", cost=np.int64(q), kcal=kc, codons=cod, partner=par, seconds=dt)
    print(f"{name}: mfe={kc:.12f} kcal/mol  ({dt:.1f} s)", flush=True)


MFE_JOBS = ["mfe_p300_weighted"]


def main(names):
    params = synth.nn_params(0)
    for name in names:
        if name in MFE_JOBS:
            mfe_job(name)
            continue
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
    main(sys.argv[1:] or list(JOBS) + MFE_JOBS)
