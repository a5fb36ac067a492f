"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow reference for the codon-constrained nearest-neighbour partition
function (C ``long double``, no rescaling; see ``codonfold_oracle.c`` for the
model and the recursions).  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the CUDA library
shares no code with it.

Functions cite the paper's sections: log Z (Section "Probability
distributions", Eq. amino-q), pair probabilities (Eq. pair-probability),
codon marginals (Eq. marginal-codon), base marginals (Eq. marginal-base),
sampling (Section "Sequence sampling") and the minimum free energy
configuration (Section "Minimization", Eq. min-problem).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "codonfold_oracle.c"
_BUILD = _HERE / "_build"
_LIB = _BUILD / "liboracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (OpenMP over the cells of one diagonal)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"liboracle.{os.getpid()}.so"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", str(tmp), str(_SRC), "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(str(build()))
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        up = ctypes.POINTER(ctypes.c_ubyte)
        _lib.or_inside.argtypes = [dp, ip, ctypes.c_int, dp, dp, up, ctypes.c_int, dp]
        _lib.or_outside.argtypes = [dp, ip, ctypes.c_int, dp, dp, up, ctypes.c_int, dp, dp, dp, dp, dp]
        _lib.or_sample.argtypes = [dp, ip, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_uint64, ip, ip]
        _lib.or_codons_of.argtypes = [ctypes.c_int, ip]
        _lib.or_mfe.argtypes = [dp, ip, ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_longlong), dp, ip, ip]
    return _lib


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _prep(params, residues, lw, pb):
    params = np.ascontiguousarray(params, dtype=np.float64)
    res = np.ascontiguousarray(residues, dtype=np.int32)
    m = int(res.size)
    lw = None if lw is None else np.ascontiguousarray(np.asarray(lw, dtype=np.float64).reshape(m, 6))
    pb = None if pb is None else np.ascontiguousarray(np.asarray(pb, dtype=np.float64).reshape(61, 61))
    return params, res, m, lw, pb


def codons_of(aa: int) -> list[int]:
    out = np.zeros(6, dtype=np.int32)
    k = _load().or_codons_of(int(aa), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return [int(x) for x in out[:k]]


def inside(params, residues, lw=None, pb=None, allow=None, any_pair=False) -> float:
    """log Z (natural log).  ``allow`` is an optional n x n 0/1 mask of permitted pairs."""
    params, res, m, lw, pb = _prep(params, residues, lw, pb)
    out = ctypes.c_double()
    al = None
    if allow is not None:
        al = np.ascontiguousarray(allow, dtype=np.uint8)
    rc = _load().or_inside(_dptr(params), res.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), m,
                           _dptr(lw), _dptr(pb),
                           None if al is None else al.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                           int(any_pair), ctypes.byref(out))
    if rc:
        raise RuntimeError(f"oracle inside failed with status {rc}")
    return out.value


def outside(params, residues, lw=None, pb=None, allow=None, any_pair=False) -> dict:
    """Inside + hand-written adjoint: log Z, P (n x n, diagonal = unpaired),
    codon marginals (m x 6 by codon slot), d logZ / d pb (61 x 61) and the joint
    codon marginals of adjacent residues ((m-1) x 6 x 6)."""
    params, res, m, lw, pb = _prep(params, residues, lw, pb)
    n = 3 * m
    P = np.zeros((n, n))
    pc = np.zeros((m, 6))
    pp = np.zeros((61, 61))
    pt = np.zeros((max(m - 1, 1), 6, 6))
    out = ctypes.c_double()
    al = None
    if allow is not None:
        al = np.ascontiguousarray(allow, dtype=np.uint8)
    rc = _load().or_outside(_dptr(params), res.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), m,
                            _dptr(lw), _dptr(pb),
                            None if al is None else al.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                            int(any_pair), ctypes.byref(out), _dptr(P), _dptr(pc), _dptr(pp), _dptr(pt))
    if rc:
        raise RuntimeError(f"oracle outside failed with status {rc}")
    return {"logZ": out.value, "P": P, "codon": pc, "pair_grad": pp, "trans": pt[: max(m - 1, 0)]}


def base_marginals(residues, codon_marg) -> np.ndarray:
    """p_i(b) = sum of the marginals of the residue's codons carrying b at i (Eq. marginal-base)."""
    res = np.asarray(residues)
    m = res.size
    out = np.zeros((3 * m, 4))
    for r in range(m):
        cods = codons_of(int(res[r]))
        for s, cid in enumerate(cods):
            c64 = sense_to_codon64(cid)
            for off in range(3):
                out[3 * r + off, (c64 >> (2 * (2 - off))) & 3] += codon_marg[r, s]
    return out


def sense_to_codon64(cid: int) -> int:
    code = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF"
    k = -1
    for c64 in range(64):
        if code[c64] != "*":
            k += 1
            if k == cid:
                return c64
    raise ValueError(cid)


def sample(params, residues, nsamples: int, seed: int, lw=None, pb=None):
    """Exact samples: (codons[ns, m] sense codon ids, partner[ns, n], -1 unpaired)."""
    params, res, m, lw, pb = _prep(params, residues, lw, pb)
    n = 3 * m
    cod = np.zeros((nsamples, m), dtype=np.int32)
    par = np.zeros((nsamples, n), dtype=np.int32)
    rc = _load().or_sample(_dptr(params), res.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), m,
                           _dptr(lw), _dptr(pb), int(nsamples), ctypes.c_uint64(seed),
                           cod.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                           par.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc:
        raise RuntimeError(f"oracle sampler failed with status {rc}")
    return cod, par


Q_SCALE = 4294967296.0  # MFE costs are integers in units of 2^-32 kcal/mol


def mfe(params, residues, lw=None, pb=None, traceback=True):
    """Minimum over (codon sequence, structure) of E - kT (sum lw + sum pb) in
    kcal/mol, by the min-sum recursions on integer costs (2^-32 kcal/mol).
    Returns (mfe_q integer cost, mfe in kcal/mol, codons[m] sense ids,
    partner[n]) of one minimiser (None, None without traceback)."""
    params, res, m, lw, pb = _prep(params, residues, lw, pb)
    n = 3 * m
    q = ctypes.c_longlong()
    kc = ctypes.c_double()
    cod = np.zeros(m, dtype=np.int32) if traceback else None
    par = np.zeros(n, dtype=np.int32) if traceback else None
    ip = ctypes.POINTER(ctypes.c_int)
    rc = _load().or_mfe(_dptr(params), res.ctypes.data_as(ip), m, _dptr(lw), _dptr(pb), ctypes.byref(q),
                        ctypes.byref(kc), None if cod is None else cod.ctypes.data_as(ip),
                        None if par is None else par.ctypes.data_as(ip))
    if rc:
        raise RuntimeError(f"oracle mfe failed with status {rc}")
    return q.value, kc.value, cod, par
