"""Python binding of the codon-constrained partition-function library (C ABI in
``include/codonfold.h``).

Only argument marshalling lives here: every step of the dynamic program runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.  If the
compiled library is missing the import fails loudly; there is no CPU path.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

from .build import LIB

AMINO_ACIDS = "ARNDCQEGHILKMFPSTWYV"
CF_OK, CF_EINVAL, CF_ENOMEM, CF_ECUDA, CF_ETIMEOUT, CF_ESTATE, CF_ENUMERIC = range(7)
CF_FP64, CF_FP32_SCALED = 0, 1
CF_NPARAMS = 181
_STATUS = {1: "CF_EINVAL", 2: "CF_ENOMEM", 3: "CF_ECUDA", 4: "CF_ETIMEOUT", 5: "CF_ESTATE", 6: "CF_ENUMERIC"}


class CFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _load() -> ctypes.CDLL:
    if not Path(LIB).exists():
        raise ImportError(f"CUDA library not built: {LIB} (run paper_2604_19718_b300.build.build())")
    lib = ctypes.CDLL(str(LIB))
    vp, dp, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
    lib.cf_load_model.argtypes = [dp, ctypes.c_size_t, ctypes.POINTER(vp)]
    lib.cf_model_free.argtypes = [vp]
    lib.cf_problem_create.argtypes = [vp, ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.cf_problem_free.argtypes = [vp]
    lib.cf_set_protein.argtypes = [vp, ctypes.c_char_p, ctypes.c_int, dp, dp]
    lib.cf_set_weights.argtypes = [vp, dp, dp]
    lib.cf_inside.argtypes = [vp, ctypes.c_int, dp]
    lib.cf_outside.argtypes = [vp, fp, vp, vp, vp]
    lib.cf_sample.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, vp, vp]
    lib.cf_last_error.argtypes = [vp]
    lib.cf_last_error.restype = ctypes.c_char_p
    lib.cf_last_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.cf_problem_length.argtypes = [vp]
    lib.cf_window_logz.argtypes = [vp, vp, vp, ctypes.c_int, vp]
    lib.cf_window_logz.restype = ctypes.c_int
    lib.cf_window_last_ms.argtypes = [vp]
    lib.cf_window_last_ms.restype = ctypes.c_float
    lib.cf_surrogate_create.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(vp)]
    lib.cf_surrogate_free.argtypes = [vp]
    lib.cf_surrogate_set_params.argtypes = [vp, vp]
    lib.cf_surrogate_get_params.argtypes = [vp, vp]
    lib.cf_surrogate_predict.argtypes = [vp, vp, vp, ctypes.c_int, vp]
    lib.cf_surrogate_grad.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp, vp]
    lib.cf_surrogate_train_step.argtypes = [vp, vp, vp, ctypes.c_int, vp, ctypes.c_float, vp]
    lib.cf_surrogate_last_ms.argtypes = [vp]
    lib.cf_surrogate_last_ms.restype = ctypes.c_float
    ip = ctypes.POINTER(ctypes.c_int)
    lib.cf_far_band_info.argtypes = [vp, ip, ip, ip, ip, ip]
    lib.cf_debug_set_range_limit.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.cf_debug_set_range_limit.restype = ctypes.c_int
    lib.cf_debug_set_wait_polls.argtypes = [ctypes.c_int, ctypes.c_ulonglong]
    lib.cf_debug_fail_alloc.argtypes = [ctypes.c_longlong]
    lib.cf_debug_set_far_dev_max.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.cf_debug_set_far_dev_max.restype = ctypes.c_int
    lib.cf_surrogate_set_path.argtypes = [vp, ctypes.c_int]
    lib.cf_surrogate_set_path.restype = ctypes.c_int
    lib.cf_debug_classify_pointer.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.cf_debug_classify_pointer.restype = ctypes.c_int
    lib.cf_sample_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, vp, vp]
    lib.cf_mfe.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double), vp, vp]
    lib.cf_set_checkpoint.argtypes = [vp, ctypes.c_int]
    lib.cf_set_checkpoint.restype = ctypes.c_int
    lib.cf_checkpointed.argtypes = [vp]
    lib.cf_checkpointed.restype = ctypes.c_int
    lib.cf_batch_create.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(vp)]
    lib.cf_batch_set_proteins.argtypes = [vp, ctypes.c_char_p, vp, vp]
    lib.cf_batch_run.argtypes = [vp, vp, vp, vp]
    lib.cf_batch_last_ms.argtypes = [vp]
    lib.cf_batch_last_ms.restype = ctypes.c_float
    lib.cf_batch_free.argtypes = [vp]
    for name in ("cf_batch_create", "cf_batch_set_proteins", "cf_batch_run", "cf_batch_free"):
        getattr(lib, name).restype = ctypes.c_int
    lib.cf_mfe_last_ms.argtypes = [vp]
    lib.cf_mfe_last_ms.restype = ctypes.c_float
    lib.cf_subopt_steps.argtypes = [vp]
    lib.cf_subopt_steps.restype = ctypes.c_longlong
    lib.cf_subopt.argtypes = [vp, ctypes.c_double, ctypes.c_int, vp, vp, vp, ctypes.POINTER(ctypes.c_int)]
    lib.cf_subopt.restype = ctypes.c_int
    lib.cf_set_layout.argtypes = [vp, ctypes.c_int]
    lib.cf_layout_states.argtypes = [vp, ctypes.POINTER(ctypes.c_int), vp]
    lib.cf_set_layout.restype = ctypes.c_int
    lib.cf_layout_states.restype = ctypes.c_int
    lib.cf_tm_spectral_radius.argtypes = [dp, ctypes.c_int, dp]
    lib.cf_tm_model_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_int,
                                       ctypes.POINTER(vp)]
    lib.cf_tm_model_radius.argtypes = [vp, dp]
    lib.cf_tm_model_free.argtypes = [vp]
    lib.cf_tm_inside.argtypes = [vp, vp, ctypes.c_int, dp]
    lib.cf_tm_last_ms.argtypes = [vp]
    lib.cf_tm_last_ms.restype = ctypes.c_float
    for name in ("cf_tm_spectral_radius", "cf_tm_model_create", "cf_tm_model_radius", "cf_tm_model_free",
                 "cf_tm_inside"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("cf_far_band_info", "cf_debug_set_wait_polls", "cf_debug_fail_alloc", "cf_sample_noalloc",
                 "cf_mfe"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("cf_surrogate_create", "cf_surrogate_free", "cf_surrogate_set_params", "cf_surrogate_get_params",
                 "cf_surrogate_predict", "cf_surrogate_grad", "cf_surrogate_train_step"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("cf_load_model", "cf_model_free", "cf_problem_create", "cf_problem_free", "cf_set_protein", "cf_set_weights",
                 "cf_inside", "cf_outside", "cf_sample", "cf_last_timing"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


def _check(status: int, handle=None):
    if status != CF_OK:
        msg = lib.cf_last_error(handle)
        raise CFError(status, msg.decode() if msg else "")


def _ptr(a):
    """Address of a numpy array or torch tensor (host or device), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------- C-ABI names

def cf_load_model(params) -> ctypes.c_void_p:
    p = np.ascontiguousarray(params, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib.cf_load_model(p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size, ctypes.byref(h)))
    return h


def cf_model_free(model) -> None:
    lib.cf_model_free(model)


def cf_problem_create(model, device: int = 0, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib.cf_problem_create(model, int(device), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def cf_problem_free(prob) -> None:
    lib.cf_problem_free(prob)


def cf_set_protein(prob, aa: str, codon_logw=None, pair_bonus=None) -> None:
    m = len(aa)
    lw = None if codon_logw is None else np.ascontiguousarray(np.asarray(codon_logw, dtype=np.float64).reshape(m, 6))
    pb = None if pair_bonus is None else np.ascontiguousarray(np.asarray(pair_bonus, dtype=np.float64).reshape(61, 61))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.cf_set_protein(prob, aa.encode(), m, None if lw is None else lw.ctypes.data_as(dp),
                              None if pb is None else pb.ctypes.data_as(dp)), prob)


def cf_set_weights(prob, m: int, codon_logw=None, pair_bonus=None) -> None:
    lw = None if codon_logw is None else np.ascontiguousarray(np.asarray(codon_logw, dtype=np.float64).reshape(m, 6))
    pb = None if pair_bonus is None else np.ascontiguousarray(np.asarray(pair_bonus, dtype=np.float64).reshape(61, 61))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.cf_set_weights(prob, None if lw is None else lw.ctypes.data_as(dp),
                              None if pb is None else pb.ctypes.data_as(dp)), prob)


def cf_inside(prob, precision: int = CF_FP32_SCALED) -> float:
    out = ctypes.c_double()
    _check(lib.cf_inside(prob, int(precision), ctypes.byref(out)), prob)
    return out.value


def cf_outside(prob, pair_prob=None, codon_marg=None, base_marg=None, pair_grad=None) -> None:
    _check(lib.cf_outside(prob, _ptr(pair_prob), _ptr(codon_marg), _ptr(base_marg), _ptr(pair_grad)), prob)


def cf_sample(prob, nsamples: int, seed: int, codons, partner) -> None:
    _check(lib.cf_sample(prob, int(nsamples), ctypes.c_uint64(seed), _ptr(codons), _ptr(partner)), prob)


def cf_last_timing(prob):
    a, b = ctypes.c_float(), ctypes.c_float()
    c, d = ctypes.c_int(), ctypes.c_int()
    _check(lib.cf_last_timing(prob, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), prob)
    return a.value, b.value, c.value, d.value


def cf_problem_length(prob) -> int:
    return int(lib.cf_problem_length(prob))


def cf_window_logz(prob, bases, offsets, logz) -> None:
    """Batched fixed-sequence log Z: bases uint8 (host array or device
    tensor), offsets int64 (nwin + 1), logz float64 (nwin), filled in place."""
    nwin = len(offsets) - 1
    _check(lib.cf_window_logz(prob, _ptr(bases), _ptr(offsets), int(nwin), _ptr(logz)), prob)


def cf_window_last_ms(prob) -> float:
    return float(lib.cf_window_last_ms(prob))


SURROGATE_NPARAMS = 63041
SURROGATE_MAX_LEN = 256


def cf_surrogate_create(device: int = 0, stream: int = 0, max_batch: int = 1024):
    h = ctypes.c_void_p()
    _check(lib.cf_surrogate_create(int(device), ctypes.c_void_p(stream), int(max_batch), ctypes.byref(h)))
    return h


def cf_surrogate_free(sur) -> None:
    lib.cf_surrogate_free(sur)


def cf_surrogate_set_params(sur, params) -> None:
    _check(lib.cf_surrogate_set_params(sur, _ptr(params)))


def cf_surrogate_get_params(sur, params) -> None:
    _check(lib.cf_surrogate_get_params(sur, _ptr(params)))


def cf_surrogate_predict(sur, bases, offsets, G_out) -> None:
    _check(lib.cf_surrogate_predict(sur, _ptr(bases), _ptr(offsets), len(offsets) - 1, _ptr(G_out)))


def cf_surrogate_grad(sur, bases, offsets, G_target, loss_out, grad_out) -> None:
    _check(lib.cf_surrogate_grad(sur, _ptr(bases), _ptr(offsets), len(offsets) - 1, _ptr(G_target),
                                 _ptr(loss_out), _ptr(grad_out)))


def cf_surrogate_train_step(sur, bases, offsets, G_target, lr: float, loss_out=None) -> None:
    _check(lib.cf_surrogate_train_step(sur, _ptr(bases), _ptr(offsets), len(offsets) - 1, _ptr(G_target),
                                       ctypes.c_float(lr), _ptr(loss_out)))


def cf_surrogate_last_ms(sur) -> float:
    return float(lib.cf_surrogate_last_ms(sur))


def cf_sample_noalloc(prob, nsamples: int, seed: int, codons, partner) -> None:
    """Sampler for callers that cannot allocate device memory: outputs must be
    device tensors; scratch comes from the library's static device array."""
    _check(lib.cf_sample_noalloc(prob, int(nsamples), ctypes.c_uint64(seed), _ptr(codons), _ptr(partner)), prob)


def cf_mfe(prob, codons=None, partner=None):
    """Minimum free energy: (integer cost in 2^-32 kcal/mol, kcal/mol); codons
    (m int32) and partner (n int32), host arrays or device tensors, are filled
    with one minimiser when given."""
    q = ctypes.c_int64()
    k = ctypes.c_double()
    _check(lib.cf_mfe(prob, ctypes.byref(q), ctypes.byref(k), _ptr(codons), _ptr(partner)), prob)
    return q.value, k.value


def cf_set_checkpoint(prob, mode: int) -> None:
    """-1 automatic (from CF_CHECKPOINT_MIN_N bases), 0 store the interior
    partial sums whole, 1 checkpoint them every 64 diagonals."""
    _check(lib.cf_set_checkpoint(prob, int(mode)), prob)


def cf_checkpointed(prob) -> bool:
    return bool(lib.cf_checkpointed(prob))


def cf_mfe_last_ms(prob) -> float:
    return float(lib.cf_mfe_last_ms(prob))


def cf_subopt_steps(prob) -> int:
    """Search steps (element expansions) of the last cf_subopt."""
    return int(lib.cf_subopt_steps(prob))


def cf_subopt(prob, m: int, n: int, gap_kcal: float, max_out: int):
    """(count, costs [k], codons [k][m], partners [k][n]) of the configurations
    within gap_kcal of the minimum (k = min(count, max_out); count is
    max_out + 1 when there are more)."""
    cost = np.zeros(max(max_out, 1), dtype=np.int64)
    cod = np.zeros((max(max_out, 1), m), dtype=np.int32)
    par = np.zeros((max(max_out, 1), n), dtype=np.int32)
    cnt = ctypes.c_int()
    _check(lib.cf_subopt(prob, float(gap_kcal), int(max_out), ctypes.c_void_p(cost.ctypes.data),
                         ctypes.c_void_p(cod.ctypes.data), ctypes.c_void_p(par.ctypes.data), ctypes.byref(cnt)), prob)
    k = min(cnt.value, max_out)
    return cnt.value, cost[:k], cod[:k], par[:k]


def cf_set_layout(prob, layout: int) -> None:
    """0 codon states (default), 1 the single-codon layout; takes effect at
    the next cf_set_protein."""
    _check(lib.cf_set_layout(prob, int(layout)), prob)


def cf_layout_states(prob, n: int):
    """(layout of the current protein, per-position state counts)."""
    lay = ctypes.c_int()
    st = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib.cf_layout_states(prob, ctypes.byref(lay), ctypes.c_void_p(st.ctypes.data)), prob)
    return lay.value, st[:n]


def _dbl(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def cf_tm_spectral_radius(A) -> float:
    A, pa = _dbl(A)
    out = ctypes.c_double()
    _check(lib.cf_tm_spectral_radius(pa, int(A.shape[0]), ctypes.byref(out)))
    return out.value


def cf_tm_model_create(V, B, S, normalize: bool = True, device: int = 0) -> ctypes.c_void_p:
    """V: 4 x g x g, B: nrho x 4 x 4 x g x g, S: g x g (binary64)."""
    V, pv = _dbl(V)
    B, pb = _dbl(B)
    S, ps = _dbl(S)
    h = ctypes.c_void_p()
    _check(lib.cf_tm_model_create(int(device), int(V.shape[1]), int(B.shape[0]), pv, pb, ps, int(bool(normalize)),
                                  ctypes.byref(h)))
    return h


def cf_tm_model_radius(model) -> np.ndarray:
    out = np.zeros(4)
    _check(lib.cf_tm_model_radius(model, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def cf_tm_model_free(model) -> None:
    lib.cf_tm_model_free(model)


def cf_tm_inside(prob, model, precision: int = CF_FP32_SCALED) -> float:
    out = ctypes.c_double()
    _check(lib.cf_tm_inside(prob, model, int(precision), ctypes.byref(out)), prob)
    return out.value


def cf_tm_last_ms(prob) -> float:
    return float(lib.cf_tm_last_ms(prob))


class TensorModel:
    """A tensor-based free energy model on one device (owns the handle)."""

    def __init__(self, V, B, S, normalize: bool = True, device: int = 0):
        self.h = cf_tm_model_create(V, B, S, normalize, device)

    def radius(self) -> np.ndarray:
        return cf_tm_model_radius(self.h)

    def close(self):
        if self.h:
            cf_tm_model_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cf_far_band_info(prob):
    """(inside largest chord departure, inside bands summed term by term,
    outside largest departure, outside gathered term by term, spread of the
    interval strengths in bits) of the last binary32 passes."""
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib.cf_far_band_info(prob, *[ctypes.byref(x) for x in v]), prob)
    return tuple(x.value for x in v)


def cf_debug_set_wait_polls(device: int, polls: int) -> None:
    _check(lib.cf_debug_set_wait_polls(int(device), ctypes.c_ulonglong(polls)))


def cf_debug_set_far_dev_max(device: int, bound: int) -> None:
    _check(lib.cf_debug_set_far_dev_max(int(device), int(bound)))


def cf_surrogate_set_path(sur, path: int) -> None:
    """Prediction path: 0 CUDA cores (FP32 activations), 1 tensor cores."""
    _check(lib.cf_surrogate_set_path(sur, int(path)))


FAR_DEV_MAX_DEFAULT = 48


RANGE_LIMIT_DEFAULT = 120
RANGE_MAXLEN_DEFAULT = 400


def cf_debug_set_range_limit(device: int, bits: int, max_length: int = RANGE_MAXLEN_DEFAULT) -> None:
    _check(lib.cf_debug_set_range_limit(int(device), int(bits), int(max_length)))


def cf_debug_fail_alloc(after: int) -> None:
    _check(lib.cf_debug_fail_alloc(int(after)))


def cf_debug_classify_pointer(memory_type: int, pointer_device: int, problem_device: int) -> int:
    return int(lib.cf_debug_classify_pointer(int(memory_type), int(pointer_device), int(problem_device)))


WAIT_POLLS_DEFAULT = 1 << 22


# ---------------------------------------------------------------- convenience

def to_letters(residues) -> str:
    return "".join(AMINO_ACIDS[int(r)] for r in residues)


_AA_BYTES = np.frombuffer(AMINO_ACIDS.encode(), dtype=np.uint8)


class Batch:
    """A batch of proteins of one length: inside and outside for all of them
    in one launch per kernel (cf_batch_*)."""

    def __init__(self, params, nprot: int, m: int, precision: int = CF_FP32_SCALED, device: int = 0,
                 stream: int = 0):
        self.model = cf_load_model(params)
        self.h = ctypes.c_void_p()
        _check(lib.cf_batch_create(self.model, int(device), ctypes.c_void_p(stream), int(nprot), int(m),
                                   int(precision), ctypes.byref(self.h)))
        self.nprot, self.m, self.n = nprot, m, 3 * m

    def set_proteins(self, proteins, codon_logw=None, pair_bonus=None):
        """proteins: nprot residue lists (or strings) of m residues, or one
        (nprot, m) integer array of residue indices."""
        if isinstance(proteins, np.ndarray) or (len(proteins) and not isinstance(proteins[0], str)):
            idx = np.asarray(proteins)
            if idx.shape != (self.nprot, self.m) or idx.dtype.kind not in "iu":
                raise ValueError("expected nprot proteins of m residues")
            if idx.size and (idx.min() < 0 or idx.max() >= len(AMINO_ACIDS)):
                raise ValueError("residue index out of range")
            letters = _AA_BYTES[idx].tobytes()
        else:
            letters = "".join(proteins).encode()
        if len(letters) != self.nprot * self.m:
            raise ValueError("expected nprot proteins of m residues")
        lw = None if codon_logw is None else np.ascontiguousarray(codon_logw, dtype=np.float64).reshape(
            self.nprot, self.m, 6)
        pb = None if pair_bonus is None else np.ascontiguousarray(pair_bonus, dtype=np.float64).reshape(61, 61)
        _check(lib.cf_batch_set_proteins(self.h, letters, _ptr(lw), _ptr(pb)))

    def run(self, pair_prob=True, codon=True):
        """Inside and outside of every protein.  pair_prob / codon: True (new
        arrays), False (not copied out), or the caller's C-contiguous output
        array ((nprot, n, n) float32 / (nprot, m, 6) float64, host or this
        device's memory), reused across runs."""
        lz = np.zeros(self.nprot)
        P = np.zeros((self.nprot, self.n, self.n), dtype=np.float32) if pair_prob is True else pair_prob
        cm = np.zeros((self.nprot, self.m, 6)) if codon is True else codon
        for arr, shape, dt in ((P, (self.nprot, self.n, self.n), "float32"), (cm, (self.nprot, self.m, 6), "float64")):
            if arr is False:
                continue
            ok = tuple(arr.shape) == shape and str(arr.dtype).endswith(dt)
            ok = ok and (arr.is_contiguous() if hasattr(arr, "is_contiguous") else arr.flags.c_contiguous)
            if not ok:
                raise ValueError(f"output array must be C-contiguous {dt} of shape {shape}")
        _check(lib.cf_batch_run(self.h, _ptr(lz), None if P is False else _ptr(P), None if cm is False else _ptr(cm)))
        return lz, P, cm

    def last_ms(self) -> float:
        return float(lib.cf_batch_last_ms(self.h))

    def close(self):
        if self.h:
            lib.cf_batch_free(self.h)
            self.h = None
        if self.model:
            cf_model_free(self.model)
            self.model = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """The window free-energy surrogate on one device (numpy conveniences)."""

    def __init__(self, params, device: int = 0, stream: int = 0, max_batch: int = 1024):
        self.h = cf_surrogate_create(device, stream, max_batch)
        self.max_batch = max_batch
        self.set_params(params)

    def set_params(self, params):
        cf_surrogate_set_params(self.h, np.ascontiguousarray(params, dtype=np.float32))

    def params(self) -> np.ndarray:
        out = np.zeros(SURROGATE_NPARAMS, dtype=np.float32)
        cf_surrogate_get_params(self.h, out)
        return out

    def predict(self, bases, offsets) -> np.ndarray:
        out = np.zeros(len(offsets) - 1, dtype=np.float32)
        cf_surrogate_predict(self.h, np.ascontiguousarray(bases, dtype=np.uint8),
                             np.ascontiguousarray(offsets, dtype=np.int64), out)
        return out

    def grad(self, bases, offsets, G):
        loss = np.zeros(1, dtype=np.float32)
        g = np.zeros(SURROGATE_NPARAMS, dtype=np.float32)
        cf_surrogate_grad(self.h, np.ascontiguousarray(bases, dtype=np.uint8),
                          np.ascontiguousarray(offsets, dtype=np.int64),
                          np.ascontiguousarray(G, dtype=np.float32), loss, g)
        return float(loss[0]), g

    def train_step(self, bases, offsets, G, lr: float) -> float:
        loss = np.zeros(1, dtype=np.float32)
        cf_surrogate_train_step(self.h, np.ascontiguousarray(bases, dtype=np.uint8),
                                np.ascontiguousarray(offsets, dtype=np.int64),
                                np.ascontiguousarray(G, dtype=np.float32), lr, loss)
        return float(loss[0])

    def close(self):
        if self.h:
            cf_surrogate_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CodonFold:
    """One protein on one device/stream; owns a model and a problem handle."""

    def __init__(self, params, device: int = 0, stream: int = 0):
        self.model = cf_load_model(params)
        self.prob = cf_problem_create(self.model, device, stream)
        self.n = 0
        self.m = 0

    def set_protein(self, residues_or_letters, codon_logw=None, pair_bonus=None):
        aa = residues_or_letters if isinstance(residues_or_letters, str) else to_letters(residues_or_letters)
        cf_set_protein(self.prob, aa, codon_logw, pair_bonus)
        self.m = len(aa)
        self.n = 3 * self.m
        return self

    def set_weights(self, codon_logw=None, pair_bonus=None):
        cf_set_weights(self.prob, self.m, codon_logw, pair_bonus)
        return self

    def inside(self, precision: int = CF_FP32_SCALED) -> float:
        return cf_inside(self.prob, precision)

    def outside(self, pair_prob=True, codon=True, pair_grad=True, base=None):
        """Host numpy outputs (pass arrays/tensors to fill them in place
        instead; False skips an output).  Returns (P, codon marginals, pair
        gradient), and the per-base marginals (n x 4) as a fourth item when
        ``base`` is given (True or an array to fill)."""
        P = np.zeros((self.n, self.n), dtype=np.float32) if pair_prob is True else pair_prob
        cm = np.zeros((self.m, 6)) if codon is True else codon
        pg = np.zeros((61, 61)) if pair_grad is True else pair_grad
        bm = np.zeros((self.n, 4)) if base is True else base
        cf_outside(self.prob, None if P is False else P, None if cm is False else cm,
                   None if bm is None or bm is False else bm, None if pg is False else pg)
        return (P, cm, pg) if base is None else (P, cm, pg, bm)

    def sample(self, nsamples: int, seed: int):
        cod = np.zeros((nsamples, self.m), dtype=np.int32)
        par = np.zeros((nsamples, self.n), dtype=np.int32)
        cf_sample(self.prob, nsamples, seed, cod, par)
        return cod, par

    def mfe(self, traceback: bool = True):
        """(cost, kcal/mol, codons[m] sense ids, partner[n]) of the minimum
        free energy configuration (None, None without traceback)."""
        cod = np.zeros(self.m, dtype=np.int32) if traceback else None
        par = np.zeros(self.n, dtype=np.int32) if traceback else None
        q, k = cf_mfe(self.prob, cod, par)
        return q, k, cod, par

    def subopt(self, gap_kcal: float, max_out: int = 1000):
        """Configurations within gap_kcal of the minimum free energy (cf_subopt)."""
        return cf_subopt(self.prob, self.m, self.n, gap_kcal, max_out)

    def tm_inside(self, model: "TensorModel", precision: int = CF_FP32_SCALED) -> float:
        """log Z of the protein under a tensor-based model (cf_tm_inside)."""
        return cf_tm_inside(self.prob, model.h, precision)

    def timing(self):
        return cf_last_timing(self.prob)

    def close(self):
        if self.prob:
            cf_problem_free(self.prob)
            self.prob = None
        if self.model:
            cf_model_free(self.model)
            self.model = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
