"""The C-ABI library loads and exports every entry point its header declares
(no compute: runs without a GPU)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def _declared():
    names = []
    for h in sorted((ROOT / "include").glob("*.h")):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names += re.findall(r"\b(cf_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_header_symbols():
    from paper_2604_19718_b300 import build
    lib = ctypes.CDLL(str(build.build()))
    names = _declared()
    assert "cf_inside" in names and "cf_outside" in names and "cf_sample" in names
    for name in names:
        assert hasattr(lib, name), f"missing export {name}"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib

    import paper_2604_19718_b300.build as b
    monkeypatch.setattr(b, "LIB", tmp_path / "missing.so")
    import paper_2604_19718_b300 as pkg
    monkeypatch.setattr(pkg, "LIB", tmp_path / "missing.so")
    try:
        pkg._load()
    except ImportError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("expected ImportError")
    importlib.reload(b)


def test_cpu_side_argument_checks():
    import numpy as np

    import paper_2604_19718_b300 as cf
    import synth
    bad = np.ones(10)
    try:
        cf.cf_load_model(bad)
    except cf.CFError as e:
        assert e.status == cf.CF_EINVAL
    else:
        raise AssertionError("expected CF_EINVAL")
    p = synth.nn_params(0)
    p[3] = np.inf
    try:
        cf.cf_load_model(p)
    except cf.CFError as e:
        assert e.status == cf.CF_EINVAL
    else:
        raise AssertionError("expected CF_EINVAL")
    m = cf.cf_load_model(synth.nn_params(0))
    cf.cf_model_free(m)


def test_pointer_rule_rejects_other_device_memory():
    """The rule the library applies to caller buffers before any launch:
    host memory is staged, device memory of the problem's device (or managed
    memory) is used in place, device memory of another device is rejected
    (CF_EINVAL) so that no kernel of the problem touches it."""
    import paper_2604_19718_b300 as cf
    host, device, managed = 1, 2, 3  # cudaMemoryType values
    unregistered = 0
    assert cf.cf_debug_classify_pointer(unregistered, -1, 0) == 0
    assert cf.cf_debug_classify_pointer(host, 0, 0) == 0
    assert cf.cf_debug_classify_pointer(device, 0, 0) == 1
    assert cf.cf_debug_classify_pointer(device, 1, 1) == 1
    assert cf.cf_debug_classify_pointer(device, 1, 0) == -1
    assert cf.cf_debug_classify_pointer(device, 0, 3) == -1
    assert cf.cf_debug_classify_pointer(managed, 1, 0) == 1


def test_noalloc_scratch_size_matches_header():
    """CF_NOALLOC_SCRATCH_BYTES as the header computes it: error word, per-warp
    states and per-warp stacks at the stated limits."""
    text = (ROOT / "include" / "codonfold.h").read_text()
    max_n = int(re.search(r"#define CF_NOALLOC_MAX_N (\d+)", text).group(1))
    warps = int(re.search(r"#define CF_NOALLOC_WARPS (\d+)", text).group(1))
    want = 256 + (warps * max_n * 4 + 255) // 256 * 256 + warps * (max_n + 64) * 8
    assert want == 4673792
    assert "4,673,792" in text
