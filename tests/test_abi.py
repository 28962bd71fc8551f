"""The C-ABI library builds, loads and exports every symbol include/rhmc.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "rhmc.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:rhmc_status_t|size_t|const char \*|long long|int)\s*(rhmc_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1808_01829_gb300 import _build, _lib

    _build.build()
    return _lib.load()


def test_all_declared_symbols_exported(lib):
    names = _declared()
    assert "rhmc_block_multishift_cg" in names and "rhmc_force" in names and "rhmc_apply_mdagm_mrhs" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_lists_match_header(lib):
    from paper_1808_01829_gb300 import _lib

    assert set(_lib.exported_symbols()) <= set(_declared())


def test_invalid_arguments_rejected_without_gpu(lib):
    """Argument checks run before any CUDA call."""
    from paper_1808_01829_gb300 import _lib

    h = ctypes.c_void_p()
    lat = _lib.Lattice((ctypes.c_int * 4)(4, 3, 4, 4), 0.1, -1)  # odd extent
    assert lib.rhmc_create(ctypes.byref(h), ctypes.byref(lat), 0) == 1
    assert b"even" in lib.rhmc_last_error()
    assert lib.rhmc_create(None, ctypes.byref(lat), 0) == 1
    assert lib.rhmc_workspace_bytes(None, 2, 4, 0) == 0
    assert lib.rhmc_destroy(None) == 0


def test_python_constants_match_header():
    """The tune keys and precision codes the binding names equal the header's enums,
    and the library's key count covers every key the header declares."""
    from paper_1808_01829_gb300 import _lib

    with open(os.path.join(ROOT, "include", "rhmc.h")) as f:
        src = f.read()
    enums = {k: int(v) for k, v in re.findall(r"^\s*(RHMC_[A-Z0-9_]+)\s*=\s*(\d+)", src, re.M)}
    for name in dir(_lib):
        if name.startswith("RHMC_TUNE_") or name in ("RHMC_FP64", "RHMC_MIXED_FP32"):
            assert enums[name] == getattr(_lib, name), name
    with open(os.path.join(ROOT, "paper_1808_01829_gb300", "csrc", "common.cuh")) as f:
        cuh = f.read()
    body = cuh[cuh.index("TUNE_HOP_RHS_PER_THREAD = 0"):cuh.index("TUNE_NKEYS")]
    internal = re.findall(r"^\s*(TUNE_[A-Z0-9_]+)", body, re.M)
    header = sorted(((v, k) for k, v in enums.items() if k.startswith("RHMC_TUNE_")))
    assert [k[len("RHMC_"):] for _, k in header] == internal
