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
    # the trajectory calls reject a null context before touching the device
    d = ctypes.c_double()
    assert lib.rhmc_gauge_action(None, None, 5.12, ctypes.byref(d), None) == 1
    assert lib.rhmc_kinetic_energy(None, None, ctypes.byref(d), None) == 1
    assert lib.rhmc_momenta_from_normals(None, None, None, None) == 1
    assert lib.rhmc_gauge_momentum(None, None, None, 5.12, 0.1, None) == 1
    assert lib.rhmc_momentum_update(None, None, None, None, 0.1, None) == 1
    assert lib.rhmc_link_update(None, None, None, 0.1, None) == 1
    prm = _lib.MdParams(5.12, 1.0, 10, 3, 1.0 / 6, 1e-7, 0, 1)
    assert lib.rhmc_md_evolve(None, None, None, None, 0, None, ctypes.byref(prm), None, None) == 1
    assert lib.rhmc_hmc_trajectory(None, None, None, None, 0, None, None, None, ctypes.byref(prm), 1e-14, 0.5, None,
                                   None, None) == 1
    assert b"null context" in lib.rhmc_last_error()


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


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's sizes and field
    offsets (compiled with gcc against include/rhmc.h; no GPU)."""
    import shutil
    import subprocess

    from paper_1808_01829_gb300 import _lib

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = {
        "rhmc_lattice_t": (_lib.Lattice, ["dims", "mass", "bc_t"]),
        "rhmc_info_t": (_lib.Info, ["iters", "dirac_calls", "reliable_updates", "refinements", "refine_iters",
                                    "true_rel_resid_max", "phase1_rel_resid_max", "per_shift_resid", "phase1_ms",
                                    "refine_ms"]),
        "rhmc_rational_t": (_lib.Rational, ["n_shifts", "alpha0", "alpha", "beta"]),
        "rhmc_md_params_t": (_lib.MdParams, ["beta", "tau", "n_steps", "n_gauge", "lambda", "tol_md", "max_iter",
                                             "precision_md"]),
        "rhmc_md_info_t": (_lib.MdInfo, ["force_evals", "gauge_force_evals", "solver_iters", "dirac_calls",
                                         "max_rel_resid"]),
        "rhmc_hmc_info_t": (_lib.HmcInfo, ["H_old", "H_new", "dH", "K", "S_g", "S_f", "accepted", "md"]),
    }
    lines = ['#include <stdio.h>', '#include "rhmc.h"', "int main(void) {"]
    for cname, (_, fields) in checks.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
               if l)
    for cname, (cls, fields) in checks.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, (pyname, _) in zip(fields, cls._fields_):
            assert int(got[f"{cname}.{f}"]) == getattr(cls, pyname).offset, (cname, f)
