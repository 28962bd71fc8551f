"""GPU parity of SBCGrQ (Algorithm 1), the per-vector SCG baseline and the
force (Eqs. (RA), (force)) against the FP64 oracle.

Criteria: every (shift, column) FP64 true residual <= tol (computed here with
the oracle's operator), and ||X_gpu - X_orc|| <= tol ||B|| / (4m^2 + sigma_s)
+ 1e-10 ||X_orc|| per column (the solution error a residual tol allows,
lambda_min >= 4m^2), with the oracle solved to 1e-13.  Force: the oracle's
force from the GPU's own X matches to 1e-12 (kernel-level parity); the full
GPU force matches the oracle's within the solution-error bound."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_solution, colrel, make_ctx, need_gpu, to_gpu
from paper_1808_01829_gb300 import synthetic as syn
from paper_1808_01829_gb300.remez import rational_approx

pytestmark = pytest.mark.gpu


def _check_solution(dims, mass, U, B, shifts, Xg, tol, Xo):
    check_solution(dims, mass, U, B, shifts, Xg, tol, Xo)


CONFIGS = [
    # dims, mass, n, (r, a, b, N), eps, tol, precision
    ((4, 4, 4, 4), 0.1, 2, (-1.0 / 8, 1e-3, 64.0, 8), 0.3, 1e-10, "fp64"),
    ((4, 4, 4, 4), 0.1, 2, (-1.0 / 8, 1e-3, 64.0, 8), 0.3, 1e-8, "mixed"),
    ((8, 8, 8, 8), 0.05, 4, (-1.0 / 16, 2e-3, 64.0, 12), 0.5, 1e-10, "fp64"),
    ((8, 8, 8, 8), 0.05, 4, (-1.0 / 16, 2e-3, 64.0, 12), 0.5, 1e-8, "mixed"),
    ((4, 6, 4, 8), 0.03, 5, (-1.0 / 20, 1e-3, 64.0, 6), 0.5, 1e-9, "mixed"),
    # widths whose rows do not tile a warp evenly (3, 6, 12 lanes per row group)
    ((4, 4, 4, 4), 0.1, 3, (-1.0 / 12, 1e-3, 64.0, 5), 0.5, 1e-9, "mixed"),
    ((4, 4, 4, 6), 0.1, 6, (-1.0 / 24, 1e-3, 64.0, 5), 0.5, 1e-10, "fp64"),
    ((4, 4, 4, 4), 0.05, 12, (-1.0 / 48, 2e-3, 64.0, 12), 0.5, 1e-8, "mixed"),
    ((6, 4, 4, 4), 0.05, 16, (-1.0 / 64, 2e-3, 64.0, 12), 0.5, 1e-8, "mixed"),
]


@pytest.mark.parametrize("dims,mass,n,rp,eps,tol,prec", CONFIGS)
def test_block_multishift_matches_oracle(dims, mass, n, rp, eps, tol, prec):
    need_gpu()
    ra = rational_approx(*rp)
    U = syn.random_links(dims, eps, 1200)
    B = syn.gaussian_pseudofermions(dims, n, 2200)
    ctx = make_ctx(dims, mass, U)
    Xg, info = ctx.block_multishift_cg(to_gpu(B), ra.beta, tol, precision=prec)
    Xg = Xg.cpu().numpy()
    assert info.true_rel_resid_max <= tol
    Xo, _, rc = oracle.sbcgrq(dims, mass, U, B, ra.beta, tol=1e-13, max_iter=20000)
    assert rc == 0
    _check_solution(dims, mass, U, B, ra.beta, Xg, tol, Xo)
    ctx.close()


def test_unsorted_shifts_and_per_shift_info():
    need_gpu()
    dims, mass, n = (4, 4, 4, 4), 0.1, 3
    U = syn.random_links(dims, 0.5, 1201)
    B = syn.gaussian_pseudofermions(dims, n, 2201)
    shifts = [0.5, 0.001, 4.0, 0.05]
    ctx = make_ctx(dims, mass, U)
    Xg, info = ctx.block_multishift_cg(to_gpu(B), shifts, 1e-10, precision="fp64")
    Xo, _, _ = oracle.sbcgrq(dims, mass, U, B, sorted(shifts), tol=1e-13)
    order = np.argsort(shifts)
    Xo_caller = np.empty_like(Xo)
    Xo_caller[order] = Xo
    _check_solution(dims, mass, U, B, shifts, Xg.cpu().numpy(), 1e-10, Xo_caller)
    assert len(info.per_shift_resid) == 4
    assert max(max(r) for r in info.per_shift_resid) <= 1e-10
    ctx.close()


def test_n1_equals_scalar_cg_iterates():
    """SBCGrQ with one right-hand side reduces to multishift CG (Sec. III)."""
    need_gpu()
    dims, mass = (8, 8, 8, 8), 0.05
    U = syn.random_links(dims, 0.5, 1202)
    B = syn.gaussian_pseudofermions(dims, 1, 2202)
    shifts = [0.002, 0.05, 1.0]
    ctx = make_ctx(dims, mass, U)
    Xg, info = ctx.block_multishift_cg(to_gpu(B), shifts, 1e-10, precision="fp64")
    xs, ks, _ = oracle.scg(dims, mass, U, B[..., 0], shifts, tol=0.5e-10)
    for s in range(3):
        assert colrel(Xg.cpu().numpy()[s], xs[s][..., None]) <= 1e-9
    assert abs(info.iters - ks) <= kcheck_slack()
    ctx.close()


def kcheck_slack():
    return 6  # host checks every 6 iterations


def test_pervector_scg_baseline_matches_oracle():
    need_gpu()
    dims, mass, n = (8, 8, 8, 8), 0.05, 4
    ra = rational_approx(-1.0 / 16, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1203)
    B = syn.gaussian_pseudofermions(dims, n, 2203)
    ctx = make_ctx(dims, mass, U)
    Xg, info = ctx.multishift_cg_pervector(to_gpu(B), ra.beta, 1e-10)
    Xo, _, _ = oracle.sbcgrq(dims, mass, U, B, ra.beta, tol=1e-13)
    _check_solution(dims, mass, U, B, ra.beta, Xg.cpu().numpy(), 1e-10 * 1.5, Xo)
    # block solver needs fewer iterations than the per-vector one summed over vectors
    _, binfo = ctx.block_multishift_cg(to_gpu(B), ra.beta, 1e-10, precision="fp64")
    assert binfo.iters < info.iters
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_force_matches_oracle(prec, tol):
    need_gpu()
    dims, mass, n = (8, 8, 8, 8), 0.05, 4
    ra = rational_approx(-1.0 / 16, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1204)
    Phi = syn.gaussian_pseudofermions(dims, n, 2204)
    ctx = make_ctx(dims, mass, U)
    G, S, info = ctx.force(to_gpu(Phi), ra.alpha0, ra.alpha, ra.beta, tol, precision=prec)
    G = G.cpu().numpy()
    Xo, _, _ = oracle.sbcgrq(dims, mass, U, Phi, ra.beta, tol=1e-13)
    Go = oracle.force(dims, U, Xo, ra.alpha)
    So = oracle.action(ra.alpha0, ra.alpha, Phi, Xo)
    # bound from the solution error of each shift
    bn = np.linalg.norm(Phi)
    bound = 2 * max(tol * bn / ((4 * mass ** 2 + b) * np.linalg.norm(Xo[s])) for s, b in enumerate(ra.beta)) + 1e-10
    assert np.linalg.norm(G - Go) / np.linalg.norm(Go) <= bound
    assert abs(S - So) / abs(So) <= bound
    ctx.close()


def test_force_kernel_parity_from_given_solutions():
    """G from supplied X (no solve): FP64 force kernel against the oracle's force of the same X."""
    need_gpu()
    dims = (6, 4, 4, 8)
    U = syn.random_links(dims, 0.5, 1205)
    ns, n = 3, 5
    X = np.stack([syn.gaussian_pseudofermions(dims, n, 2205 + s) for s in range(ns)])
    alpha = [0.3, 1.1, 0.07]
    ctx = make_ctx(dims, 0.1, U)
    G, _, _ = ctx.force(to_gpu(X[0]), 0.5, alpha, [0.1, 0.2, 0.3], 1e-8, X=to_gpu(X))
    Go = oracle.force(dims, U, X, alpha)
    assert np.linalg.norm(G.cpu().numpy() - Go) <= 1e-12 * np.linalg.norm(Go)
    ctx.close()


def test_force_given_solutions_resets_info():
    """With the solutions supplied (no solve) rhmc_force zeroes every info field except the
    caller's per_shift_resid pointer, which it leaves in place."""
    need_gpu()
    import ctypes

    from paper_1808_01829_gb300 import _lib
    from paper_1808_01829_gb300.api import PRECISION, _doubles, _ptr, _stream

    dims, ns, n = (4, 4, 4, 4), 2, 3
    U = syn.random_links(dims, 0.5, 1206)
    X = to_gpu(np.stack([syn.gaussian_pseudofermions(dims, n, 2206 + s) for s in range(ns)]))
    ctx = make_ctx(dims, 0.1, U)
    G = torch.empty((ctx.V, 4, 3, 3), dtype=torch.complex128, device=X.device)
    buf = (ctypes.c_double * (ns * n))(*([-1.0] * (ns * n)))
    info = _lib.Info()
    info.iters, info.phase1_ms, info.refine_ms = 7, 2.0, 3.5
    info.per_shift_resid = ctypes.cast(buf, ctypes.POINTER(ctypes.c_double))
    S = ctypes.c_double(0.0)
    rc = ctx.lib.rhmc_force(ctx._h, _ptr(X[0]), n, 0.5, _doubles([0.3, 1.1]), _doubles([0.1, 0.2]), ns, 1e-8, 0,
                            PRECISION["mixed"], _ptr(X), _ptr(G), ctypes.byref(S), None, ctypes.byref(info),
                            _stream(X))
    torch.cuda.synchronize()
    assert rc == 0
    assert ctypes.cast(info.per_shift_resid, ctypes.c_void_p).value == ctypes.addressof(buf)
    assert (info.iters, info.phase1_ms, info.refine_ms) == (0, 0.0, 0.0)
    assert list(buf) == [-1.0] * (ns * n)
    ctx.close()


def test_breakdown_on_rank_deficient_block():
    need_gpu()
    from paper_1808_01829_gb300._lib import RhmcError

    dims = (4, 4, 4, 4)
    U = syn.random_links(dims, 0.5, 1206)
    B = syn.gaussian_pseudofermions(dims, 2, 2206)
    B[..., 1] = B[..., 0]
    ctx = make_ctx(dims, 0.1, U)
    with pytest.raises(RhmcError, match="BREAKDOWN"):
        ctx.block_multishift_cg(to_gpu(B), [0.01, 0.1], 1e-10, precision="fp64")
    ctx.close()


def test_not_converged_reported():
    need_gpu()
    dims = (8, 8, 8, 8)
    U = syn.random_links(dims, 0.5, 1207)
    B = syn.gaussian_pseudofermions(dims, 2, 2207)
    ctx = make_ctx(dims, 0.01, U)
    X, info = ctx.block_multishift_cg(to_gpu(B), [1e-4, 0.1], 1e-10, max_iter=5, precision="fp64",
                                      allow_not_converged=True)
    assert info.iters <= 8 and info.true_rel_resid_max > 1e-10
    ctx.close()


def test_mixed_residuals_native_fp64_and_double_float_agree():
    """The mixed solver's residual operator: double-float (default) and native FP64 both
    reach the tolerance, with solutions within the solution-error bound of the oracle."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    dims, mass, n = (8, 8, 8, 8), 0.05, 4
    ra = rational_approx(-1.0 / 16, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1208)
    B = syn.gaussian_pseudofermions(dims, n, 2208)
    ctx = make_ctx(dims, mass, U)
    Xo, _, _ = oracle.sbcgrq(dims, mass, U, B, ra.beta, tol=1e-13)
    try:
        for native in (0, 1):
            lib.rhmc_tune_set(5, native)
            Xg, info = ctx.block_multishift_cg(to_gpu(B), ra.beta, 1e-9, precision="mixed")
            assert info.true_rel_resid_max <= 1e-9
            _check_solution(dims, mass, U, B, ra.beta, Xg.cpu().numpy(), 1e-9, Xo)
    finally:
        lib.rhmc_tune_set(5, 0)
    ctx.close()


@pytest.mark.parametrize("native", [0, 1])
def test_mixed_reported_residuals_match_oracle(native):
    """The per-shift true residuals the mixed solver reports (its FP64-accurate check of
    the returned solutions: double-float operator and fused subtraction, or native FP64)
    agree with the oracle's FP64 residuals of the same solutions."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    dims, mass, n = (8, 8, 8, 8), 0.05, 4
    ra = rational_approx(-1.0 / 16, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1212)
    B = syn.gaussian_pseudofermions(dims, n, 2212)
    ctx = make_ctx(dims, mass, U)
    try:
        lib.rhmc_tune_set(5, native)
        Xg, info = ctx.block_multishift_cg(to_gpu(B), ra.beta, 1e-9, precision="mixed")
    finally:
        lib.rhmc_tune_set(5, 0)
    Xg = Xg.cpu().numpy()
    bn = np.linalg.norm(B.reshape(-1, n), axis=0)
    for s, sig in enumerate(ra.beta):
        R = B - oracle.apply_A(dims, mass, U, Xg[s], sigma=sig)
        ro = np.linalg.norm(R.reshape(-1, n), axis=0) / bn
        rg = np.asarray(info.per_shift_resid[s])
        assert np.all(np.abs(rg - ro) <= 1e-2 * ro + 1e-13), (s, rg, ro)
    ctx.close()


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 4, 10)])
def test_tensor_core_shift_update_matches_oracle(dims):
    """Mixed solve at n_pf = 16 with the shifted updates on tcgen05 (three-piece TF32 split): same
    oracle criteria as the CUDA-core path; both paths reach the tolerance."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    mass, n = 0.05, 16
    ra = rational_approx(-1.0 / 64, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1209)
    B = syn.gaussian_pseudofermions(dims, n, 2209)
    ctx = make_ctx(dims, mass, U)
    Xo, _, _ = oracle.sbcgrq(dims, mass, U, B, ra.beta, tol=1e-13)
    try:
        lib.rhmc_tune_set(14, 1)  # shifted updates in HBM (no stored basis)
        for mode in (1, 2):
            lib.rhmc_tune_set(6, mode)
            Xg, info = ctx.block_multishift_cg(to_gpu(B), ra.beta, 1e-8, precision="mixed")
            assert info.true_rel_resid_max <= 1e-8
            _check_solution(dims, mass, U, B, ra.beta, Xg.cpu().numpy(), 1e-8, Xo)
    finally:
        lib.rhmc_tune_set(6, 0)
        lib.rhmc_tune_set(14, 0)
    ctx.close()


@pytest.mark.parametrize("variant", [0, 2, 5, 9, 10, 11])
def test_shifted_update_kernels_many_shifts(variant):
    """Both FP32 shifted-update kernels (column owners, built-in; lane slices) on a
    mixed solve with 40 shifts at n = 16 (the column-owner kernel splits them over
    launches) match the oracle."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    dims, mass, n = (4, 4, 4, 8), 0.05, 16
    shifts = list(np.geomspace(2e-3, 60.0, 40))
    U = syn.random_links(dims, 0.5, 1240)
    B = syn.gaussian_pseudofermions(dims, n, 2240)
    ctx = make_ctx(dims, mass, U)
    try:
        lib.rhmc_tune_set(6, variant)
        lib.rhmc_tune_set(14, 1)  # shifted updates in HBM (no stored basis)
        Xg, info = ctx.block_multishift_cg(to_gpu(B), shifts, 1e-9, precision="mixed")
    finally:
        lib.rhmc_tune_set(6, 0)
        lib.rhmc_tune_set(14, 0)
    assert info.true_rel_resid_max <= 1e-9
    Xo, _, rc = oracle.sbcgrq(dims, mass, U, B, shifts, tol=1e-13, max_iter=20000)
    assert rc == 0
    _check_solution(dims, mass, U, B, shifts, Xg.cpu().numpy(), 1e-9, Xo)
    ctx.close()


@pytest.mark.parametrize("scalar", [0, 1])
@pytest.mark.parametrize("n", [16, 5])
def test_fp32_bulk_fma_forms(scalar, n):
    """The FP32 Gram and Y = C + A M kernels with packed FP32x2 FMAs (built-in)
    and with scalar FMAs (RHMC_TUNE_AXPY_SCALAR = 1) both give mixed solves
    that match the oracle, at n = 16 (packed Gram) and odd n."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    dims, mass = (4, 4, 4, 8), 0.05
    shifts = [1e-3, 0.02, 0.3, 4.0]
    U = syn.random_links(dims, 0.5, 1250 + n)
    B = syn.gaussian_pseudofermions(dims, n, 2250 + n)
    ctx = make_ctx(dims, mass, U)
    try:
        lib.rhmc_tune_set(12, scalar)
        Xg, info = ctx.block_multishift_cg(to_gpu(B), shifts, 1e-9, precision="mixed")
    finally:
        lib.rhmc_tune_set(12, 0)
    assert info.true_rel_resid_max <= 1e-9
    Xo, _, rc = oracle.sbcgrq(dims, mass, U, B, shifts, tol=1e-13, max_iter=20000)
    assert rc == 0
    _check_solution(dims, mass, U, B, shifts, Xg.cpu().numpy(), 1e-9, Xo)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_no_defect_correction_reports_true_residuals(precision):
    """RHMC_TUNE_NO_DEFECT_CORRECTION = 1 with an iteration cap: NOT_CONVERGED, no
    corrections, and the reported per-(shift, column) residuals are the true
    relative residuals of the returned solutions (oracle operator)."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    dims, mass, n = (4, 4, 4, 8), 0.02, 4
    shifts = [2e-3, 0.05, 1.0]
    U = syn.random_links(dims, 0.5, 1260)
    B = syn.gaussian_pseudofermions(dims, n, 2260)
    ctx = make_ctx(dims, mass, U)
    ctx.tune_set(_lib.RHMC_TUNE_NO_DEFECT_CORRECTION, 1)
    Xg, info = ctx.block_multishift_cg(to_gpu(B), shifts, 1e-12, max_iter=18, precision=precision,
                                       allow_not_converged=True)
    ctx.tune_set(_lib.RHMC_TUNE_NO_DEFECT_CORRECTION, 0)
    assert info.refinements == 0 and info.iters == 18
    X = Xg.cpu().numpy()
    bn = np.linalg.norm(B.reshape(-1, n), axis=0)
    got = np.asarray(info.per_shift_resid).reshape(len(shifts), n)
    for s, sig in enumerate(shifts):
        R = B - oracle.apply_A(dims, mass, U, X[s], sigma=sig)
        want = np.linalg.norm(R.reshape(-1, n), axis=0) / bn
        assert np.allclose(got[s], want, rtol=1e-6, atol=0), (s, got[s], want)
    assert got.max() > 1e-12  # 18 iterations do not reach the tolerance
    ctx.close()


@pytest.mark.parametrize("cap,gemm,chunk", [(256, 0, 0), (256, 1, 0), (256, 0, 5), (14, 0, 0), (1, 0, 0)])
def test_stored_basis_assembly_matches_oracle(cap, gemm, chunk):
    """Mixed solve with the shifted solutions assembled from the stored block basis
    (RHMC_TUNE_BASIS_ITERS): both assembly GEMMs, FP64 sums of 5-block partial
    products, a capacity of 14 iterations (the solve switches to the shifted
    updates part way) and the mode off (1); every shift matches the oracle."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    dims, mass, n = (4, 4, 4, 8), 0.03, 16
    ra = rational_approx(-1.0 / 64, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1270)
    B = syn.gaussian_pseudofermions(dims, n, 2270)
    ctx = make_ctx(dims, mass, U)
    ctx.tune_set(_lib.RHMC_TUNE_BASIS_ITERS, cap)
    ctx.tune_set(_lib.RHMC_TUNE_BASIS_GEMM, gemm)
    ctx.tune_set(_lib.RHMC_TUNE_BASIS_CHUNK, chunk)
    try:
        Xg, info = ctx.block_multishift_cg(to_gpu(B), ra.beta, 1e-9, precision="mixed")
    finally:
        for key in (_lib.RHMC_TUNE_BASIS_ITERS, _lib.RHMC_TUNE_BASIS_GEMM, _lib.RHMC_TUNE_BASIS_CHUNK):
            ctx.tune_set(key, 0)
    assert info.true_rel_resid_max <= 1e-9
    # every shift kept being updated to the end of the multishift phase (after a switch
    # from the stored basis too): what is left for the corrections is FP32 drift
    assert info.phase1_rel_resid_max <= 1e-4
    if cap == 14:
        assert info.iters > 14
    Xo, _, rc = oracle.sbcgrq(dims, mass, U, B, ra.beta, tol=1e-13, max_iter=20000)
    assert rc == 0
    _check_solution(dims, mass, U, B, ra.beta, Xg.cpu().numpy(), 1e-9, Xo)
    ctx.close()


def test_force_double_float_matches_native_fp64():
    """The double-float force path (built-in) and the native FP64 one
    (RHMC_TUNE_NATIVE_FP64_RESIDUALS) agree to 1e-12 from the same solutions,
    and both match the oracle's force of those solutions."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    dims, mass, n = (6, 4, 4, 8), 0.05, 5
    ra = rational_approx(-1.0 / 20, 1e-3, 64.0, 6)
    U = syn.random_links(dims, 0.5, 1250)
    Phi = syn.gaussian_pseudofermions(dims, n, 2250)
    ctx = make_ctx(dims, mass, U)
    P = to_gpu(Phi)
    X, _ = ctx.block_multishift_cg(P, ra.beta, 1e-10, precision="fp64")
    G_df, S_df, _ = ctx.force(P, ra.alpha0, ra.alpha, ra.beta, 1e-10, X=X)
    try:
        lib.rhmc_tune_set(5, 1)
        G_64, S_64, _ = ctx.force(P, ra.alpha0, ra.alpha, ra.beta, 1e-10, X=X)
    finally:
        lib.rhmc_tune_set(5, 0)
    g_df, g_64 = G_df.cpu().numpy(), G_64.cpu().numpy()
    assert np.linalg.norm(g_df - g_64) <= 1e-12 * np.linalg.norm(g_64)
    assert S_df == S_64
    Go = oracle.force(dims, U, X.cpu().numpy(), ra.alpha).reshape(g_64.shape)
    assert np.linalg.norm(g_df - Go) <= 1e-12 * np.linalg.norm(Go)
    ctx.close()


@pytest.mark.parametrize("n", [1, 5, 16])
def test_nxn_double_float_and_fp64_agree(n):
    """The mixed solve's base n x n steps (alpha_k; rho_k, delta_k): double-float on the
    FP32 units (built-in) and native FP64 both reach the tolerance with solutions within
    the oracle's solution-error bound, in the same number of iterations (the recursions
    differ by about 1e-13 relative)."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    dims, mass = (8, 4, 4, 6), 0.05
    ra = rational_approx(-1.0 / 16, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1210)
    B = syn.gaussian_pseudofermions(dims, n, 2210)
    ctx = make_ctx(dims, mass, U)
    Xo, _, _ = oracle.sbcgrq(dims, mass, U, B, ra.beta, tol=1e-13)
    iters = []
    try:
        for fp64 in (0, 1):
            ctx.tune_set(_lib.RHMC_TUNE_NXN_FP64, fp64)
            Xg, info = ctx.block_multishift_cg(to_gpu(B), ra.beta, 1e-9, precision="mixed")
            assert info.true_rel_resid_max <= 1e-9
            _check_solution(dims, mass, U, B, ra.beta, Xg.cpu().numpy(), 1e-9, Xo)
            iters.append(info.iters)
    finally:
        ctx.tune_set(_lib.RHMC_TUNE_NXN_FP64, 0)
    assert abs(iters[0] - iters[1]) <= 1, iters
    ctx.close()
