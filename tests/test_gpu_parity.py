"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Every comparison is element by element on the same seeded inputs.  FP64 mode
must agree to rounding (relative 1e-11 for single products, 1e-9 after a
degree-7 filter whose scaled polynomial amplifies rounding by its condition);
the FP32-storage mode to 1e-5 relative (FP32 unit round-off 6e-8 times the
filter's growth).  Eigenvalues in FP64 mode: 1e-6 Ha (spec tolerance).
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import cuda_available, gpu_system, rel_err, to_dev, torch

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def tiny_pair():
    from oracle.operators import Discretisation
    s = W.tiny(seed=11)
    return Discretisation(s), gpu_system(s)


@pytest.fixture(scope="module")
def ho_pair():
    from oracle.operators import Discretisation
    s = W.harmonic(cells=3, half=6.0)
    return Discretisation(s), gpu_system(s)


@pytest.mark.parametrize("N", [1, 7, 33, 70])
def test_apply_H_M_Minv(tiny_pair, N):
    d, G = tiny_pair
    X = W.random_block(d.system, N, seed=100 + N)
    Xd = to_dev(X)
    assert rel_err(G.apply_H(Xd), d.apply_H_assembled(X)) < 1e-11
    assert rel_err(G.apply_M(Xd), d.apply_M_assembled(X)) < 1e-12
    assert rel_err(G.apply_Minv(Xd), d.apply_Minv_block(X)) < 1e-10


def test_padded_leading_dimension(tiny_pair):
    d, G = tiny_pair
    X = W.random_block(d.system, 9, seed=7)
    big = torch.zeros((X.shape[0], 16), dtype=torch.float64, device="cuda")
    big[:, :9] = to_dev(X)
    out = torch.full_like(big, 7.0)
    G.apply_H(big[:, :9], out[:, :9])
    assert rel_err(out[:, :9], d.apply_H_assembled(X)) < 1e-11
    assert torch.all(out[:, 9:] == 7.0)       # columns beyond N untouched


def test_classical_only_system(ho_pair):
    d, G = ho_pair
    X = W.random_block(d.system, 5, seed=3)
    Xd = to_dev(X)
    assert rel_err(G.apply_H(Xd), d.apply_H_assembled(X)) < 1e-11
    assert rel_err(G.apply_Minv(Xd), d.apply_Minv_block(X)) < 1e-12


def _bounds(d, N):
    from oracle.chfsi import dense_eigs
    H, M, act = d.dense_active()
    import scipy.linalg as sla
    ev = sla.eigh(H, M, eigvals_only=True)
    return ev[N - 1], ev.max() * 1.05, ev[0]


@pytest.mark.parametrize("N,m", [(10, 7), (33, 4)])
def test_chfsi_step_fp64(tiny_pair, N, m):
    from oracle.chfsi import chebyshev_filter_scaled
    d, G = tiny_pair
    X = W.initial_block(d.system, N, seed=1)
    a, b, a0 = _bounds(d, N)
    ref = chebyshev_filter_scaled(d.apply_Htilde, X, m, a, b, a0)
    Xd = to_dev(X)
    G.chfsi_step(Xd, m, a, b, a0, precision="fp64")
    assert rel_err(Xd, ref) < 1e-9
    # bitwise reproducible
    Xd2 = to_dev(X)
    G.chfsi_step(Xd2, m, a, b, a0, precision="fp64")
    assert torch.equal(Xd, Xd2)


@pytest.mark.parametrize("tail", [0, 2])
def test_chfsi_step_fp32(tiny_pair, tail):
    from oracle.chfsi import chebyshev_filter_scaled
    d, G = tiny_pair
    N, m = 12, 7
    X = W.initial_block(d.system, N, seed=2)
    a, b, a0 = _bounds(d, N)
    ref = chebyshev_filter_scaled(d.apply_Htilde, X, m, a, b, a0)
    Xd = to_dev(X)
    G.chfsi_step(Xd, m, a, b, a0, precision="fp32", fp64_tail=tail)
    err = rel_err(Xd, ref)
    assert err < 2e-5, err


def test_rayleigh_ritz_fp64(tiny_pair):
    from oracle.chfsi import cholqr, rayleigh_ritz
    d, G = tiny_pair
    N = 10
    X = W.initial_block(d.system, N, seed=4)
    Q, _ = cholqr(X)
    eps_ref, Xr, res_ref = rayleigh_ritz(d.apply_H_assembled, d.apply_M_assembled, Q)
    Xd = to_dev(X)
    eps, res = G.rayleigh_ritz(Xd)
    np.testing.assert_allclose(eps, eps_ref, atol=1e-9, rtol=1e-10)
    np.testing.assert_allclose(res, res_ref, atol=1e-8, rtol=1e-6)
    # Ritz vectors are M-orthonormal: X^T M X = I
    MX = G.apply_M(Xd)
    gram = (Xd.T @ MX).cpu().numpy()
    np.testing.assert_allclose(gram, np.eye(N), atol=1e-10)


def test_upper_bound_matches_oracle(tiny_pair):
    from oracle.chfsi import lanczos_upper_bound
    d, G = tiny_pair
    v0 = W.lanczos_start(d.system)
    ref = lanczos_upper_bound(d.apply_Htilde, d.apply_M_assembled, v0, 10)
    b = G.upper_bound(to_dev(v0), 10)
    assert abs(b - ref) < 1e-8 * abs(ref)
    H, M, act = d.dense_active()
    import scipy.linalg as sla
    assert b >= sla.eigh(H, M, eigvals_only=True).max() * (1 - 1e-12)


def test_chfsi_converges_to_dense_tiny(tiny_pair):
    from oracle.chfsi import dense_eigs
    d, G = tiny_pair
    N, m, nconv = 10, 12, 7
    X = to_dev(W.initial_block(d.system, N, seed=1))
    eps, res, it, b = G.solve(X, m, tol=1e-9, v0=to_dev(W.lanczos_start(d.system)), n_conv=nconv)
    ref = dense_eigs(d, N)
    assert res[:nconv].max() < 1e-9
    np.testing.assert_allclose(eps[:nconv], ref[:nconv], atol=1e-9)


def test_error_paths(tiny_pair):
    from paper_1610_02121_gb300 import EfeError
    d, G = tiny_pair
    X = to_dev(W.initial_block(d.system, 4, seed=1))
    with pytest.raises(EfeError) as e:
        G.chfsi_step(X, 3, 1.0, 0.5, 0.0)            # a > b
    assert e.value.code == 1
    Xr = to_dev(W.initial_block(d.system, 4, seed=1))
    Xr[:, 3] = float("nan")                           # non-finite block
    with pytest.raises(EfeError) as e:
        G.rayleigh_ritz(Xr)
    assert e.value.code == 3
    V = torch.full((G.n_qpoints,), float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(EfeError) as e:
        G.set_potential(V)
    assert e.value.code == 6
    G.set_potential_analytic()                         # restore


def test_rank_deficient_block_shifted_cholqr(tiny_pair):
    """Duplicated and nearly collinear columns: Rayleigh-Ritz takes shifted
    Cholesky-QR passes and still returns M-orthonormal Ritz vectors whose Ritz
    values interlace the exact spectrum (eps_k >= lambda_k, Cauchy)."""
    from oracle.chfsi import dense_eigs
    d, G = tiny_pair
    N = 6
    ref = dense_eigs(d, N)
    for kind in ("duplicate", "collinear"):
        # generic columns (unit-vector columns make every product exact and
        # leave no rounding noise for the shifted passes to lift)
        X = to_dev(W.random_block(d.system, N, seed=2))
        if kind == "duplicate":
            X[:, 4] = X[:, 1]
        else:
            X[:, 5] = X[:, 0] + 1e-11 * X[:, 3]
        n0 = G.rr_shifted_passes()
        eps, res = G.rayleigh_ritz(X)
        assert G.rr_shifted_passes() > n0
        assert np.all(np.isfinite(eps)) and np.all(np.isfinite(res))
        assert np.all(np.diff(eps) >= 0)
        assert np.all(eps >= ref[:N] - 1e-10)
        MX = G.apply_M(X)
        gram = (X.T @ MX).cpu().numpy()
        assert np.abs(gram - np.eye(N)).max() < 1e-10


def test_hydrogen_config1_converged():
    """6x6x6 cells, degree 4, 20-bohr box, hydrogenic enrichment, N = 8, m = 20, FP64,
    residual < 1e-8: eigenvalues against the oracle's assembled problem (sparse
    shift-invert, the plain definition) and the closed form -1/2 for 1s."""
    import scipy.sparse.linalg as ssl
    from oracle.operators import Discretisation
    s = W.hydrogen()
    G = gpu_system(s)
    N, m, nconv = 8, 20, 5
    X = to_dev(W.initial_block(s, N, seed=1))
    eps, res, it, b = G.solve(X, m, tol=1e-8, v0=to_dev(W.lanczos_start(s)), n_conv=nconv)
    assert res[:nconv].max() < 1e-8
    d = Discretisation(s)
    act = np.nonzero(d.active)[0]
    H = d.H[act][:, act].tocsc()
    M = d.M[act][:, act].tocsc()
    ref = np.sort(ssl.eigsh(H, k=nconv, M=M, sigma=-0.6, which="LM")[0])
    np.testing.assert_allclose(eps[:nconv], ref, atol=1e-6)
    assert abs(eps[0] + 0.5) < 1e-3
    assert np.ptp(eps[1:4]) < 1e-7          # 2p triplet (cubic symmetry about the nucleus)


@pytest.mark.parametrize("N", [17, 135, 300])
@pytest.mark.parametrize("prec,tols", [("tf32", [(1, 3e-3), (7, 2e-2)]), ("tf32x3", [(1, 1e-5), (7, 5e-5)]),
                                       ("bf16", [(1, 3e-2)])])
def test_chfsi_step_tf32_tensor_cores(tiny_pair, N, prec, tols):
    """tcgen05 cell products (FP32 accumulation, FP32 vector storage).  One TF32
    pass: one degree agrees with the FP64 oracle to TF32 accuracy (unit round-off
    2^-11, bound 3e-3 relative), a degree-7 filter to 2e-2.  The 3-term split
    (tf32x3) is FP32-grade: FP32 round-off 6e-8 times the cancellation factor
    ||H|| ||Y|| / ||H Y|| (about 30 here) gives ~2e-6 per degree; bounds 1e-5
    (one degree) and 5e-5 (seven degrees).  BF16 operands (kind::f16, unit
    round-off 2^-8, eight times TF32's): one degree to 3e-2.  N = 300 spans two
    160-column tensor-core tiles with a ragged tail; N = 17 one partial tile."""
    from oracle.chfsi import chebyshev_filter_scaled
    d, G = tiny_pair
    X = W.random_block(d.system, N, seed=30 + N)
    a, b, a0 = _bounds(d, 10)
    for m, tol in tols:
        ref = chebyshev_filter_scaled(d.apply_Htilde, X, m, a, b, a0)
        Xd = to_dev(X)
        G.chfsi_step(Xd, m, a, b, a0, precision=prec, fp64_tail=0)
        err = rel_err(Xd, ref)
        assert err < tol, (m, err)


@pytest.mark.parametrize("prec,tol,atol", [("tf32", 1e-7, 1e-5), ("tf32x3", 1e-9, 1e-8), ("bf16", 1e-6, 1e-4)])
def test_chfsi_converges_mixed_tiny(tiny_pair, prec, tol, atol):
    """Mixed precision (tensor-core filter, FP64 tail degrees, FP64 CholQR and
    Rayleigh-Ritz) reaches the dense eigenvalues: within 1e-5 Ha with one TF32
    pass, within 1e-8 Ha with the FP32-grade 3-term split, within 1e-4 Ha with
    BF16 operands."""
    from oracle.chfsi import dense_eigs
    d, G = tiny_pair
    N, m, nconv = 10, 12, 7
    X = to_dev(W.initial_block(d.system, N, seed=1))
    eps, res, it, b = G.solve(X, m, tol=tol, precision=prec, fp64_tail=2,
                              v0=to_dev(W.lanczos_start(d.system)), n_conv=nconv, max_iter=300)
    ref = dense_eigs(d, N)
    np.testing.assert_allclose(eps[:nconv], ref[:nconv], atol=atol)


def test_fp64_tensor_engine_products(tiny_pair):
    """FP64-grade products on the BF16 tensor cores (error-free 7-digit slicing)
    and the FP64-grade enrichment coupling on the FP32 pipe (double-float sums)
    that comes with them: the H, M and M^-1 applies (N > 8 use both) and the
    filter agree with the FP64 oracle to FP64-level tolerances, and
    Rayleigh-Ritz (tall products through the engine) reproduces the oracle's
    Ritz values."""
    from oracle.chfsi import chebyshev_filter_scaled, cholqr, rayleigh_ritz
    d, G = tiny_pair
    G.set_fp64_engine("tensor")
    try:
        for N in (9, 33, 135, 200):
            X = W.random_block(d.system, N, seed=60 + N)
            assert rel_err(G.apply_H(to_dev(X)), d.apply_H_assembled(X)) < 1e-10
            assert rel_err(G.apply_M(to_dev(X)), d.apply_M_assembled(X)) < 1e-12
            assert rel_err(G.apply_Minv(to_dev(X)), d.apply_Minv_block(X)) < 1e-10
        N, m = 33, 7
        X = W.initial_block(d.system, N, seed=3)
        a, b, a0 = _bounds(d, N)
        ref = chebyshev_filter_scaled(d.apply_Htilde, X, m, a, b, a0)
        Xd = to_dev(X)
        G.chfsi_step(Xd, m, a, b, a0, precision="fp64")
        assert rel_err(Xd, ref) < 1e-8
        X = W.initial_block(d.system, 20, seed=4)
        Q, _ = cholqr(X)
        eps_ref, _, res_ref = rayleigh_ritz(d.apply_H_assembled, d.apply_M_assembled, Q)
        eps, res = G.rayleigh_ritz(to_dev(X))
        np.testing.assert_allclose(eps, eps_ref, atol=1e-9, rtol=1e-10)
    finally:
        G.set_fp64_engine("dfma")


def test_fp64_tensor_engine_converges(tiny_pair):
    from oracle.chfsi import dense_eigs
    d, G = tiny_pair
    G.set_fp64_engine("tensor")
    try:
        N, m, nconv = 12, 12, 7
        X = to_dev(W.initial_block(d.system, N, seed=1))
        eps, res, it, b = G.solve(X, m, tol=1e-9, precision="tf32x3", fp64_tail=2,
                                  v0=to_dev(W.lanczos_start(d.system)), n_conv=nconv, max_iter=300)
        ref = dense_eigs(d, N)
        np.testing.assert_allclose(eps[:nconv], ref[:nconv], atol=1e-8)
    finally:
        G.set_fp64_engine("dfma")


@pytest.mark.parametrize("which,N", [("tiny", 150), ("hydrogen", 8), ("hydrogen", 40)])
def test_fp64_tensor_engine_gram(tiny_pair, which, N):
    """Cholesky-QR and Rayleigh-Ritz with the tensor-core A^T B (K split into
    segments of 256-row exact groups, FP64 partial tiles, symmetric tiles only
    above the diagonal) give the DFMA path's Ritz values."""
    if which == "tiny":
        G = tiny_pair[1]
        s = tiny_pair[0].system
    else:
        s = W.hydrogen(cells=6, half=10.0, tau=1e-8, max_depth=6)
        G = gpu_system(s)
    X = to_dev(W.random_block(s, N, seed=91))
    G.set_fp64_engine("dfma")
    e_ref, r_ref = G.rayleigh_ritz(X.clone())
    G.set_fp64_engine("tensor")
    try:
        e, r = G.rayleigh_ritz(X.clone())
    finally:
        G.set_fp64_engine("dfma")
    np.testing.assert_allclose(e, e_ref, rtol=1e-10, atol=1e-10 * np.abs(e_ref).max())


# --- persistent tensor-core kernels with several work items per CTA --------------
# The tcgen05 kernels are persistent (one CTA per SM walks the work items).  On
# the small meshes above every CTA gets one item; with the grid capped, each CTA
# walks many items, so the double TMEM accumulator alternation, the mbarrier
# phase flips across items and the stage ring wrap-around all run under the
# oracle comparison.

@pytest.fixture(scope="module")
def mid_pair():
    from oracle.operators import Discretisation
    s = W.tiny(seed=11, cells=(4, 4, 4), max_depth=3)   # 64 cells, 8 per parity colour
    return Discretisation(s), gpu_system(s)


def _mid_bounds(d, X):
    from oracle.chfsi import cholqr, lanczos_upper_bound, rayleigh_ritz
    Q, _ = cholqr(X)
    eps, _, _ = rayleigh_ritz(d.apply_H_assembled, d.apply_M_assembled, Q)
    b = lanczos_upper_bound(d.apply_Htilde, d.apply_M_assembled, W.lanczos_start(d.system), 10)
    return eps.max(), 1.05 * b, eps.min()


@pytest.mark.parametrize("prec,tols", [("tf32", [(1, 6e-3), (7, 4e-2)]), ("tf32x3", [(1, 1e-5), (7, 5e-5)]),
                                       ("bf16", [(1, 6e-2)])])
def test_tensor_core_cells_many_items_per_cta(mid_pair, prec, tols):
    """k_cell_tc3 capped at 2 CTAs: N = 300 is two 160-column tiles, so each CTA
    walks 8 (cell, tile) items per colour launch; the capped and uncapped
    launches agree bit for bit (the items are independent and the scatter order
    per colour is fixed).  Against the oracle: the 3-term split keeps the
    one-item bounds; one TF32 pass errs by about 2 u_tf32 = 2^-10 times the
    cancellation factor max(|H||Y|) / max|H Y| of the cell products, which is larger on this
    mesh (its cells are twice the size of the 2x3x2 case's): 3.3e-3 measured
    for one degree, bounds 6e-3 and 4e-2."""
    from oracle.chfsi import chebyshev_filter_scaled
    d, G = mid_pair
    N = 300
    X = W.random_block(d.system, N, seed=77)
    a, b, a0 = _mid_bounds(d, W.initial_block(d.system, 20, seed=1))
    for m, tol in tols:
        ref = chebyshev_filter_scaled(d.apply_Htilde, X, m, a, b, a0)
        G.set_grid_cap(2)
        try:
            Xd = to_dev(X)
            G.chfsi_step(Xd, m, a, b, a0, precision=prec, fp64_tail=0)
        finally:
            G.set_grid_cap(0)
        err = rel_err(Xd, ref)
        assert err < tol, (m, err)
        Xu = to_dev(X)
        G.chfsi_step(Xu, m, a, b, a0, precision=prec, fp64_tail=0)
        assert torch.equal(Xd, Xu)


def test_fp64_engine_many_items_per_cta(mid_pair):
    """k_oz on one CTA: CELL mode (N = 135: 8 cells x 2 column tiles per colour),
    ROWS (the Rayleigh-Ritz rotations: 39 row tiles x 2 column tiles) and GRAM
    (the Gram and projection products: 3 tile pairs, 20 groups of 256 rows each)
    all walk many items on that one CTA.  H apply and a degree-7 FP64 filter
    against the oracle, Ritz values against the oracle's Cholesky-QR + RR."""
    from oracle.chfsi import chebyshev_filter_scaled, cholqr, rayleigh_ritz
    d, G = mid_pair
    N = 135
    X = W.random_block(d.system, N, seed=78)
    a, b, a0 = _mid_bounds(d, W.initial_block(d.system, 20, seed=1))
    ref_f = chebyshev_filter_scaled(d.apply_Htilde, X, 7, a, b, a0)
    Q, _ = cholqr(X)
    eps_ref, _, _ = rayleigh_ritz(d.apply_H_assembled, d.apply_M_assembled, Q)
    G.set_fp64_engine("tensor")
    G.set_grid_cap(1)
    try:
        assert rel_err(G.apply_H(to_dev(X)), d.apply_H_assembled(X)) < 1e-10
        Xd = to_dev(X)
        G.chfsi_step(Xd, 7, a, b, a0, precision="fp64")
        assert rel_err(Xd, ref_f) < 1e-8
        eps, _ = G.rayleigh_ritz(to_dev(X))
    finally:
        G.set_grid_cap(0)
        G.set_fp64_engine("dfma")
    np.testing.assert_allclose(eps, eps_ref, atol=1e-9, rtol=1e-10)


def test_in_place_products_rejected(tiny_pair):
    import ctypes as C
    d, G = tiny_pair
    X = to_dev(W.random_block(d.system, 4, seed=5))
    keep = X.clone()
    for fn in (G.L.efe_apply_H, G.L.efe_apply_M):
        rc = fn(G.h, C.c_void_p(X.data_ptr()), X.stride(0), 4, C.c_void_p(X.data_ptr()), X.stride(0), G._stream())
        assert rc == 1
    # overlapping by one column
    big = to_dev(np.zeros((X.shape[0], 9)))
    rc = G.L.efe_apply_M(G.h, C.c_void_p(big.data_ptr()), 9, 5, C.c_void_p(big[:, 4:].data_ptr()), 9, G._stream())
    assert rc == 1
    torch.cuda.synchronize()
    assert torch.equal(X, keep)
    # (M^E)^-1 works on a copy: in place is allowed
    Y = G.apply_Minv(X, X.clone())
    Z = X.clone()
    G.apply_Minv(Z, Z)
    assert torch.equal(Y, Z)


# --- the large-N code paths (280-atom cluster, N ~ 2200), driven on small inputs --------
# Rayleigh-Ritz in column panels, the FP64 engine's tall products with K > 256
# (several exact accumulation groups) and with operand images in row panels,
# the blocked multi-CTA Cholesky / triangular inverse / block Jacobi
# eigensolver, and the FP32 recurrence slots living inside the FP64 workspace
# (N a multiple of 8) -- each forced through EFE_OPT_* on the tiny mesh and
# compared with the oracle.

def _rr_ref(d, X):
    from oracle.chfsi import cholqr, rayleigh_ritz
    Q, _ = cholqr(X)
    return rayleigh_ritz(d.apply_H_assembled, d.apply_M_assembled, Q)


@pytest.mark.parametrize("engine", ["dfma", "tensor"])
@pytest.mark.parametrize("N", [40, 150])
def test_rayleigh_ritz_panels_and_blocked_dense(tiny_pair, engine, N):
    """Forced: two column panels, blocked dense kernels, and (tensor engine)
    image panels of 256 rows, so the Gram products accumulate over K panels and
    the rotations run in row panels; N = 150 takes one K group (256) in the
    tall products.  Ritz values, residuals and M-orthonormality against the
    oracle's Cholesky-QR + Rayleigh-Ritz."""
    d, G = tiny_pair
    X = W.initial_block(d.system, N, seed=4)
    eps_ref, _, res_ref = _rr_ref(d, X)
    G.set_fp64_engine(engine)
    G.set_option("rr_panels", 1)
    G.set_option("dense_blocked", 1)
    G.set_option("image_rows", 256)
    try:
        Xd = to_dev(X)
        eps, res = G.rayleigh_ritz(Xd)
        MX = G.apply_M(Xd)
    finally:
        G.set_option("image_rows", 0)
        G.set_option("dense_blocked", 0)
        G.set_option("rr_panels", 0)
        G.set_fp64_engine("dfma")
    np.testing.assert_allclose(eps, eps_ref, atol=1e-9, rtol=1e-10)
    np.testing.assert_allclose(res, res_ref, atol=1e-8, rtol=1e-6)
    gram = (Xd.T @ MX).cpu().numpy()
    np.testing.assert_allclose(gram, np.eye(N), atol=1e-10)


def test_tall_products_long_K_match_dfma(tiny_pair):
    """The FP64 engine's tall products with K = N = 400 (two exact groups of
    256 and 144; the triangular X R^-1 in column panels of 384 and 16) and
    256-row image panels give the DFMA path's Ritz values to FP64 rounding, and
    both match the oracle."""
    d, G = tiny_pair
    N = 400
    X = to_dev(W.random_block(d.system, N, seed=93))
    G.set_fp64_engine("dfma")
    Xa = X.clone()
    e_ref, _ = G.rayleigh_ritz(Xa)
    G.set_fp64_engine("tensor")
    G.set_option("image_rows", 256)
    try:
        Xb = X.clone()
        e, _ = G.rayleigh_ritz(Xb)
    finally:
        G.set_option("image_rows", 0)
        G.set_fp64_engine("dfma")
    np.testing.assert_allclose(e, e_ref, rtol=1e-10, atol=1e-10 * np.abs(e_ref).max())
    eps_ref, _, _ = _rr_ref(d, W.random_block(d.system, N, seed=93))
    np.testing.assert_allclose(e, eps_ref, rtol=1e-9, atol=1e-9 * np.abs(eps_ref).max())


@pytest.mark.parametrize("prec,N,tail,tol", [("tf32x3", 64, 2, 5e-5), ("fp32", 16, 0, 2e-5), ("tf32x3", 304, 0, 5e-5)])
def test_mixed_filter_slots_inside_fp64_workspace(tiny_pair, prec, N, tol, tail):
    """N a multiple of 8: the FP32 recurrence slots and the cell-product output
    live inside the FP64 workspace (no padding columns); a degree-7 filter
    against the oracle at the mixed-mode tolerances, then a Rayleigh-Ritz call
    (which overwrites that workspace) and the same filter again, bitwise equal."""
    from oracle.chfsi import chebyshev_filter_scaled
    d, G = tiny_pair
    X = W.random_block(d.system, N, seed=70 + N)
    a, b, a0 = _bounds(d, 10)
    ref = chebyshev_filter_scaled(d.apply_Htilde, X, 7, a, b, a0)
    Xd = to_dev(X)
    G.chfsi_step(Xd, 7, a, b, a0, precision=prec, fp64_tail=tail)
    assert rel_err(Xd, ref) < tol
    G.rayleigh_ritz(to_dev(W.random_block(d.system, N, seed=1)))
    Xe = to_dev(X)
    G.chfsi_step(Xe, 7, a, b, a0, precision=prec, fp64_tail=tail)
    assert torch.equal(Xd, Xe)


@pytest.mark.parametrize("cols", [0, 1])
@pytest.mark.parametrize("prec,N,tol", [("tf32x3", 24, 5e-5), ("tf32x3", 300, 5e-5), ("fp32", 12, 2e-5)])
def test_mixed_filter_grouped_coupling(tiny_pair, prec, N, tol, cols):
    """The many-function enrichment coupling of the mixed degrees (columns
    products over 32-node blocks -- dense tiles (cols 0) or each node's own
    entries (cols 1); rows products over the functions that share a support,
    FP32 over 64-node chunks, FP64 across chunks and items), forced on the tiny
    mesh: a degree-7 filter against the oracle at the mixed-mode tolerances of
    the dense-tile path."""
    from oracle.chfsi import chebyshev_filter_scaled
    d, G = tiny_pair
    X = W.random_block(d.system, N, seed=80 + N)
    a, b, a0 = _bounds(d, 10)
    ref = chebyshev_filter_scaled(d.apply_Htilde, X, 7, a, b, a0)
    G.set_option("coupling_sparse", 1)
    G.set_option("coupling_cols", cols)
    try:
        Xd = to_dev(X)
        G.chfsi_step(Xd, 7, a, b, a0, precision=prec, fp64_tail=0)
    finally:
        G.set_option("coupling_cols", 0)
        G.set_option("coupling_sparse", 0)
    assert rel_err(Xd, ref) < tol


@pytest.mark.parametrize("engine,prec", [("dfma", "tf32x3"), ("tensor", "fp64")])
def test_bounded_wait_runs_out_then_recovers(tiny_pair, engine, prec):
    """Failure path of the tensor-core kernels without a GPU fault: with the test
    stall on, the MMA warp first waits on an mbarrier that nothing completes; the
    bounded wait (about a second) runs out, the CTA drains its bulk copies and
    MMAs, frees its TMEM, and the call returns EFE_ERR_TIMEOUT.  The next normal
    call on the same handle succeeds and matches the oracle."""
    from oracle.chfsi import chebyshev_filter_scaled
    from paper_1610_02121_gb300 import EfeError
    d, G = tiny_pair
    N, m = 12, 3
    X = W.initial_block(d.system, N, seed=2)
    a, b, a0 = _bounds(d, N)
    G.set_fp64_engine(engine)
    try:
        G.set_option("test_stall", 1)
        try:
            with pytest.raises(EfeError) as e:
                G.chfsi_step(to_dev(X), m, a, b, a0, precision=prec, fp64_tail=0)
            assert e.value.code == 5
        finally:
            G.set_option("test_stall", 0)
        ref = chebyshev_filter_scaled(d.apply_Htilde, X, m, a, b, a0)
        Xd = to_dev(X)
        G.chfsi_step(Xd, m, a, b, a0, precision=prec, fp64_tail=0)
        assert rel_err(Xd, ref) < (1e-5 if prec == "tf32x3" else 1e-8)
    finally:
        G.set_fp64_engine("dfma")


# --- heavy nuclei and the classical-only basis (the DoF x degree comparison) -----

def test_heavy_z_products_and_filter():
    """Heavy-Z stand-in (Z = 79, Slater 1s/2s/2p of a gold-like core, seeded
    Gaussian perturbation) on a 2x2x2-cell mesh: H, M, M^-1 products and a
    degree-7 FP64 filter against the oracle, and the FP64-grade tensor-core
    engine against the same oracle values."""
    from oracle.chfsi import chebyshev_filter_scaled
    from oracle.operators import Discretisation
    s = W.tiny_heavy()
    d = Discretisation(s)
    G = gpu_system(s)
    X = W.random_block(s, 12, seed=3)
    Xd = to_dev(X)
    assert rel_err(G.apply_H(Xd), d.apply_H_assembled(X)) < 1e-11
    assert rel_err(G.apply_M(Xd), d.apply_M_assembled(X)) < 1e-12
    assert rel_err(G.apply_Minv(Xd), d.apply_Minv_block(X)) < 1e-10
    a, b, a0 = _bounds(d, 12)
    ref = chebyshev_filter_scaled(d.apply_Htilde, X, 7, a, b, a0)
    for engine in ("dfma", "tensor"):
        G.set_fp64_engine(engine)
        try:
            Xf = to_dev(X)
            G.chfsi_step(Xf, 7, a, b, a0, precision="fp64")
        finally:
            G.set_fp64_engine("dfma")
        assert rel_err(Xf, ref) < 1e-8, engine


def test_bare_z14_enriched_closed_form():
    """A bare Z = 14 nucleus in a 20-bohr box with hydrogenic 1s/2s/2p enrichment
    on 6^3 coarse cells (3.3 bohr): the GPU's converged FP64 ChFSI eigenvalues
    against the oracle's assembled problem (sparse shift-invert, 1e-6 Ha) and
    against the closed form -Z^2/2n^2 (1s -98, n = 2 -24.5 Ha) within 5e-4 Ha."""
    import scipy.sparse.linalg as ssl
    from oracle.operators import Discretisation
    s = W.bare_nucleus(Z=14.0)
    G = gpu_system(s)
    X = to_dev(W.initial_block(s, 8, seed=1))
    eps, res, it, b = G.solve(X, 20, tol=1e-8, v0=to_dev(W.lanczos_start(s)), n_conv=5)
    assert res[:5].max() < 1e-8
    d = Discretisation(s)
    act = np.nonzero(d.active)[0]
    H = d.H[act][:, act].tocsc()
    M = d.M[act][:, act].tocsc()
    ref = np.sort(ssl.eigsh(H, k=5, M=M, sigma=-100.0, which="LM")[0])
    np.testing.assert_allclose(eps[:5], ref, atol=1e-6)
    np.testing.assert_allclose(eps[:5], [-98.0, -24.5, -24.5, -24.5, -24.5], atol=5e-4)


def test_bare_z14_classical_only_products():
    """The classical-only basis (n_E = 0) on a mesh graded towards a Z = 14
    nucleus (the basis of the DoF x degree comparison's classical runs): H and
    M^-1 products against the oracle."""
    from oracle.operators import Discretisation
    s = W.bare_nucleus(Z=14.0, enriched=False, h_min=0.8, half=4.0, h_max=2.0)
    d = Discretisation(s)
    G = gpu_system(s)
    X = W.random_block(s, 9, seed=6)
    Xd = to_dev(X)
    assert rel_err(G.apply_H(Xd), d.apply_H_assembled(X)) < 1e-11
    assert rel_err(G.apply_Minv(Xd), d.apply_Minv_block(X)) < 1e-12
