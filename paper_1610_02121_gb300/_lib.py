"""ctypes binding of the C ABI in include/efe.h (argument marshalling only).

Every step of the computation runs in the CUDA library ``libefe.so``; this
module only converts Python/NumPy descriptions into the C descriptors and
passes device pointers of torch tensors plus the current CUDA stream.  There
is no fallback: if the library is missing, importing this module raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libefe.so")

EFE_OK = 0
ERRORS = {1: "EFE_ERR_ARG", 2: "EFE_ERR_CUDA", 3: "EFE_ERR_CHOL", 4: "EFE_ERR_NOCONV",
          5: "EFE_ERR_TIMEOUT", 6: "EFE_ERR_NAN", 7: "EFE_ERR_ALLOC", 8: "EFE_ERR_STATE"}
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "tf32x3": 4}

# the symbols declared in include/efe.h
SYMBOLS = ["efe_create", "efe_destroy", "efe_last_error", "efe_sizes", "efe_qpoints", "efe_set_potential",
           "efe_set_potential_analytic", "efe_reserve", "efe_apply_H", "efe_apply_M", "efe_apply_Minv",
           "efe_upper_bound", "efe_chfsi_step", "efe_rayleigh_ritz", "efe_rr_shifted_passes", "efe_enable_timing",
           "efe_kernel_stats", "efe_kernel_stats_fp64",
           "efe_launch_count", "efe_apply_M_noalloc", "efe_set_fp64_engine", "efe_set_option", "efe_density", "efe_xc_lda",
           "efe_hartree", "efe_fermi", "efe_anderson", "efe_scf_init", "efe_scf_step", "efe_sad_density",
           "efe_descriptors", "efe_learned_density", "efe_density_log_ratio", "efe_mlp_param_count",
           "efe_mlp_work_elems", "efe_mlp_scratch_elems", "efe_mlp_forward", "efe_mlp_backward", "efe_wmse",
           "efe_adam", "efe_autotune", "efe_batch_create", "efe_batch_destroy", "efe_batch_last_error",
           "efe_batch_graph_nodes", "efe_batch_chfsi_step"]


class EfeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(C.Structure):
    _fields_ = [("degree", C.c_int32), ("n_cells", C.c_int32 * 3), ("breaks", C.POINTER(C.c_double) * 3),
                ("n_gauss", C.c_int32)]


class AtomsDesc(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("xyz", C.POINTER(C.c_double)), ("Z", C.POINTER(C.c_double))]


class BasisDesc(C.Structure):
    _fields_ = [("n_funcs", C.c_int32), ("atom", C.POINTER(C.c_int32)), ("n", C.POINTER(C.c_int32)),
                ("l", C.POINTER(C.c_int32)), ("m", C.POINTER(C.c_int32)), ("kind", C.POINTER(C.c_int32)),
                ("zeta", C.POINTER(C.c_double)), ("r0", C.POINTER(C.c_double)), ("t", C.POINTER(C.c_double)),
                ("quad_tau", C.c_double), ("quad_max_depth", C.c_int32), ("quad_n", C.c_int32)]


class PotentialDesc(C.Structure):
    _fields_ = [("nuclear", C.c_int32), ("n_terms", C.c_int32), ("A", C.POINTER(C.c_double)),
                ("s", C.POINTER(C.c_double)), ("c", C.POINTER(C.c_double)), ("omega", C.c_double)]


class ScfParams(C.Structure):
    _fields_ = [("n_electrons", C.c_double), ("kT", C.c_double), ("mix_beta", C.c_double), ("n_hist", C.c_int32),
                ("poisson_tol", C.c_double), ("poisson_max_steps", C.c_int32), ("lanczos_k", C.c_int32)]


class ScfResult(C.Structure):
    _fields_ = [("band", C.c_double), ("xc", C.c_double), ("hartree", C.c_double), ("zz", C.c_double),
                ("double_counting", C.c_double), ("total", C.c_double), ("fermi_level", C.c_double),
                ("drho", C.c_double), ("n_out", C.c_double), ("upper_bound", C.c_double),
                ("poisson_steps", C.c_int32), ("filter_passes", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AtomShells(C.Structure):
    _fields_ = [("n_shells", C.c_int32), ("n", C.c_int32 * 3), ("zeta", C.c_double * 3), ("occ", C.c_double * 3)]


class DescParams(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("species_Z", C.c_double * 4), ("n_radial", C.c_int32),
                ("radial_mu", C.c_double * 16), ("radial_sigma", C.c_double), ("n_ang", C.c_int32),
                ("ang_mu", C.c_double * 8), ("ang_sigma", C.c_double), ("r_cut", C.c_double),
                ("standardise", C.c_int32), ("offset", C.c_double * 96), ("scale", C.c_double * 96)]


class MlpShape(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("dims", C.c_int32 * 9)]


KB_HA_PER_K = 3.166811563e-6   # Boltzmann constant (Ha/K)


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    P64 = C.POINTER(C.c_int64)
    PD = C.POINTER(C.c_double)
    sig = {
        "efe_create": [C.POINTER(MeshDesc), C.POINTER(AtomsDesc), C.POINTER(BasisDesc), C.POINTER(vp)],
        "efe_destroy": [vp],
        "efe_last_error": [vp],
        "efe_sizes": [vp, P64, P64, P64, P64, P64],
        "efe_qpoints": [vp, vp, vp],
        "efe_set_potential": [vp, vp, vp],
        "efe_set_potential_analytic": [vp, C.POINTER(PotentialDesc), vp],
        "efe_reserve": [vp, i32],
        "efe_apply_H": [vp, vp, i64, i32, vp, i64, vp],
        "efe_apply_M": [vp, vp, i64, i32, vp, i64, vp],
        "efe_apply_Minv": [vp, vp, i64, i32, vp, i64, vp],
        "efe_upper_bound": [vp, vp, i32, PD, vp],
        "efe_chfsi_step": [vp, vp, i64, i32, i32, dbl, dbl, dbl, i32, i32, vp],
        "efe_rayleigh_ritz": [vp, vp, i64, i32, PD, PD, vp],
        "efe_enable_timing": [vp, i32],
        "efe_kernel_stats": [vp, P64, PD, P64, i32],
        "efe_kernel_stats_fp64": [vp, P64, PD, PD, i32],
        "efe_rr_shifted_passes": [vp, P64],
        "efe_launch_count": [P64],
        "efe_apply_M_noalloc": [vp, vp, i64, i32, vp, i64, vp],
        "efe_set_fp64_engine": [vp, i32],
        "efe_set_option": [vp, i32, i64],
        "efe_density": [vp, vp, i64, i32, vp, vp, i32, vp],
        "efe_xc_lda": [vp, vp, vp, vp, vp],
        "efe_hartree": [vp, vp, vp, vp, dbl, i32, C.POINTER(C.c_int32), vp],
        "efe_fermi": [PD, i32, dbl, dbl, PD, PD],
        "efe_anderson": [vp, vp, vp, i32, dbl, vp, vp],
        "efe_scf_init": [vp, C.POINTER(ScfParams), vp],
        "efe_scf_step": [vp, vp, i64, i32, i32, i32, i32, i32, vp, vp, PD, PD, C.POINTER(ScfResult), vp],
        "efe_sad_density": [vp, C.POINTER(AtomShells), dbl, vp, vp],
        "efe_descriptors": [vp, C.POINTER(DescParams), vp, i32, vp],
        "efe_learned_density": [vp, vp, vp, dbl, dbl, vp, i32, vp],
        "efe_density_log_ratio": [vp, vp, vp, dbl, vp, i32, vp],
        "efe_mlp_param_count": [C.POINTER(MlpShape)],
        "efe_mlp_work_elems": [C.POINTER(MlpShape), i64],
        "efe_mlp_scratch_elems": [C.POINTER(MlpShape), i64],
        "efe_mlp_forward": [C.POINTER(MlpShape), vp, vp, i64, vp, vp, i32, vp],
        "efe_mlp_backward": [C.POINTER(MlpShape), vp, vp, i64, vp, vp, vp, vp, i32, vp],
        "efe_wmse": [vp, vp, vp, i64, vp, PD, i32, vp],
        "efe_adam": [vp, vp, vp, vp, i64, dbl, dbl, dbl, dbl, i32, i32, vp],
        "efe_autotune": [vp, i32, i32, C.POINTER(C.c_int32), PD],
        "efe_batch_create": [C.POINTER(vp), i32, C.POINTER(vp)],
        "efe_batch_destroy": [vp],
        "efe_batch_last_error": [vp],
        "efe_batch_graph_nodes": [vp, P64, P64],
        "efe_batch_chfsi_step": [vp, C.POINTER(vp), P64, C.POINTER(C.c_int32), i32, PD, PD, PD, i32, i32, i32, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = (C.c_char_p if name in ("efe_last_error", "efe_batch_last_error") else
                     C.c_int64 if name in ("efe_mlp_param_count", "efe_mlp_work_elems", "efe_mlp_scratch_elems")
                     else C.c_int)
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def launch_count():
    n = C.c_int64()
    lib().efe_launch_count(C.byref(n))
    return n.value


def fermi(eps, n_electrons, kT):
    """Fermi-Dirac occupations and Fermi level (host routine of the library)."""
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    occ = np.zeros_like(eps)
    mu = C.c_double()
    rc = lib().efe_fermi(_dptr(eps), len(eps), float(n_electrons), float(kT), _dptr(occ), C.byref(mu))
    if rc != EFE_OK:
        raise EfeError(rc, "efe_fermi: not enough states for the electron count")
    return occ, mu.value


def check_block(X, rows, like=None):
    """Validate a vector block before its pointer goes to the library: a 2-D FP64
    tensor with ``rows`` rows, unit column stride and leading dimension >= N, on
    a CUDA device; with ``like``, also the same shape as that block.  Raises
    ValueError (shape, dtype, strides) or TypeError (not a tensor) before any
    device work, so that a wrong block never reaches a kernel."""
    if not hasattr(X, "dim") or not hasattr(X, "dtype"):
        raise TypeError("vector block must be a torch tensor")
    if X.dim() != 2:
        raise ValueError(f"vector block must be 2-D, got {X.dim()}-D")
    if str(X.dtype) != "torch.float64":
        raise ValueError(f"vector block must be float64, got {X.dtype}")
    if X.shape[0] != rows:
        raise ValueError(f"vector block has {X.shape[0]} rows, the system has {rows} (nodes + enrichment)")
    if X.shape[1] < 1:
        raise ValueError("vector block has no columns")
    if X.stride(1) != 1 or X.stride(0) < X.shape[1]:
        raise ValueError("vector block needs unit column stride and leading dimension >= N")
    if like is not None and tuple(X.shape) != tuple(like.shape):
        raise ValueError(f"output block shape {tuple(X.shape)} differs from input {tuple(like.shape)}")
    if not X.is_cuda:
        raise ValueError("vector block must live on a CUDA device")
    return C.c_void_p(X.data_ptr()), X.stride(0), X.shape[1]


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class System:
    """One enriched-FE discretisation living on the current CUDA device."""

    def __init__(self, system):
        import torch  # device memory and streams only
        self._torch = torch
        self.L = lib()
        self.system = system
        self._keep = []
        md = MeshDesc()
        md.degree = system["p"]
        for d in range(3):
            b = np.ascontiguousarray(system["breaks"][d], dtype=np.float64)
            self._keep.append(b)
            md.n_cells[d] = len(b) - 1
            md.breaks[d] = _dptr(b)
        md.n_gauss = system["n_gauss"]
        ad = AtomsDesc()
        xyz = np.ascontiguousarray(system["atoms"], dtype=np.float64).reshape(-1)
        Z = np.ascontiguousarray(system["Z"], dtype=np.float64)
        self._keep += [xyz, Z]
        ad.n_atoms = len(Z)
        ad.xyz = _dptr(xyz)
        ad.Z = _dptr(Z)
        bd = BasisDesc()
        f = system["funcs"]
        cols = {
            "atom": np.array([x["atom"] for x in f], dtype=np.int32),
            "n": np.array([x["n"] for x in f], dtype=np.int32),
            "l": np.array([x["l"] for x in f], dtype=np.int32),
            "m": np.array([x["m"] for x in f], dtype=np.int32),
            "kind": np.array([0 if x["kind"] == "hydrogenic" else 1 for x in f], dtype=np.int32),
        }
        dcols = {k: np.array([x[k] for x in f], dtype=np.float64) for k in ("zeta", "r0", "t")}
        self._keep += list(cols.values()) + list(dcols.values())
        bd.n_funcs = len(f)
        for k, v in cols.items():
            setattr(bd, k, _iptr(v))
        for k, v in dcols.items():
            setattr(bd, k, _dptr(v))
        q = system["quad"]
        bd.quad_tau = q["tau"]
        bd.quad_max_depth = q["max_depth"]
        bd.quad_n = q["n"]
        h = C.c_void_p()
        rc = self.L.efe_create(C.byref(md), C.byref(ad), C.byref(bd), C.byref(h))
        self.h = h
        if rc != EFE_OK:
            msg = self.L.efe_last_error(h).decode() if h.value else "efe_create failed"
            self.close()
            raise EfeError(rc, msg)
        n = [C.c_int64() for _ in range(5)]
        self._check(self.L.efe_sizes(h, *[C.byref(x) for x in n]))
        self.n_nodes, self.n_enrich, self.n_qpoints, self.n_cells, self.n_coupling = [x.value for x in n]
        self.rows = self.n_nodes + self.n_enrich

    # -- plumbing ------------------------------------------------------------
    def _check(self, rc):
        if rc != EFE_OK:
            raise EfeError(rc, self.L.efe_last_error(self.h).decode())

    def _stream(self):
        return C.c_void_p(self._torch.cuda.current_stream().cuda_stream)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.efe_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _block(self, X, like=None):
        return check_block(X, self.rows, like)

    # -- API -------------------------------------------------------------------
    def qpoints(self):
        t = self._torch.empty((self.n_qpoints, 4), dtype=self._torch.float64, device="cuda")
        self._check(self.L.efe_qpoints(self.h, C.c_void_p(t.data_ptr()), self._stream()))
        return t

    def set_potential(self, V):
        assert V.is_cuda and V.dtype == self._torch.float64 and V.numel() == self.n_qpoints
        self._check(self.L.efe_set_potential(self.h, C.c_void_p(V.data_ptr()), self._stream()))

    def set_potential_analytic(self, pot=None):
        pot = pot if pot is not None else self.system["potential"]
        A = np.ascontiguousarray(pot["gauss_A"], dtype=np.float64)
        s = np.ascontiguousarray(pot["gauss_s"], dtype=np.float64)
        c = np.ascontiguousarray(pot["gauss_c"], dtype=np.float64).reshape(-1)
        pd = PotentialDesc(int(bool(pot["nuclear"])), len(A), _dptr(A), _dptr(s), _dptr(c), float(pot["omega"]))
        self._check(self.L.efe_set_potential_analytic(self.h, C.byref(pd), self._stream()))

    def reserve(self, N):
        self._check(self.L.efe_reserve(self.h, int(N)))

    def _apply(self, fn, X, Y=None):
        px, ldx, N = self._block(X)
        if Y is None:
            Y = self._torch.empty_like(X)
        py, ldy, _ = self._block(Y, like=X)
        self._check(fn(self.h, px, ldx, N, py, ldy, self._stream()))
        return Y

    def apply_H(self, X, Y=None):
        return self._apply(self.L.efe_apply_H, X, Y)

    def apply_M(self, X, Y=None):
        return self._apply(self.L.efe_apply_M, X, Y)

    def apply_M_noalloc(self, X, Y):
        """M^E X through the allocation-free entry point (caller provides Y)."""
        return self._apply(self.L.efe_apply_M_noalloc, X, Y)

    def apply_Minv(self, X, Y=None):
        return self._apply(self.L.efe_apply_Minv, X, Y)

    def upper_bound(self, v0, k=10):
        b = C.c_double()
        self._check(self.L.efe_upper_bound(self.h, C.c_void_p(v0.data_ptr()), int(k), C.byref(b), self._stream()))
        return b.value

    def chfsi_step(self, X, m, a, b, a0, precision="fp64", fp64_tail=0):
        px, ldx, N = self._block(X)
        self._check(self.L.efe_chfsi_step(self.h, px, ldx, N, int(m), float(a), float(b), float(a0),
                                          PREC[precision], int(fp64_tail), self._stream()))
        return X

    def rayleigh_ritz(self, X, residuals=True):
        """Cholesky-QR + Rayleigh-Ritz in place; returns the Ritz values and (when
        ``residuals``) the residual norms, else None."""
        px, ldx, N = self._block(X)
        eig = np.zeros(N)
        res = np.zeros(N) if residuals else None
        self._check(self.L.efe_rayleigh_ritz(self.h, px, ldx, N, _dptr(eig), _dptr(res) if residuals else None,
                                             self._stream()))
        return eig, res

    def solve(self, X, m, tol=1e-8, max_iter=200, precision="fp64", fp64_tail=0, v0=None, n_conv=None,
              k_lanczos=10):
        """ChFSI for the current potential (Sec. V): Rayleigh-Ritz on X for a and
        a0, a Lanczos bound b, then filter -> Cholesky-QR + Rayleigh-Ritz until the
        residuals of the lowest ``n_conv`` Ritz pairs are below ``tol``.  Loop
        control only; every step is a library call."""
        eps, res = self.rayleigh_ritz(X)
        if v0 is None:
            v0 = X[:, -1].contiguous()
        b = self.upper_bound(v0, k_lanczos)
        it = 0
        for it in range(1, max_iter + 1):
            self.chfsi_step(X, m, eps.max(), b, eps.min(), precision=precision, fp64_tail=fp64_tail)
            eps, res = self.rayleigh_ritz(X)
            if res[:n_conv].max() < tol:
                break
        return eps, res, it, b

    # -- self-consistent field ---------------------------------------------------
    def _qvec(self, t):
        assert t.is_cuda and t.dtype == self._torch.float64 and t.is_contiguous() and t.numel() == self.n_qpoints
        return C.c_void_p(t.data_ptr())

    def density(self, X, occ, rho=None, precision="fp64"):
        """rho = 2 sum_i occ_i psi_i^2 at the quadrature points (Eq. Rho); precision "fp64" or
        "fp32" (orbital values in FP32, squares and sums in FP64)."""
        px, ldx, N = self._block(X)
        occ = self._torch.as_tensor(occ, dtype=self._torch.float64, device=X.device).contiguous()
        if rho is None:
            rho = self._torch.empty(self.n_qpoints, dtype=self._torch.float64, device=X.device)
        self._check(self.L.efe_density(self.h, px, ldx, N, C.c_void_p(occ.data_ptr()), self._qvec(rho),
                                       PREC[precision], self._stream()))
        return rho

    def xc_lda(self, rho):
        exc = self._torch.empty_like(rho)
        vxc = self._torch.empty_like(rho)
        self._check(self.L.efe_xc_lda(self.h, self._qvec(rho), self._qvec(exc), self._qvec(vxc), self._stream()))
        return exc, vxc

    def hartree(self, rho, phi=None, tol=1e-12, max_steps=3):
        """V_H at the quadrature points, the nodal potential and the number of exact-solve corrections."""
        vh = self._torch.empty_like(rho)
        if phi is None:
            phi = self._torch.zeros(self.n_nodes, dtype=self._torch.float64, device=rho.device)
        it = C.c_int32()
        self._check(self.L.efe_hartree(self.h, self._qvec(rho), self._qvec(vh), C.c_void_p(phi.data_ptr()),
                                       float(tol), int(max_steps), C.byref(it), self._stream()))
        return vh, phi, it.value

    def anderson(self, rho_in_hist, rho_out_hist, beta):
        """Next input density from n (rho_in, rho_out) pairs (n x n_qpoints tensors, oldest first)."""
        n = rho_in_hist.shape[0]
        assert rho_in_hist.is_contiguous() and rho_out_hist.is_contiguous() and rho_out_hist.shape[0] == n
        out = self._torch.empty(self.n_qpoints, dtype=self._torch.float64, device=rho_in_hist.device)
        self._check(self.L.efe_anderson(self.h, C.c_void_p(rho_in_hist.data_ptr()),
                                        C.c_void_p(rho_out_hist.data_ptr()), int(n), float(beta),
                                        C.c_void_p(out.data_ptr()), self._stream()))
        return out

    def scf_init(self, n_electrons, kT=500 * KB_HA_PER_K, beta=0.5, n_hist=5, poisson_tol=1e-12,
                 poisson_max_steps=3, lanczos_k=10):
        p = ScfParams(float(n_electrons), float(kT), float(beta), int(n_hist), float(poisson_tol),
                      int(poisson_max_steps), int(lanczos_k))
        self._check(self.L.efe_scf_init(self.h, C.byref(p), self._stream()))

    def scf_step(self, X, rho_in, rho_out, m, passes=1, precision="fp64", fp64_tail=0):
        """One SCF iteration (Sec. V); rho_in is overwritten with the next mixed density."""
        px, ldx, N = self._block(X)
        eig = np.zeros(N)
        occ = np.zeros(N)
        r = ScfResult()
        self._check(self.L.efe_scf_step(self.h, px, ldx, N, int(m), int(passes), PREC[precision], int(fp64_tail),
                                        self._qvec(rho_in), self._qvec(rho_out), _dptr(eig), _dptr(occ),
                                        C.byref(r), self._stream()))
        out = r.as_dict()
        out["eig"] = eig
        out["occ"] = occ
        return out

    # -- learned initial density -------------------------------------------------
    def sad_density(self, shells, n_electrons=0.0):
        """Superposition of atomic densities; shells[I] = [(n, zeta, electrons), ...] per atom."""
        arr = (AtomShells * max(1, len(shells)))()
        for i, sh in enumerate(shells):
            arr[i].n_shells = len(sh)
            for k, (n, z, o) in enumerate(sh):
                arr[i].n[k] = int(n)
                arr[i].zeta[k] = float(z)
                arr[i].occ[k] = float(o)
        rho = self._torch.empty(self.n_qpoints, dtype=self._torch.float64, device="cuda")
        self._check(self.L.efe_sad_density(self.h, arr, float(n_electrons), self._qvec(rho), self._stream()))
        return rho

    def descriptors(self, params, precision="fp32"):
        dt = self._torch.float32 if precision == "fp32" else self._torch.float64
        nf = params.n_species * (params.n_radial + params.n_ang)
        D = self._torch.empty((self.n_qpoints, nf), dtype=dt, device="cuda")
        self._check(self.L.efe_descriptors(self.h, C.byref(params), C.c_void_p(D.data_ptr()), PREC[precision],
                                           self._stream()))
        return D

    def learned_density(self, rho_sad, y, floor, n_electrons):
        prec = "fp32" if y.dtype == self._torch.float32 else "fp64"
        rho = self._torch.empty_like(rho_sad)
        self._check(self.L.efe_learned_density(self.h, self._qvec(rho_sad), C.c_void_p(y.data_ptr()), float(floor),
                                               float(n_electrons), self._qvec(rho), PREC[prec], self._stream()))
        return rho

    def density_log_ratio(self, rho, rho_sad, floor, precision="fp32"):
        dt = self._torch.float32 if precision == "fp32" else self._torch.float64
        y = self._torch.empty(self.n_qpoints, dtype=dt, device="cuda")
        self._check(self.L.efe_density_log_ratio(self.h, self._qvec(rho), self._qvec(rho_sad), float(floor),
                                                 C.c_void_p(y.data_ptr()), PREC[precision], self._stream()))
        return y

    def autotune(self, N, precision="tf32x3"):
        """Pick the tensor-core cell kernel's column tile for N columns; returns (tile, ms per tile)."""
        t = C.c_int32()
        ms = np.zeros(3)
        self._check(self.L.efe_autotune(self.h, int(N), PREC[precision], C.byref(t), _dptr(ms)))
        return t.value, ms

    OPTIONS = {"grid_cap": 1, "image_rows": 2, "rr_panels": 3, "dense_blocked": 4, "coupling_sparse": 5,
               "test_stall": 6, "coupling_cols": 7}

    def set_option(self, name, value):
        """Test/tuning control of the library (EFE_OPT_*): grid_cap (CTAs of the
        persistent tensor-core kernels), image_rows (FP64-engine image panel rows),
        rr_panels (1: panelled Rayleigh-Ritz), dense_blocked (1: multi-CTA dense
        kernels), coupling_sparse (1: many-function mixed coupling); 0 restores
        the size-based default."""
        self._check(self.L.efe_set_option(self.h, self.OPTIONS[name], int(value)))

    def set_grid_cap(self, max_ctas):
        """Cap the persistent tensor-core kernels at max_ctas CTAs (0: one per SM)."""
        self.set_option("grid_cap", max_ctas)

    def set_fp64_engine(self, engine):
        """0: FP64 DFMA products; 1 (or "tensor"): FP64-grade products on the BF16 tensor cores."""
        e = {"dfma": 0, "tensor": 1}.get(engine, engine)
        self._check(self.L.efe_set_fp64_engine(self.h, int(e)))

    def enable_timing(self, on=True):
        self._check(self.L.efe_enable_timing(self.h, int(bool(on))))

    def kernel_stats_fp64(self, reset=True):
        """FP64 tensor engine: (launches, total ms, algorithmic FP64 flops) since the last reset."""
        n = C.c_int64()
        ms = C.c_double()
        fl = C.c_double()
        self._check(self.L.efe_kernel_stats_fp64(self.h, C.byref(n), C.byref(ms), C.byref(fl), int(bool(reset))))
        return n.value, ms.value, fl.value

    def rr_shifted_passes(self):
        """Shifted Cholesky-QR passes Rayleigh-Ritz has needed on this system so far."""
        n = C.c_int64()
        self._check(self.L.efe_rr_shifted_passes(self.h, C.byref(n)))
        return n.value

    def kernel_stats(self, reset=True):
        n = C.c_int64()
        ms = C.c_double()
        cc = C.c_int64()
        self._check(self.L.efe_kernel_stats(self.h, C.byref(n), C.byref(ms), C.byref(cc), int(bool(reset))))
        return n.value, ms.value, cc.value


class Mlp:
    """Fully connected network on the device (SiLU hidden layers, scalar output):
    flat parameter tensor, forward / backward / Adam through the C ABI."""

    def __init__(self, dims, precision="fp32", params=None, seed=0):
        import torch
        self._torch = torch
        self.L = lib()
        self.dims = list(dims)
        self.shape = MlpShape(len(dims) - 1, (C.c_int32 * 9)(*(list(dims) + [0] * (9 - len(dims)))))
        self.prec = precision
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        self.n_params = self.L.efe_mlp_param_count(C.byref(self.shape))
        if self.n_params < 0:
            raise EfeError(1, "invalid network shape")
        if params is None:
            rng = np.random.Generator(np.random.PCG64(seed))
            parts = []
            for a, b in zip(dims[:-1], dims[1:]):
                lim = 1.0 / np.sqrt(a)
                parts.append(rng.uniform(-lim, lim, size=a * b))
                parts.append(np.zeros(b))
            params = np.concatenate(parts)
        self.params = torch.as_tensor(np.asarray(params), dtype=self.dtype).cuda().contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self._n = -1

    def _bufs(self, n):
        if n > self._n:
            t = self._torch
            self.work = t.empty(self.L.efe_mlp_work_elems(C.byref(self.shape), n), dtype=self.dtype, device="cuda")
            self.scratch = t.empty(self.L.efe_mlp_scratch_elems(C.byref(self.shape), n), dtype=self.dtype,
                                   device="cuda")
            self._n = n

    def _stream(self):
        return C.c_void_p(self._torch.cuda.current_stream().cuda_stream)

    def _chk(self, rc, what):
        if rc != EFE_OK:
            raise EfeError(rc, what)

    def forward(self, X):
        n = X.shape[0]
        self._bufs(n)
        y = self._torch.empty(n, dtype=self.dtype, device="cuda")
        self._chk(self.L.efe_mlp_forward(C.byref(self.shape), C.c_void_p(self.params.data_ptr()),
                                         C.c_void_p(X.data_ptr()), n, C.c_void_p(y.data_ptr()),
                                         C.c_void_p(self.work.data_ptr()), PREC[self.prec], self._stream()),
                  "efe_mlp_forward")
        return y

    def backward(self, X, dy):
        """Gradients of sum dy * y for the X of the last forward call."""
        n = X.shape[0]
        g = self._torch.empty_like(self.params)
        self._chk(self.L.efe_mlp_backward(C.byref(self.shape), C.c_void_p(self.params.data_ptr()),
                                          C.c_void_p(X.data_ptr()), n, C.c_void_p(self.work.data_ptr()),
                                          C.c_void_p(dy.data_ptr()), C.c_void_p(g.data_ptr()),
                                          C.c_void_p(self.scratch.data_ptr()), PREC[self.prec], self._stream()),
                  "efe_mlp_backward")
        return g

    def wmse(self, yh, y, c):
        dy = self._torch.empty_like(yh)
        loss = C.c_double()
        self._chk(self.L.efe_wmse(C.c_void_p(yh.data_ptr()), C.c_void_p(y.data_ptr()), C.c_void_p(c.data_ptr()),
                                  yh.numel(), C.c_void_p(dy.data_ptr()), C.byref(loss), PREC[self.prec],
                                  self._stream()), "efe_wmse")
        return loss.value, dy

    def adam(self, g, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        self._chk(self.L.efe_adam(C.c_void_p(self.params.data_ptr()), C.c_void_p(g.data_ptr()),
                                  C.c_void_p(self.m.data_ptr()), C.c_void_p(self.v.data_ptr()), self.n_params,
                                  float(lr), float(b1), float(b2), float(eps), self.t, PREC[self.prec],
                                  self._stream()), "efe_adam")


class Batch:
    """Independent systems whose ChFSI filter steps run as one CUDA graph."""

    def __init__(self, systems):
        self.L = lib()
        self.systems = list(systems)
        arr = (C.c_void_p * len(self.systems))(*[s.h.value for s in self.systems])
        b = C.c_void_p()
        rc = self.L.efe_batch_create(arr, len(self.systems), C.byref(b))
        self.b = b
        if rc != EFE_OK:
            msg = self.L.efe_batch_last_error(b).decode() if b.value else "efe_batch_create failed"
            self.close()
            raise EfeError(rc, msg)

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            self.L.efe_batch_destroy(self.b)
            self.b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def chfsi_step(self, Xs, m, a, b, a0, precision="fp64", fp64_tail=0, graph=True):
        import torch
        n = len(self.systems)
        ptr = (C.c_void_p * n)(*[X.data_ptr() for X in Xs])
        ld = np.array([X.stride(0) for X in Xs], dtype=np.int64)
        N = np.array([X.shape[1] for X in Xs], dtype=np.int32)
        av, bv, a0v = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, a0))
        rc = self.L.efe_batch_chfsi_step(self.b, ptr, ld.ctypes.data_as(C.POINTER(C.c_int64)),
                                         N.ctypes.data_as(C.POINTER(C.c_int32)), int(m), _dptr(av), _dptr(bv),
                                         _dptr(a0v), PREC[precision], int(fp64_tail), int(bool(graph)),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
        if rc != EFE_OK:
            raise EfeError(rc, self.L.efe_batch_last_error(self.b).decode())

    def graph_nodes(self):
        a, k = C.c_int64(), C.c_int64()
        self.L.efe_batch_graph_nodes(self.b, C.byref(a), C.byref(k))
        return a.value, k.value
