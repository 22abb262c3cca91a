"""ctypes binding of the hub C ABI (include/hub.h): argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HUB_F64, HUB_F32, HUB_MIXED_BF16, HUB_MIXED_F16 = 0, 1, 2, 3
STATUS_NAMES = {0: "HUB_OK", -1: "HUB_EINVAL", -2: "HUB_ENOMEM", -3: "HUB_ECUDA",
                -4: "HUB_ENOTSPD", -5: "HUB_ENONFINITE", -6: "HUB_ENOCONV", -7: "HUB_ETIMEOUT"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def library_path() -> str:
    return os.path.join(_HERE, "libhub.so")


class HubError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class scf_params(C.Structure):
    _fields_ = [("nspin", C.c_int), ("ncol", C.c_int), ("ld", C.c_int), ("degree", C.c_int),
                ("max_iter", C.c_int), ("first_passes", C.c_int), ("lanczos_steps", C.c_int),
                ("pulay_history", C.c_int), ("natoms", C.c_int), ("pulay_beta", C.c_double),
                ("kT", C.c_double), ("n_elec", C.c_double), ("tol_e_atom", C.c_double),
                ("tol_D", C.c_double), ("ladder", C.c_int), ("ladder_tol", C.c_double),
                ("density", C.c_int), ("kerker_kappa", C.c_double), ("tol_rho", C.c_double),
                ("cg_tol", C.c_double)]


class scf_result(C.Structure):
    _fields_ = [("iter", C.c_int), ("converged", C.c_int), ("E", C.c_double),
                ("E_band", C.c_double), ("E_U", C.c_double), ("dE", C.c_double),
                ("dD", C.c_double), ("mu", C.c_double), ("bf16_terms", C.c_int),
                ("jacobi_sweeps", C.c_int), ("E_H", C.c_double), ("E_x", C.c_double),
                ("drho", C.c_double), ("cg_iters", C.c_int)]


_P, _I, _D = C.c_void_p, C.c_int, C.c_double
_PD, _PI = C.POINTER(C.c_double), C.POINTER(C.c_int)
_SIGS = {
    "hub_create_grid": [C.POINTER(C.c_void_p), _I, _I, _I, _D, _D, _D, _I, _I, _PD, _I, _P],
    "hub_destroy": [_P],
    "hub_last_error": [_P],
    "hub_set_veff": [_P, _P],
    "hub_set_atoms_projectors": [_P, _I, _PD, _PI, _PI, _PD, _PD, _PD, _PI, _PD, _PD, _PD],
    "hub_num_hubbard_atoms": [_P, _PI],
    "hub_set_occupation_matrix": [_P, _I, _PD, _PD],
    "hub_apply_H": [_P, _I, _P, _P, _I, _I],
    "hub_chefsi_filter": [_P, _I, _P, _I, _I, _I, _D, _D, _D, _P],
    "hub_rayleigh_ritz": [_P, _I, _P, _I, _I, _PD, _P],
    "hub_occupation": [_P, _I, _P, _I, _I, _PD, _D, _PD, _PD, _PD],
    "hub_hubbard_forces": [_P, _I, _P, _I, _I, _PD, _D, _PD, _P],
    "hub_hubbard_stress": [_P, _I, _P, _I, _I, _PD, _D, _PD, _P],
    "hub_gram": [_P, _P, _I, _P, _I, _I, _D, _P],
    "hub_gram_noalloc": [_P, _I, _P, _I, C.c_longlong, _I, _I, _D, _P, _P],
    "hub_lanczos_bound": [_P, _I, _I, _P, _PD, _PD],
    "hub_scf_begin": [_P, C.POINTER(scf_params), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), _PD],
    "hub_scf_iterate": [_P, C.POINTER(scf_result)],
    "hub_scf_run": [_P, C.POINTER(scf_result)],
    "hub_scf_get": [_P, _PD, _PD, _PD],
    "hub_scf_density": [_P, _P],
    "hub_scf_set_density": [_P, _P],
    "hub_num_projectors": [_P, _PI],
    "hub_project": [_P, _P, _I, _I, _PD],
    "hub_expand": [_P, _PD, _I, _P, _I, _D],
    "hub_scf_forces": [_P, _PD, _PD],
    "hub_kscf_create": [C.POINTER(C.c_void_p), _I, C.POINTER(C.c_void_p), _PD, C.POINTER(scf_params),
                        C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), _PD, _PD],
    "hub_kscf_iterate": [_P, C.POINTER(scf_result)],
    "hub_kscf_run": [_P, C.POINTER(scf_result)],
    "hub_kscf_get": [_P, _PD, _PD, _PD, _PD],
    "hub_kscf_last_error": [_P],
    "hub_kscf_iterate_batch": [_I, C.POINTER(C.c_void_p), C.POINTER(scf_result), _P],
    "hub_kscf_run_batch": [_I, C.POINTER(C.c_void_p), C.POINTER(scf_result), _P],
    "hub_kscf_destroy": [_P],
    "hub_extrapolate_occupations": [_I, _I, _PD, _PD, _I, _PD, _PD, _PD],
    "hub_cutoff_radius": [_I, _D, _D, _PD],
    "hub_fermi_dirac": [_I, _PD, _PD, _D, _D, _D, _PD, _PD],
    "hub_density": [_P, _P, _I, _I, _PD, _D, _P],
    "hub_hartree": [_P, _P, _P, _D, _I, _PI, _PD],
    "hub_lda_exchange": [_P, _I, _P, _P, _P, _P, _PD],
    "hub_kerker": [_P, _P, _P, _D, _D, _I, _PI],
    "hub_version": [C.c_char_p, _I],
    "hub_set_bf16_terms": [_P, _I],
    "hub_autotune": [_P, _I, _P, _I, _I, _PI],
    "hub_batch_filter": [_I, C.POINTER(C.c_void_p), _PI, C.POINTER(C.c_void_p), _PI, _PI, _I, _PD, _PD, _PD, _P],
    "hub_descriptors": [_I, _PD, _PI, _PD, _I, _PI, _I, _D, _I, _D, _P, _P],
    "hub_mlp_create": [C.POINTER(C.c_void_p), _I, _I, _I, _I, _I, C.c_ulonglong, _P],
    "hub_mlp_destroy": [_P],
    "hub_mlp_last_error": [_P],
    "hub_mlp_num_params": [_P, C.POINTER(C.c_longlong)],
    "hub_mlp_set_params": [_P, C.POINTER(C.c_float)],
    "hub_mlp_get_params": [_P, C.POINTER(C.c_float)],
    "hub_mlp_set_normalization": [_P, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float)],
    "hub_mlp_fit_normalization": [_P, _P, _P, _I],
    "hub_mlp_forward": [_P, _P, _I, _P],
    "hub_mlp_loss_grad": [_P, _P, _P, _I, C.POINTER(C.c_float), C.POINTER(C.c_float)],
    "hub_mlp_train_step": [_P, _P, _P, _I, C.c_float, C.POINTER(C.c_float)],
    "hub_set_tuning": [_P, _I, _I, _I],
    "hub_get_tuning": [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "hub_projector_stats": [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)],
    "hub_alu_peaks": [_PD, _PD, _P],
    "hub_profile": [_P, _I],
    "hub_profile_read": [_P, _I, _PD, C.POINTER(C.c_longlong)],
    "hub_launch_count": [_P, C.POINTER(C.c_longlong)],
}

KERNEL_KINDS = ["stencil", "gather", "transform", "scatter", "gram", "gram_reduce", "rotate",
                "cholesky", "tri_inverse", "dgemm", "jacobi", "eig_misc", "occupation",
                "lanczos", "copy", "table", "force", "density"]


def batch_filter(hubs, spins, Xs, degree: int, a, b, a_low, stream=None):
    """X_i <- p_m(H_i) X_i for every system i in one CUDA graph (hub_batch_filter)."""
    import torch
    lib = load_library()
    n = len(hubs)
    if len(Xs) != n:
        raise ValueError("batch_filter: one block per system")
    for hb, x in zip(hubs, Xs):
        hb._blk(x, "batch_filter X")
    st = stream if stream is not None else torch.cuda.current_stream()
    hs = (C.c_void_p * n)(*[hb.h.value for hb in hubs])
    xs = (C.c_void_p * n)(*[x.data_ptr() for x in Xs])
    sp = np.ascontiguousarray(spins, dtype=np.int32)
    nc = np.ascontiguousarray([x.shape[0] for x in Xs], dtype=np.int32)
    ld = np.ascontiguousarray([x.shape[1] for x in Xs], dtype=np.int32)
    av, bv, lv = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, a_low))
    rc = lib.hub_batch_filter(n, hs, _iptr(sp), xs, _iptr(nc), _iptr(ld), int(degree), _dptr(av), _dptr(bv),
                              _dptr(lv), C.c_void_p(st.cuda_stream))
    if rc != 0:
        msg = lib.hub_last_error(hubs[0].h)
        raise HubError(rc, f"hub_batch_filter: {msg.decode() if msg else ''}")


def load_library(path: str | None = None) -> C.CDLL:
    """Load libhub.so (raises OSError if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or library_path()
    if not os.path.exists(p):
        raise OSError(f"libhub.so not found at {p}; build it with "
                      "`python -m paper_2507_23612_gb300.build`")
    lib = C.CDLL(p)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_char_p if name in ("hub_last_error", "hub_mlp_last_error", "hub_kscf_last_error") else C.c_int
    if path is None:
        _LIB = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(_PI)


def _tptr(t):
    """Device pointer of a torch CUDA tensor (must be contiguous)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


class Hub:
    """One grid / k-point / precision handle (hub_create_grid ... hub_destroy)."""

    def __init__(self, n, L, fd_half_order: int = 6, kpt=None, complex_: bool = False,
                 prec: int = HUB_F64, stream=None):
        import torch
        self.lib = load_library()
        self.n = tuple(int(v) for v in n)
        self.Nd = self.n[0] * self.n[1] * self.n[2]
        self.prec = prec
        self.complex = bool(complex_)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        k = np.ascontiguousarray(kpt if kpt is not None else [0.0, 0.0, 0.0], dtype=np.float64)
        rc = self.lib.hub_create_grid(C.byref(h), *self.n, *[float(x) for x in L], int(fd_half_order),
                                      int(self.complex), _dptr(k), int(prec),
                                      C.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise HubError(rc, "hub_create_grid failed")
        self.h = h
        self.nhub = 0

    # ------------------------------------------------------------------ helpers
    def _check(self, rc, what):
        if rc != 0:
            msg = self.lib.hub_last_error(self.h)
            raise HubError(rc, f"{what}: {msg.decode() if msg else ''}")

    def _blk(self, X, what):
        """A block argument: a contiguous CUDA tensor [ncol, ld] of the handle's element type
        with ld >= Nd (a wrong element size would make the kernels read past the tensor)."""
        if X.dtype != self.dtype:
            raise ValueError(f"{what}: expected {self.dtype}, got {X.dtype}")
        if X.dim() != 2 or (X.shape[0] > 0 and X.shape[1] < self.Nd):
            raise ValueError(f"{what}: expected a [ncol, ld >= {self.Nd}] block, got {tuple(X.shape)}")
        return X.shape

    def _vec(self, t, dtype, what, n=None):
        """A vector argument: a contiguous CUDA tensor of dtype with at least n (default Nd)
        elements."""
        if t.dtype != dtype:
            raise ValueError(f"{what}: expected {dtype}, got {t.dtype}")
        if t.numel() < (self.Nd if n is None else n):
            raise ValueError(f"{what}: expected at least {self.Nd if n is None else n} elements")

    @property
    def dtype(self):
        import torch
        if self.complex:
            return torch.complex128 if self.prec == HUB_F64 else torch.complex64
        return torch.float64 if self.prec == HUB_F64 else torch.float32

    def close(self):
        if getattr(self, "h", None):
            self.lib.hub_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ setup
    def set_bf16_terms(self, terms: int):
        self._check(self.lib.hub_set_bf16_terms(self.h, int(terms)), "hub_set_bf16_terms")

    def set_veff(self, veff):
        import torch
        self._vec(veff, torch.float64, "set_veff")
        self._check(self.lib.hub_set_veff(self.h, _tptr(veff)), "hub_set_veff")

    def set_atoms(self, atoms):
        """atoms: objects with pos, kb_l, kb_rs, kb_gamma, kb_rc, hub_l, hub_rs, hub_rc, hub_U."""
        nat = len(atoms)
        pos = np.ascontiguousarray([a.pos for a in atoms], dtype=np.float64).reshape(-1)
        nch = np.ascontiguousarray([len(a.kb_l) for a in atoms], dtype=np.int32)
        kb_l = np.ascontiguousarray([l for a in atoms for l in a.kb_l] or [0], dtype=np.int32)
        kb_rs = np.ascontiguousarray([r for a in atoms for r in a.kb_rs] or [1.0], dtype=np.float64)
        kb_g = np.ascontiguousarray([g for a in atoms for g in a.kb_gamma] or [0.0], dtype=np.float64)
        kb_rc = np.ascontiguousarray([a.kb_rc for a in atoms], dtype=np.float64)
        hl = np.ascontiguousarray([a.hub_l for a in atoms], dtype=np.int32)
        hrs = np.ascontiguousarray([a.hub_rs for a in atoms], dtype=np.float64)
        hrc = np.ascontiguousarray([a.hub_rc for a in atoms], dtype=np.float64)
        hU = np.ascontiguousarray([a.hub_U for a in atoms], dtype=np.float64)
        self._check(self.lib.hub_set_atoms_projectors(
            self.h, nat, _dptr(pos), _iptr(nch), _iptr(kb_l), _dptr(kb_rs), _dptr(kb_g),
            _dptr(kb_rc), _iptr(hl), _dptr(hrs), _dptr(hrc), _dptr(hU)), "hub_set_atoms_projectors")
        n = C.c_int()
        self._check(self.lib.hub_num_hubbard_atoms(self.h, C.byref(n)), "hub_num_hubbard_atoms")
        self.nhub = n.value
        self.natoms = nat

    def set_occupation_matrix(self, spin: int, D, D_im=None):
        Dr = np.ascontiguousarray(np.real(D), dtype=np.float64).reshape(-1)
        Di = None if D_im is None else np.ascontiguousarray(D_im, dtype=np.float64).reshape(-1)
        if D_im is None and np.iscomplexobj(D):
            Di = np.ascontiguousarray(np.imag(D), dtype=np.float64).reshape(-1)
        self._check(self.lib.hub_set_occupation_matrix(self.h, spin, _dptr(Dr),
                                                       None if Di is None else _dptr(Di)),
                    "hub_set_occupation_matrix")

    # ------------------------------------------------------------------ hot path
    def apply_H(self, spin: int, X, Y):
        ncol, ld = self._blk(X, "apply_H X")
        self._blk(Y, "apply_H Y")
        self._check(self.lib.hub_apply_H(self.h, spin, _tptr(X), _tptr(Y), ncol, ld), "hub_apply_H")

    def chefsi_filter(self, spin: int, X, degree: int, a: float, b: float, a_low: float, work=None):
        ncol, ld = self._blk(X, "chefsi_filter X")
        if work is not None:
            self._vec(work, self.dtype, "chefsi_filter work", ld * ncol)
        self._check(self.lib.hub_chefsi_filter(self.h, spin, _tptr(X), ncol, ld, degree, a, b, a_low,
                                               _tptr(work)), "hub_chefsi_filter")

    def rayleigh_ritz(self, spin: int, X, work=None) -> np.ndarray:
        ncol, ld = self._blk(X, "rayleigh_ritz X")
        if work is not None:
            self._vec(work, self.dtype, "rayleigh_ritz work", ld * ncol)
        eig = np.zeros(ncol)
        self._check(self.lib.hub_rayleigh_ritz(self.h, spin, _tptr(X), ncol, ld, _dptr(eig),
                                               _tptr(work)), "hub_rayleigh_ritz")
        return eig

    def gram(self, A, B, alpha: float, G):
        """G (device [ncol_a, ncol_b], float64; complex128 on a complex handle) =
        alpha * conj(A) B^T for row-stored blocks."""
        import torch
        na, ld = self._blk(A, "gram A")
        nb, ldb = self._blk(B, "gram B")
        self._vec(G, torch.complex128 if self.complex else torch.float64, "gram G", na * nb)
        if ld != ldb:
            raise ValueError("A and B need the same leading dimension")
        self._check(self.lib.hub_gram(self.h, _tptr(A), na, _tptr(B), nb, ld, float(alpha), _tptr(G)),
                    "hub_gram")

    def occupation(self, spin: int, X, f, kweight: float = 1.0):
        ncol, ld = self._blk(X, "occupation X")
        f = np.ascontiguousarray(f, dtype=np.float64)
        Dr = np.zeros((max(self.nhub, 1), 5, 5))
        Di = np.zeros_like(Dr)
        eu = C.c_double()
        self._check(self.lib.hub_occupation(self.h, spin, _tptr(X), ncol, ld, _dptr(f), kweight,
                                            _dptr(Dr), _dptr(Di), C.byref(eu)), "hub_occupation")
        return Dr[:self.nhub], Di[:self.nhub], eu.value

    def hubbard_forces(self, spin: int, X, f, kweight: float = 1.0, work=None) -> np.ndarray:
        """Hubbard forces (natoms, 3) of one (spin, k) block with the D last set for `spin`."""
        ncol, ld = self._blk(X, "hubbard_forces X")
        if work is not None:
            self._vec(work, self.dtype, "hubbard_forces work", ld * ncol)
        f = np.ascontiguousarray(f, dtype=np.float64)
        F = np.zeros((max(self.natoms, 1), 3))
        self._check(self.lib.hub_hubbard_forces(self.h, spin, _tptr(X), ncol, ld, _dptr(f), kweight,
                                                _dptr(F), _tptr(work)), "hub_hubbard_forces")
        return F[:self.natoms]

    def hubbard_stress(self, spin: int, X, f, kweight: float = 1.0, work=None) -> np.ndarray:
        """Hubbard stress (3, 3), Ha/bohr^3, of one (spin, k) block with the D last set for `spin`."""
        ncol, ld = self._blk(X, "hubbard_stress X")
        if work is not None:
            self._vec(work, self.dtype, "hubbard_stress work", ld * ncol)
        f = np.ascontiguousarray(f, dtype=np.float64)
        sig = np.zeros(9)
        self._check(self.lib.hub_hubbard_stress(self.h, spin, _tptr(X), ncol, ld, _dptr(f), kweight,
                                                _dptr(sig), _tptr(work)), "hub_hubbard_stress")
        return sig.reshape(3, 3)

    def lanczos_bound(self, spin: int, steps: int, v0):
        self._vec(v0, self.dtype, "lanczos_bound v0")
        lo, up = C.c_double(), C.c_double()
        self._check(self.lib.hub_lanczos_bound(self.h, spin, steps, _tptr(v0), C.byref(lo), C.byref(up)),
                    "hub_lanczos_bound")
        return lo.value, up.value

    def autotune(self, spin: int, X) -> int:
        ncol, ld = self._blk(X, "autotune X")
        v = C.c_int()
        self._check(self.lib.hub_autotune(self.h, spin, _tptr(X), ncol, ld, C.byref(v)), "hub_autotune")
        return v.value

    def set_tuning(self, stencil_variant: int = -1, gemm_split: int = -1, gather_form: int = -1):
        self._check(self.lib.hub_set_tuning(self.h, int(stencil_variant), int(gemm_split), int(gather_form)),
                    "hub_set_tuning")

    def get_tuning(self) -> dict:
        v, n, g, f = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.hub_get_tuning(self.h, C.byref(v), C.byref(n), C.byref(g), C.byref(f)),
                    "hub_get_tuning")
        return {"stencil_variant": v.value, "n_variants": n.value, "gemm_split": g.value, "gather_form": f.value}

    # ------------------------------------------------------------------ measurement
    def profile(self, enable: int):
        self._check(self.lib.hub_profile(self.h, int(enable)), "hub_profile")

    def profile_read(self) -> dict:
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            t, n = C.c_double(), C.c_longlong()
            self._check(self.lib.hub_profile_read(self.h, k, C.byref(t), C.byref(n)), "hub_profile_read")
            if n.value:
                out[name] = (t.value, n.value)
        return out

    def projector_stats(self) -> dict:
        fp, sp = C.c_longlong(), C.c_longlong()
        self._check(self.lib.hub_projector_stats(self.h, C.byref(fp), C.byref(sp)), "hub_projector_stats")
        return {"function_points": fp.value, "site_points": sp.value}

    def launch_count(self) -> int:
        n = C.c_longlong()
        self._check(self.lib.hub_launch_count(self.h, C.byref(n)), "hub_launch_count")
        return n.value

    # ------------------------------------------------------------------ SCF driver
    def scf_begin(self, params: scf_params, Xs, v0s, D0):
        for x in Xs:
            self._blk(x, "scf_begin X")
        for v in v0s:
            self._vec(v, self.dtype, "scf_begin v0")
        self._scf_keep = (list(Xs), list(v0s))
        xa = (C.c_void_p * len(Xs))(*[t.data_ptr() for t in Xs])
        va = (C.c_void_p * len(v0s))(*[t.data_ptr() for t in v0s])
        D0 = np.ascontiguousarray(D0, dtype=np.float64).reshape(-1)
        self._scf_D0 = D0
        self._check(self.lib.hub_scf_begin(self.h, C.byref(params), xa, va, _dptr(D0)), "hub_scf_begin")
        self._scf_params = params

    def scf_iterate(self) -> dict:
        r = scf_result()
        self._check(self.lib.hub_scf_iterate(self.h, C.byref(r)), "hub_scf_iterate")
        return {k: getattr(r, k) for k, _ in scf_result._fields_}

    def scf_run(self) -> dict:
        r = scf_result()
        rc = self.lib.hub_scf_run(self.h, C.byref(r))
        out = {k: getattr(r, k) for k, _ in scf_result._fields_}
        if rc not in (0, -6):
            self._check(rc, "hub_scf_run")
        out["status"] = rc
        return out

    def scf_get(self):
        p = self._scf_params
        eig = np.zeros(p.nspin * p.ncol)
        occ = np.zeros_like(eig)
        D = np.zeros(p.nspin * max(self.nhub, 1) * 25)
        self._check(self.lib.hub_scf_get(self.h, _dptr(eig), _dptr(occ), _dptr(D)), "hub_scf_get")
        return (eig.reshape(p.nspin, p.ncol), occ.reshape(p.nspin, p.ncol),
                D[:p.nspin * self.nhub * 25].reshape(p.nspin, self.nhub, 5, 5))


    def scf_forces(self, stress: bool = False):
        """Hubbard forces (natoms, 3) of the SCF's last iteration, and its stress (3, 3) when asked."""
        F = np.zeros((max(self.natoms, 1), 3))
        sig = np.zeros(9) if stress else None
        self._check(self.lib.hub_scf_forces(self.h, _dptr(F), None if sig is None else _dptr(sig)),
                    "hub_scf_forces")
        return (F[:self.natoms], sig.reshape(3, 3)) if stress else F[:self.natoms]

    def scf_set_density(self, rho):
        """Starting density of a density-mode SCF (before its first iteration)."""
        import torch
        self._vec(rho, torch.float64, "scf_set_density rho")
        self._check(self.lib.hub_scf_set_density(self.h, _tptr(rho)), "hub_scf_set_density")

    def num_projectors(self) -> int:
        n = C.c_int()
        self._check(self.lib.hub_num_projectors(self.h, C.byref(n)), "hub_num_projectors")
        return n.value

    def project(self, X) -> np.ndarray:
        """C[p, n] = dV <proj_p|x_n> for every projector row (complex on complex handles)."""
        ncol, ld = self._blk(X, "project X")
        npj = self.num_projectors()
        cw = 2 if self.complex else 1
        out = np.zeros(max(npj * ncol * cw, 1))
        self._check(self.lib.hub_project(self.h, _tptr(X), ncol, ld, _dptr(out)), "hub_project")
        out = out[:npj * ncol * cw]
        if cw == 2:
            return (out[0::2] + 1j * out[1::2]).reshape(npj, ncol)
        return out.reshape(npj, ncol)

    def expand(self, W, Y, alpha: float = 1.0):
        """Y[g, n] += alpha sum_p proj_p(g) W[p, n] (W host, [nproj, ncol])."""
        ncol, ld = self._blk(Y, "expand Y")
        W = np.asarray(W)
        if self.complex:
            Wf = np.empty(W.size * 2)
            Wf[0::2], Wf[1::2] = np.real(W).ravel(), np.imag(W).ravel()
        else:
            Wf = np.ascontiguousarray(np.real(W), dtype=np.float64).ravel()
        self._check(self.lib.hub_expand(self.h, _dptr(Wf), ncol, _tptr(Y), ld, float(alpha)), "hub_expand")

    def scf_density(self, rho):
        """Output density of the last density-SCF iteration (summed over spins) into rho."""
        import torch
        self._vec(rho, torch.float64, "scf_density rho")
        self._check(self.lib.hub_scf_density(self.h, _tptr(rho)), "hub_scf_density")

    # ------------------------------------------------------------------ density SCF steps
    def density(self, X, f, scale, rho):
        """rho += scale * sum_n f_n |x_n|^2 (rho: device double [Nd])."""
        import torch
        ncol, ld = self._blk(X, "density X")
        self._vec(rho, torch.float64, "density rho")
        f = np.ascontiguousarray(f, dtype=np.float64)
        self._check(self.lib.hub_density(self.h, _tptr(X), ncol, ld, _dptr(f), float(scale), _tptr(rho)),
                    "hub_density")

    def hartree(self, rho, V, tol=1e-10, max_iter=20000):
        """V (warm start in, solution out) and (CG iterations, E_H)."""
        import torch
        self._vec(rho, torch.float64, "hartree rho")
        self._vec(V, torch.float64, "hartree V")
        it, eh = C.c_int(), C.c_double()
        self._check(self.lib.hub_hartree(self.h, _tptr(rho), _tptr(V), tol, max_iter, C.byref(it),
                                         C.byref(eh)), "hub_hartree")
        return it.value, eh.value

    def lda_exchange(self, rhos, vxs) -> float:
        import torch
        for t in list(rhos) + list(vxs):
            self._vec(t, torch.float64, "lda_exchange")
        ex = C.c_double()
        two = len(rhos) == 2
        self._check(self.lib.hub_lda_exchange(self.h, len(rhos), _tptr(rhos[0]), _tptr(rhos[1]) if two else None,
                                              _tptr(vxs[0]), _tptr(vxs[1]) if two else None, C.byref(ex)),
                    "hub_lda_exchange")
        return ex.value

    def kerker(self, r, z, kappa, tol=1e-10, max_iter=20000) -> int:
        import torch
        self._vec(r, torch.float64, "kerker r")
        self._vec(z, torch.float64, "kerker z")
        it = C.c_int()
        self._check(self.lib.hub_kerker(self.h, _tptr(r), _tptr(z), kappa, tol, max_iter, C.byref(it)),
                    "hub_kerker")
        return it.value


def fermi_dirac(eig, weights, kT: float, n_elec: float, degeneracy: float):
    """(f, mu) for the states eig with k-point weights (hub_fermi_dirac)."""
    lib = load_library()
    e = np.ascontiguousarray(eig, dtype=np.float64).ravel()
    wv = np.ascontiguousarray(np.broadcast_to(np.asarray(weights, dtype=np.float64), e.shape)).ravel()
    f = np.zeros_like(e)
    mu = C.c_double()
    rc = lib.hub_fermi_dirac(e.size, _dptr(e), _dptr(wv), float(kT), float(n_elec), float(degeneracy),
                             _dptr(f), C.byref(mu))
    if rc:
        raise HubError(rc, "hub_fermi_dirac: bad arguments")
    return f, mu.value


def cutoff_radius(l: int, rs: float, tau: float) -> float:
    """Radius beyond which N r^l exp(-r^2/(2 rs^2)) stays below tau (hub_cutoff_radius)."""
    lib = load_library()
    rc = C.c_double()
    rc_ = lib.hub_cutoff_radius(int(l), float(rs), float(tau), C.byref(rc))
    if rc_:
        raise HubError(rc_, "hub_cutoff_radius: bad arguments")
    return rc.value


def extrapolate_occupations(D_hist, D_atomic, R_hist):
    """Starting D of the next MD step from up to three converged D sets (oldest first) and
    the positions of those steps plus the new one (hub_extrapolate_occupations).
    Returns (D, (alpha, beta))."""
    lib = load_library()
    Da = np.ascontiguousarray(D_atomic, dtype=np.float64)
    n = Da.size
    nh = len(D_hist)
    Dh = np.ascontiguousarray(np.stack([np.asarray(d, dtype=np.float64).reshape(-1) for d in D_hist])
                              if nh else np.zeros(1), dtype=np.float64)
    R = [np.asarray(r, dtype=np.float64).reshape(-1) for r in R_hist]
    natoms = R[0].size // 3 if R else 0
    Rh = np.ascontiguousarray(np.concatenate(R) if R else np.zeros(1), dtype=np.float64)
    coef = np.zeros(2)
    out = np.zeros(n)
    rc = lib.hub_extrapolate_occupations(n, nh, _dptr(Dh), _dptr(Da.reshape(-1)), natoms, _dptr(Rh),
                                         _dptr(coef), _dptr(out))
    if rc:
        raise HubError(rc, "hub_extrapolate_occupations: bad arguments")
    return out.reshape(Da.shape), (float(coef[0]), float(coef[1]))


def descriptors(pos, species, L, centers, out, nspecies=2, rc=6.0, nrad=16, eta=0.4, stream=None):
    """Per-atom local-environment descriptors into the device float tensor `out`."""
    import torch
    lib = load_library()
    st = stream if stream is not None else torch.cuda.current_stream()
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1)
    sp = np.ascontiguousarray(species, dtype=np.int32)
    Lv = np.ascontiguousarray(L, dtype=np.float64)
    ce = np.ascontiguousarray(centers, dtype=np.int32)
    rc_ = lib.hub_descriptors(len(sp), _dptr(pos), _iptr(sp), _dptr(Lv), len(ce), _iptr(ce), nspecies,
                              float(rc), nrad, float(eta), _tptr(out), C.c_void_p(st.cuda_stream))
    if rc_ != 0:
        raise HubError(rc_, "hub_descriptors")


class MLP:
    """Warm-start model handle (hub_mlp_*)."""

    def __init__(self, n_in, n_hidden=256, n_layers=3, n_out=30, fp16=True, seed=0, stream=None):
        import torch
        self.lib = load_library()
        st = stream if stream is not None else torch.cuda.current_stream()
        m = C.c_void_p()
        rc = self.lib.hub_mlp_create(C.byref(m), n_in, n_hidden, n_layers, n_out, int(fp16), seed,
                                     C.c_void_p(st.cuda_stream))
        if rc != 0:
            raise HubError(rc, "hub_mlp_create")
        self.m = m
        n = C.c_longlong()
        self.lib.hub_mlp_num_params(self.m, C.byref(n))
        self.nparams = n.value
        self.sizes = [n_in] + [n_hidden] * n_layers + [n_out]

    def _check(self, rc, what):
        if rc != 0:
            msg = self.lib.hub_mlp_last_error(self.m)
            raise HubError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "m", None):
            self.lib.hub_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(self.lib.hub_mlp_set_params(self.m, a.ctypes.data_as(C.POINTER(C.c_float))), "set_params")

    def get_params(self):
        a = np.zeros(self.nparams, dtype=np.float32)
        self._check(self.lib.hub_mlp_get_params(self.m, a.ctypes.data_as(C.POINTER(C.c_float))), "get_params")
        return a

    def set_normalization(self, mu_in, sd_in, mu_out, sd_out):
        arrs = [np.ascontiguousarray(v, dtype=np.float32) for v in (mu_in, sd_in, mu_out, sd_out)]
        self._check(self.lib.hub_mlp_set_normalization(self.m, *[v.ctypes.data_as(C.POINTER(C.c_float)) for v in arrs]),
                    "set_normalization")

    def fit_normalization(self, X, T):
        self._check(self.lib.hub_mlp_fit_normalization(self.m, _tptr(X), _tptr(T), X.shape[0]), "fit_normalization")

    def forward(self, X, Y):
        self._check(self.lib.hub_mlp_forward(self.m, _tptr(X), X.shape[0], _tptr(Y)), "forward")

    def loss_grad(self, X, T):
        loss = C.c_float()
        g = np.zeros(self.nparams, dtype=np.float32)
        self._check(self.lib.hub_mlp_loss_grad(self.m, _tptr(X), _tptr(T), X.shape[0], C.byref(loss),
                                               g.ctypes.data_as(C.POINTER(C.c_float))), "loss_grad")
        return loss.value, g

    def train_step(self, X, T, lr):
        loss = C.c_float()
        self._check(self.lib.hub_mlp_train_step(self.m, _tptr(X), _tptr(T), X.shape[0], float(lr), C.byref(loss)),
                    "train_step")
        return loss.value


def alu_peaks(stream=None) -> dict:
    """Measured FP64 and FP32 FMA throughput of the current device (GFLOP/s)."""
    import torch
    lib = load_library()
    st = stream if stream is not None else torch.cuda.current_stream()
    f64, f32 = C.c_double(), C.c_double()
    rc = lib.hub_alu_peaks(C.byref(f64), C.byref(f32), C.c_void_p(st.cuda_stream))
    if rc != 0:
        raise HubError(rc, "hub_alu_peaks")
    return {"fp64_gflops": f64.value, "fp32_gflops": f32.value}
