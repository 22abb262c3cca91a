"""The k-point SCF driver's host orchestration (Fermi level over k-weighted states, the
energy sums, Pulay mixing of the real and imaginary parts of D, bounds bookkeeping) run on
the CPU: the library handles are replaced by stand-ins built from the oracle's Hamiltonian,
filter, Rayleigh-Ritz and occupation matrices, and the driver must reproduce the oracle's
k-point SCF."""
import numpy as np
import pytest

from oracle import hubbard as o
import workloads as w


class OracleHandle:
    """The Hub methods the driver calls, on numpy blocks [ncol, Nd], by the oracle."""

    def __init__(self, wl, k):
        self.ham = o.Hamiltonian(o.Grid(wl.n, wl.L, k, wl.fd_half_order), wl.veff, wl.atoms)
        self.D = {}

    def set_occupation_matrix(self, spin, D, D_im=None):
        self.D[spin] = np.asarray(D) + (0 if D_im is None else 1j * np.asarray(D_im))

    def _h(self, spin):
        D = self.D[spin]
        self.ham.set_occupation(D if self.ham.grid.is_complex else np.real(D))
        return self.ham

    def lanczos_bound(self, spin, steps, v0):
        return o.lanczos_bounds(self._h(spin), v0, steps)

    def chefsi_filter(self, spin, X, degree, a, b, a_low):
        X[:] = o.chebyshev_filter(self._h(spin), X.T, degree, a, b, a_low).T

    def rayleigh_ritz(self, spin, X):
        lam, Xn = o.rayleigh_ritz(self._h(spin), X.T)
        X[:] = Xn.T
        return lam

    def occupation(self, spin, X, f, kweight=1.0):
        D = o.occupation_matrices(self._h(spin), X.T, f, kweight)
        return np.real(D), np.imag(D), None

    def close(self):
        pass


@pytest.fixture(scope="module")
def built():
    from paper_2507_23612_gb300 import build as b
    b.build()


K = (0.3, -0.2, 0.25)


@pytest.mark.parametrize("kpts,kw", [([(0.0, 0.0, 0.0)], [1.0]),
                                     ([K, tuple(-np.asarray(K))], [0.5, 0.5]),
                                     ([K], [1.0])], ids=["gamma", "pair", "bloch"])
def test_driver_reproduces_the_oracle_kpoint_scf(built, kpts, kw):
    from paper_2507_23612_gb300.kpoint_scf import KpointSCF
    wl = w.small_test_system(n=(8, 8, 10), ncol=8, natoms=2, seed=11)
    nk = len(kpts)
    X0 = [[wl.orbitals(complex_=any(kpts[k])) for k in range(nk)]]
    v0 = [[wl.lanczos_start(complex_=any(kpts[k])) for k in range(nk)]]
    if nk == 2:
        X0[0][1], v0[0][1] = np.conj(X0[0][0]), np.conj(v0[0][0])
    kwargs = dict(n_elec=6.0, kT=0.01, degree=12, max_iter=80, tol_e_atom=1e-9, tol_D=1e-7)
    ref = o.scf_model_a_kpoints(wl.n, wl.L, kpts, kw, wl.veff, wl.atoms, wl.D0,
                                [[x.T for x in X0[0]]], lanczos_v0s=v0, **kwargs)
    scf = KpointSCF(wl, kpts, kw, hub_factory=lambda k: OracleHandle(wl, k))
    res = scf.run([[x.copy() for x in X0[0]]], v0, wl.D0, **kwargs)
    assert ref["converged"] and res["converged"]
    assert abs(res["E"] - ref["E"]) < 1e-9 * abs(ref["E"])
    np.testing.assert_allclose(res["D"], ref["D"], atol=1e-7)
    assert abs(res["mu"] - ref["mu"]) < 1e-7


def test_gamma_with_an_unpaired_bloch_point_is_rejected(built):
    from paper_2507_23612_gb300.kpoint_scf import KpointSCF
    wl = w.small_test_system(n=(8, 8, 10), ncol=8, natoms=2, seed=11)
    scf = KpointSCF(wl, [(0.0, 0.0, 0.0), K], [0.5, 0.5], hub_factory=lambda k: OracleHandle(wl, k))
    X0 = [[wl.orbitals(), wl.orbitals(complex_=True)]]
    v0 = [[wl.lanczos_start(), wl.lanczos_start(complex_=True)]]
    with pytest.raises(ValueError):
        scf.run(X0, v0, wl.D0, n_elec=6.0, kT=0.01, degree=12, max_iter=3, first_passes=1)


def test_driver_spin_polarized_pair(built):
    from paper_2507_23612_gb300.kpoint_scf import KpointSCF
    wl = w.small_test_system(n=(8, 8, 10), ncol=8, natoms=2, seed=11, nspin=2)
    kpts, kw = [K, tuple(-np.asarray(K))], [0.5, 0.5]
    X0 = [[wl.orbitals(spin=s, complex_=True) for _ in range(2)] for s in range(2)]
    v0 = [[wl.lanczos_start(spin=s, complex_=True) for _ in range(2)] for s in range(2)]
    for s in range(2):
        X0[s][1], v0[s][1] = np.conj(X0[s][0]), np.conj(v0[s][0])
    kwargs = dict(n_elec=6.0, kT=0.01, degree=12, max_iter=80, tol_e_atom=1e-9, tol_D=1e-7)
    ref = o.scf_model_a_kpoints(wl.n, wl.L, kpts, kw, wl.veff, wl.atoms, wl.D0,
                                [[x.T for x in X0[s]] for s in range(2)], lanczos_v0s=v0, **kwargs)
    scf = KpointSCF(wl, kpts, kw, hub_factory=lambda k: OracleHandle(wl, k))
    res = scf.run([[x.copy() for x in X0[s]] for s in range(2)], v0, wl.D0, **kwargs)
    assert ref["converged"] and res["converged"]
    assert abs(res["E"] - ref["E"]) < 1e-9 * abs(ref["E"])
    np.testing.assert_allclose(res["D"], ref["D"], atol=1e-7)
