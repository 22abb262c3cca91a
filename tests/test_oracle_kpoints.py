"""Pins for the oracle's SCF with Brillouin-zone sampling: one Gamma point reproduces the
Gamma-point SCF, a k-set closed under k -> -k keeps D real, and the CheFSI SCF reaches the
fixed point of the same SCF driven by a dense eigensolver (real and complex D)."""
import numpy as np
import pytest

from oracle import hubbard as o
import workloads as w

K = (0.3, -0.2, 0.25)


def _case(nspin=1):
    return w.small_test_system(n=(8, 8, 10), ncol=8, natoms=2, seed=11, nspin=nspin)


def _run(wl, kpts, kweights, solver, conj_pairs=False, **kw):
    """With conj_pairs, the k-point -k starts from the complex conjugate of the +k start (the
    exact symmetry H_-k = conj(H_k) then holds at every iteration, not only at the fixed point)."""
    nk = len(kpts)
    X0s = [[wl.orbitals(spin=s, complex_=any(kpts[k])).T for k in range(nk)] for s in range(wl.nspin)]
    v0s = [[wl.lanczos_start(spin=s, complex_=any(kpts[k])) for k in range(nk)] for s in range(wl.nspin)]
    if conj_pairs:
        for s in range(wl.nspin):
            X0s[s][1], v0s[s][1] = np.conj(X0s[s][0]), np.conj(v0s[s][0])
    return o.scf_model_a_kpoints(wl.n, wl.L, kpts, kweights, wl.veff, wl.atoms, wl.D0, X0s,
                                 n_elec=6.0, kT=0.01, degree=12, lanczos_v0s=v0s, eig_solver=solver,
                                 max_iter=80, tol_e_atom=1e-8, tol_D=1e-6, **kw)


def test_gamma_only_is_the_gamma_point_scf():
    wl = _case()
    r = _run(wl, [(0.0, 0.0, 0.0)], [1.0], "chefsi")
    ref = o.scf_model_a((wl.n, wl.L, (0, 0, 0), 6), wl.veff, wl.atoms, wl.D0, [wl.orbitals().T],
                        n_elec=6.0, kT=0.01, degree=12, lanczos_v0s=[wl.lanczos_start()], max_iter=80,
                        tol_e_atom=1e-8, tol_D=1e-6)
    assert r["converged"] and ref["converged"]
    assert r["iterations"] == ref["iterations"]
    assert abs(r["E"] - ref["E"]) < 1e-12 * abs(ref["E"])


def test_time_reversal_pair_keeps_D_real_and_matches_the_dense_scf():
    wl = _case()
    kpts = [K, tuple(-np.asarray(K))]
    r = _run(wl, kpts, [0.5, 0.5], "chefsi", conj_pairs=True)
    d = _run(wl, kpts, [0.5, 0.5], "dense")
    assert r["converged"] and d["converged"]
    assert np.max(np.abs(r["D"].imag)) < 1e-10
    assert abs(r["E"] - d["E"]) / len(wl.atoms) < 1e-7
    np.testing.assert_allclose(r["D"], d["D"], atol=1e-5)
    # the -k eigenvalues are those of +k (conjugate Hamiltonians)
    np.testing.assert_allclose(r["eig"][0][0], r["eig"][0][1], atol=1e-8)


def test_single_bloch_point_with_complex_D_matches_the_dense_scf():
    wl = _case()
    r = _run(wl, [K], [1.0], "chefsi")
    d = _run(wl, [K], [1.0], "dense")
    assert r["converged"] and d["converged"]
    assert np.max(np.abs(r["D"].imag)) > 1e-6          # complex Hermitian D
    np.testing.assert_allclose(r["D"], np.conj(np.swapaxes(r["D"], -1, -2)), atol=1e-12)
    assert abs(r["E"] - d["E"]) / len(wl.atoms) < 1e-7


def test_gamma_with_an_unpaired_bloch_point_is_rejected():
    wl = _case()
    with pytest.raises(ValueError):
        _run(wl, [(0.0, 0.0, 0.0), K], [0.5, 0.5], "chefsi", first_passes=1)


@pytest.fixture(scope="module")
def lib():
    from paper_2507_23612_gb300 import build as b
    b.build()
    from paper_2507_23612_gb300 import binding
    return binding.load_library()


@pytest.mark.parametrize("kT", [0.01, 0.0])
def test_library_fermi_level_matches_the_oracle(lib, kT):
    from paper_2507_23612_gb300.binding import fermi_dirac
    rng = np.random.default_rng(3)
    eigs = [np.sort(rng.uniform(-1.0, 1.0, 9)) for _ in range(3)]
    wts = [0.25, 0.25, 0.5]
    f_ref, mu_ref = o.fermi_dirac(eigs, wts, kT, 7.0, 2.0)
    f, mu = fermi_dirac(np.concatenate(eigs), np.repeat(wts, 9), kT, 7.0, 2.0)
    np.testing.assert_allclose(f, np.concatenate(f_ref), atol=1e-12)
    if kT > 0:
        assert abs(mu - mu_ref) < 1e-12
        assert abs(2.0 * np.sum(np.repeat(wts, 9) * f) - 7.0) < 1e-10


def test_library_fermi_level_rejects_too_many_electrons(lib):
    from paper_2507_23612_gb300.binding import HubError, fermi_dirac
    with pytest.raises(HubError):
        fermi_dirac([0.0, 1.0], [1.0, 1.0], 0.01, 5.0, 2.0)
