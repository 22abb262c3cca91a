"""Pins for the self-consistent density SCF oracle (model B): the FD Poisson solve against
the real-space stencil and the continuum Coulomb law, the Dirac exchange constant, the
exchange potential as the derivative of the exchange energy, the spin-scaling relation,
the Kerker operator against the stencil, Pulay on a linear fixed point, and the SCF against
a dense-eigensolver SCF with the band-structure energy equal to the directly evaluated
functional at every iteration."""
from math import pi

import numpy as np
import pytest

import workloads as w
from oracle import hubbard as hb
from oracle import density_scf as ds


def _grid(n=(12, 10, 14), L=(3.6, 3.0, 4.2)):
    return hb.Grid(n, L)


def test_laplacian_symbol_matches_the_stencil_on_plane_waves():
    g = _grid()
    x = g.coords()
    sig = ds.laplacian_symbol(g)
    for j in [(0, 0, 1), (1, 2, 0), (5, 4, 6), (-3, 1, 2)]:
        q = 2 * pi * np.array(j) / g.L
        e = np.exp(1j * x @ q)[:, None]
        Le = hb.laplacian(e, g)[:, 0]
        k = tuple(np.mod([j[2], j[1], j[0]], [g.n[2], g.n[1], g.n[0]]))
        np.testing.assert_allclose(Le, sig[k] * e[:, 0], atol=1e-10 * abs(sig[k]))


def test_hartree_solves_the_fd_poisson_problem():
    g = _grid()
    rng = np.random.default_rng(1)
    rho = rng.uniform(0.0, 2.0, g.Nd)
    v = ds.hartree_potential(rho, g)
    lhs = hb.laplacian(v[:, None], g)[:, 0]
    np.testing.assert_allclose(lhs, -4 * pi * (rho - rho.mean()), atol=1e-10)
    assert abs(v.mean()) < 1e-12
    assert ds.hartree_energy(rho, g) > 0


def test_hartree_plane_wave_is_the_coulomb_law():
    # rho = rho0 + A cos(q x): V_H = 4 pi A cos(q x) / q^2 and E_H = pi A^2 Omega / q^2 in the
    # continuum; the 12th-order FD symbol at q h = 2 pi / 32 differs by ~1e-13 relative
    g = hb.Grid((32, 8, 8), (9.6, 2.4, 2.4))
    x = g.coords()[:, 0]
    q = 2 * pi / g.L[0]
    A = 0.3
    rho = 1.0 + A * np.cos(q * x)
    v = ds.hartree_potential(rho, g)
    np.testing.assert_allclose(v, 4 * pi * A * np.cos(q * x) / q ** 2, rtol=0, atol=1e-9)
    omega = g.Nd * g.dV
    assert abs(ds.hartree_energy(rho, g) - pi * A * A * omega / q ** 2) < 1e-9 * pi * A * A * omega / q ** 2


def test_dirac_exchange_constant_and_uniform_gas():
    # textbook value of (3/4)(3/pi)^(1/3)
    assert abs(ds.C_X - 0.7385587663820224) < 1e-15
    g = _grid()
    rho = np.full(g.Nd, 0.37)
    v, E = ds.lda_exchange([rho], g)
    omega = g.Nd * g.dV
    assert abs(E - (-0.7385587663820224 * 0.37 ** (4 / 3) * omega)) < 1e-13
    np.testing.assert_allclose(v[0], -(3 / pi) ** (1 / 3) * 0.37 ** (1 / 3), rtol=1e-14)


@pytest.mark.parametrize("nspin", [1, 2])
def test_exchange_potential_is_the_derivative_of_the_energy(nspin):
    g = _grid((6, 5, 7), (1.8, 1.5, 2.1))
    rng = np.random.default_rng(2)
    rhos = [rng.uniform(0.1, 1.0, g.Nd) for _ in range(nspin)]
    v, _ = ds.lda_exchange(rhos, g)
    eps = 1e-6
    for s in range(nspin):
        for idx in (0, 17, g.Nd - 1):
            up = [r.copy() for r in rhos]
            dn = [r.copy() for r in rhos]
            up[s][idx] += eps
            dn[s][idx] -= eps
            d = (ds.lda_exchange(up, g)[1] - ds.lda_exchange(dn, g)[1]) / (2 * eps * g.dV)
            assert abs(d - v[s][idx]) < 1e-7 * abs(v[s][idx])


def test_spin_scaling_relation():
    g = _grid((6, 5, 7), (1.8, 1.5, 2.1))
    rng = np.random.default_rng(3)
    a, b = rng.uniform(0.0, 1.0, g.Nd), rng.uniform(0.0, 1.0, g.Nd)
    E_ab = ds.lda_exchange([a, b], g)[1]
    assert abs(E_ab - 0.5 * (ds.lda_exchange([2 * a], g)[1] + ds.lda_exchange([2 * b], g)[1])) < 1e-12 * abs(E_ab)
    # an unpolarized density split evenly is the one-channel functional
    rho = a + b
    v2, E2 = ds.lda_exchange([rho / 2, rho / 2], g)
    v1, E1 = ds.lda_exchange([rho], g)
    assert abs(E2 - E1) < 1e-12 * abs(E1)
    np.testing.assert_allclose(v2[0], v1[0], rtol=1e-13)


def test_kerker_operator():
    g = _grid()
    rng = np.random.default_rng(4)
    r = rng.standard_normal(g.Nd)
    kappa = 0.7
    P = ds.kerker(r, g, kappa)
    # (-L + kappa^2) P r = -L r, with L the real-space stencil
    lhs = -hb.laplacian(P[:, None], g)[:, 0] + kappa ** 2 * P
    np.testing.assert_allclose(lhs, -hb.laplacian(r[:, None], g)[:, 0], atol=1e-9)
    assert np.max(np.abs(ds.kerker(np.ones(g.Nd), g, kappa))) < 1e-14     # constants removed
    np.testing.assert_allclose(ds.kerker(r, g, 0.0), r - r.mean(), atol=1e-12)


def test_pulay_reaches_a_linear_fixed_point():
    g = hb.Grid((4, 4, 4), (2.0, 2.0, 2.0))
    rng = np.random.default_rng(5)
    n = g.Nd + 10
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(rng.uniform(-0.6, 0.6, n)) @ Q.T
    b = rng.standard_normal(n)
    b[:g.Nd] -= b[:g.Nd].mean()
    fixed = np.linalg.solve(np.eye(n) - A, b)
    mixer = ds.PreconditionedPulay(g, 0, hist=20, beta=0.5)       # identity preconditioner
    x = np.zeros(n)
    for _ in range(40):
        x = mixer.mix(x, A @ x + b)
    assert np.max(np.abs(x - fixed)) < 1e-8
    # history 1 is preconditioned linear mixing
    m1 = ds.PreconditionedPulay(g, g.Nd, hist=1, beta=0.3, kappa=0.5)
    x0 = rng.standard_normal(n)
    x1 = A @ x0 + b
    step = m1.mix(x0, x1)
    expect = x0 + 0.3 * np.concatenate([ds.kerker((x1 - x0)[:g.Nd], g, 0.5), (x1 - x0)[g.Nd:]])
    np.testing.assert_allclose(step, expect, atol=1e-13)


def _scf(solver, nspin=1, **kw):
    wl = w.small_test_system(n=(10, 10, 12), ncol=8, natoms=2, seed=11, nspin=nspin)
    X0s = [wl.orbitals(spin=s).T for s in range(nspin)]
    v0s = [wl.lanczos_start(spin=s) for s in range(nspin)]
    return wl, ds.scf_model_b((wl.n, wl.L, (0, 0, 0), 6), wl.veff, wl.atoms, wl.D0, X0s,
                              n_elec=6.0, kT=0.01, degree=12, lanczos_v0s=v0s, eig_solver=solver,
                              max_iter=60, **kw)


def test_model_b_scf_matches_the_dense_eigensolver_scf():
    wl, r = _scf("chefsi")
    _, d = _scf("dense")
    assert r["converged"] and d["converged"]
    print({"iterations": (r["iterations"], d["iterations"]), "E": (r["E"], d["E"])})
    assert abs(r["E"] - d["E"]) / len(wl.atoms) < 1e-7
    assert wl.dV * np.sum(np.abs(r["rho"][0] - d["rho"][0])) < 1e-3
    assert np.max(np.abs(r["D"] - d["D"])) < 1e-4
    for res in (r, d):
        # the band-structure form with double counting is the functional itself
        assert max(abs(a - b) for a, b in zip(res["hist_E"], res["hist_direct"])) < 1e-10
        assert abs(wl.dV * np.sum(res["rho"][0]) - 6.0) < 1e-10
        assert res["hist_drho"][-1] < 1e-4
        assert res["E_H"] > 0 and res["E_x"] < 0


def test_model_b_scf_spin_polarized():
    wl, r = _scf("chefsi", nspin=2)
    assert r["converged"]
    assert max(abs(a - b) for a, b in zip(r["hist_E"], r["hist_direct"])) < 1e-10
    assert abs(wl.dV * (np.sum(r["rho"][0]) + np.sum(r["rho"][1])) - 6.0) < 1e-10


def _basis_case():
    g = hb.Grid((20, 18, 22), (6.0, 5.4, 6.6))
    atoms = [w.Atom("Ti", np.array([1.0, 2.0, 3.0])), w.Atom("O", np.array([4.5, 1.2, 0.4]))]
    return g, ds.density_basis_atoms(atoms)


def test_density_in_the_basis_is_recovered_exactly():
    g, basis = _basis_case()
    c = np.array([[0.7, -0.2, 1.3], [0.1, 0.9, 0.4]])
    rho = ds.expand_density(g, basis, c)
    np.testing.assert_allclose(ds.fit_density_coefficients(g, basis, rho), c, atol=1e-9)


def test_fit_is_the_orthogonal_projection():
    g, basis = _basis_case()
    rng = np.random.default_rng(8)
    rho = rng.uniform(0.0, 1.0, g.Nd)
    c = ds.fit_density_coefficients(g, basis, rho)
    B = ds.density_basis_matrix(g, basis)
    resid = rho - B @ c.ravel()
    # the residual is orthogonal to every basis function, so any other coefficients fit worse
    assert np.max(np.abs(g.dV * (B.T @ resid))) < 1e-10 * np.max(np.abs(g.dV * (B.T @ rho)))
    worse = rho - B @ (c.ravel() + 1e-3 * rng.standard_normal(c.size))
    assert np.sum(worse ** 2) > np.sum(resid ** 2)


def test_expanded_density_carries_the_electron_count():
    g, basis = _basis_case()
    rho = ds.expand_density(g, basis, np.array([[0.7, 0.2, 1.3], [0.1, 0.9, 0.4]]), n_elec=12.0)
    assert abs(g.dV * np.sum(rho) - 12.0) < 1e-12


def test_density_basis_driver_on_the_cpu():
    # the warm start's DensityBasis with the library handle replaced by the oracle's basis
    # matrix: its Gram matrix (expand the unit vectors, project them), fit and scaled
    # expansion reproduce the oracle's fit and expansion
    torch = pytest.importorskip("torch")
    from paper_2507_23612_gb300.warmstart import DensityBasis

    wl = w.rutile_snapshot((1, 1, 1), 0.1, seed=2, h_target=0.5, nspin=1)
    g = hb.Grid(wl.n, wl.L)

    class BasisHandle:
        def __init__(self, atoms_):
            self.B = ds.density_basis_matrix(g, atoms_)

        def num_projectors(self):
            return self.B.shape[1]

        def project(self, X):
            return g.dV * (self.B.T @ X.cpu().numpy().T)

        def expand(self, W, Y, alpha=1.0):
            Y += torch.tensor((alpha * (self.B @ np.asarray(W))).T, dtype=Y.dtype)

        def close(self):
            pass

    basis = DensityBasis(wl, device=torch.device("cpu"), hub_factory=BasisHandle)
    rng = np.random.default_rng(6)
    rho = rng.uniform(0.0, 1.0, wl.Nd)
    c = basis.fit(torch.tensor(rho))
    c_ref = ds.fit_density_coefficients(g, ds.density_basis_atoms(wl.atoms), rho)
    np.testing.assert_allclose(c, c_ref, rtol=1e-9, atol=1e-12)
    rho0 = basis.expand(c, wl.n_elec).numpy()
    ref = ds.expand_density(g, ds.density_basis_atoms(wl.atoms), c_ref, n_elec=wl.n_elec)
    np.testing.assert_allclose(rho0, ref, rtol=1e-9, atol=1e-12)
