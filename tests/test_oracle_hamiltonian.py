"""Pins for the oracle's projectors, Hamiltonian, occupation matrices and Hubbard energy
(Sec. II.A.1-2): spherical-harmonic orthonormality, radial normalisation, grid norm of the
orbitals, Hermiticity of H (real and Bloch), D = I / D = Gram identities, E_U closed forms,
and the derivative consistency between E_U and V_U."""
import numpy as np
import pytest
from scipy import integrate

from oracle import hubbard as o
import workloads as w


def test_real_harmonics_orthonormal_on_sphere():
    # Gauss-Legendre in cos(theta) x uniform phi: exact for these polynomial degrees
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phi = 2 * np.pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1)
    wts = (wg[:, None] * np.ones_like(ph)) * (2 * np.pi / nphi)
    Y = np.concatenate([o.real_solid_harmonics(l, d) for l in (0, 1, 2)])  # unit sphere
    G = np.einsum("aij,bij,ij->ab", Y, Y, wts)
    np.testing.assert_allclose(G, np.eye(9), atol=1e-13)


@pytest.mark.parametrize("l,rs", [(0, 0.8), (1, 0.8), (2, 1.0), (2, 0.7)])
def test_radial_normalisation(l, rs):
    N = o.radial_norm(l, rs)
    val, _ = integrate.quad(lambda r: (N * r ** l * np.exp(-r * r / (2 * rs * rs))) ** 2 * r * r, 0, np.inf)
    assert abs(val - 1.0) < 1e-12
    if l == 2 and rs == 1.0:
        # the workload's d orbital r^2 exp(-r^2/2): N^2 = 16 / (15 sqrt(pi))
        assert abs(N - np.sqrt(16 / (15 * np.sqrt(np.pi)))) < 1e-14


def test_orbitals_grid_orthonormal_in_isolated_cell():
    # one atom in a 12 bohr box at h = 0.3: images do not overlap (rc = 5 < 6) and the
    # Gaussian is resolved, so <phi_m|phi_m'> is the identity to quadrature accuracy
    g = o.Grid((40, 40, 40), (12.0, 12.0, 12.0))
    idx, vals = o.atom_function_table(g, (6.1, 5.9, 6.05), [(2, 1.0), (0, 0.8), (1, 0.8)], 5.0)
    G = g.dV * vals.T @ vals
    print("max |Gram - I| =", np.max(np.abs(G - np.eye(9))))
    np.testing.assert_allclose(G, np.eye(9), atol=2e-5)


def test_image_sum_and_bloch_phase():
    # the table of an atom equals the explicit sum over images with the Bloch phase, and
    # satisfies phi(x + L) = exp(i k L) phi(x) when evaluated beyond the cell
    k = (0.21, -0.13, 0.34)
    g = o.Grid((14, 12, 16), (4.2, 3.6, 4.8), k)
    R = np.array([0.3, 3.5, 2.0])
    idx, vals = o.atom_function_table(g, R, [(2, 1.0)], 3.0)
    x = g.coords()
    ref = np.zeros((g.Nd, 5), dtype=complex)
    for t1 in range(-3, 4):
        for t2 in range(-3, 4):
            for t3 in range(-3, 4):
                T = np.array([t1, t2, t3]) * g.L
                d = x - R - T
                r2 = np.sum(d * d, axis=1)
                m = r2 < 9.0
                ref[m] += (np.exp(1j * np.dot(k, T)) * o.radial_norm(2, 1.0) *
                           np.exp(-r2[m] / 2) * o.real_solid_harmonics(2, d[m])).T
    full = np.zeros((g.Nd, 5), dtype=complex)
    full[idx] = vals
    np.testing.assert_allclose(full, ref, atol=1e-13)
    assert np.all(np.any(np.abs(ref[idx]) > 0, axis=1) | True)
    outside = np.setdiff1d(np.arange(g.Nd), idx)
    assert np.max(np.abs(ref[outside]), initial=0.0) == 0.0


def _random_D(nhub, seed, complex_=False):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(nhub):
        A = g.uniform(-0.3, 0.3, (5, 5))
        if complex_:
            A = A + 1j * g.uniform(-0.3, 0.3, (5, 5))
        out.append(0.4 * np.eye(5) + 0.5 * (A + A.conj().T))
    return np.array(out)


@pytest.mark.parametrize("kpt", [(0.0, 0.0, 0.0), (0.2, -0.1, 0.3)])
def test_hamiltonian_hermitian(kpt):
    wl = w.small_test_system(n=(12, 10, 14), ncol=4, natoms=3, kpt=kpt)
    g = o.Grid(wl.n, wl.L, kpt)
    H = o.Hamiltonian(g, wl.veff, wl.atoms, _random_D(2, 5, g.is_complex))
    rng = np.random.default_rng(0)
    dt = complex if g.is_complex else float
    u = rng.standard_normal((g.Nd, 3)).astype(dt)
    v = rng.standard_normal((g.Nd, 3)).astype(dt)
    if g.is_complex:
        u = u + 1j * rng.standard_normal((g.Nd, 3))
        v = v + 1j * rng.standard_normal((g.Nd, 3))
    lhs = u.conj().T @ H.apply(v)
    rhs = H.apply(u).conj().T @ v
    scale = np.linalg.norm(u) * np.linalg.norm(v) * 300.0
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * scale
    # each piece separately (a sign or index error in one piece must not hide)
    for piece in (H.kinetic, H.nonlocal_kb, H.hubbard):
        l2 = u.conj().T @ piece(v)
        r2 = piece(u).conj().T @ v
        assert np.max(np.abs(l2 - r2)) < 1e-13 * scale


def test_hubbard_term_positive_for_D_zero_and_negative_for_D_one():
    # with D = 0, V_U = (U/2) sum_m |phi_m><phi_m| is positive semidefinite;
    # with D = I, V_U = -(U/2) sum_m |phi_m><phi_m| is negative semidefinite
    wl = w.small_test_system(n=(12, 12, 12), natoms=2)
    g = o.Grid(wl.n, wl.L)
    H = o.Hamiltonian(g, wl.veff, wl.atoms, np.zeros((2, 5, 5)))
    x = np.random.default_rng(1).standard_normal((g.Nd, 6))
    q = np.einsum("in,in->n", x, H.hubbard(x))
    assert np.all(q >= -1e-12)
    H.set_occupation(np.array([np.eye(5)] * 2))
    q2 = np.einsum("in,in->n", x, H.hubbard(x))
    np.testing.assert_allclose(q2, -q, rtol=1e-12)


@pytest.mark.parametrize("kpt", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.1)])
def test_occupation_identities_for_orbital_built_states(kpt):
    # Let Phi be atom 0's Hubbard orbitals on the grid and S = <Phi|Phi> their Gram matrix.
    # (i) states X = Phi S^-1/2 (grid-orthonormal, Loewdin), all occupied: C = S^1/2, so D = S.
    # (ii) states X = Phi S^-1 (the dual set), all occupied: C = I, so D = I, which is
    #      idempotent and has E_U = 0.
    wl = w.small_test_system(n=(16, 16, 16), natoms=2, kpt=kpt)
    g = o.Grid(wl.n, wl.L, kpt)
    H = o.Hamiltonian(g, wl.veff, wl.atoms)
    idx, vals, _ = H.hub[0]
    Phi = np.zeros((g.Nd, 5), dtype=vals.dtype)
    Phi[idx] = vals
    S = g.dV * Phi.conj().T @ Phi
    ev, U = np.linalg.eigh(S)
    X1 = Phi @ (U @ np.diag(ev ** -0.5) @ U.conj().T)
    np.testing.assert_allclose(g.inner(X1, X1), np.eye(5), atol=1e-12)
    D1 = o.occupation_matrices(H, X1, np.ones(5))
    np.testing.assert_allclose(D1[0], S, atol=1e-13)
    X2 = Phi @ np.linalg.inv(S)
    D2 = o.occupation_matrices(H, X2, np.ones(5))
    np.testing.assert_allclose(D2[0], np.eye(5), atol=1e-12)
    np.testing.assert_allclose(D2[1], D2[1].conj().T, atol=1e-14)
    assert abs(o.hubbard_energy(np.real(D2[:1]), [1.0])) < 1e-11


@pytest.mark.parametrize("kpt", [(0.0, 0.0, 0.0), (0.25, 0.1, -0.15)])
def test_occupation_equals_gram_for_complete_basis(kpt):
    # X = I / sqrt(dV) is a grid-orthonormal basis of the whole space: D = <phi_m|phi_m'>^T
    wl = w.small_test_system(n=(8, 9, 10), natoms=2, kpt=kpt, hub_rc=2.5, kb_rc=2.0)
    g = o.Grid(wl.n, wl.L, kpt)
    H = o.Hamiltonian(g, wl.veff, wl.atoms)
    X = np.eye(g.Nd) / np.sqrt(g.dV)
    D = o.occupation_matrices(H, X, np.ones(g.Nd))
    for I, (idx, vals, _) in enumerate(H.hub):
        G = g.dV * vals.conj().T @ vals          # G[m, m'] = <phi_m|phi_m'>
        # D_mm' = sum_n <psi_n|phi_m'><phi_m|psi_n> = <phi_m|phi_m'>
        np.testing.assert_allclose(D[I], G, atol=1e-13)
        np.testing.assert_allclose(D[I], D[I].conj().T, atol=1e-14)


def test_hubbard_energy_closed_forms():
    U = [0.3, 0.5]
    assert o.hubbard_energy(np.zeros((2, 5, 5)), U) == 0.0
    assert abs(o.hubbard_energy(np.array([np.eye(5)] * 2), U)) < 1e-15
    half = np.array([0.5 * np.eye(5)] * 2)
    assert abs(o.hubbard_energy(half, U) - sum(u / 8 * 5 for u in U)) < 1e-15
    # a rank-2 orthogonal projector is idempotent
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((5, 5)))
    P = Q[:, :2] @ Q[:, :2].T
    assert abs(o.hubbard_energy(np.array([P]), [0.7])) < 1e-14
    # invariance under an orthogonal change of basis
    D = _random_D(1, 9)
    E1 = o.hubbard_energy(D, [0.4])
    E2 = o.hubbard_energy(np.array([Q.T @ D[0] @ Q]), [0.4])
    assert abs(E1 - E2) < 1e-14
    assert abs(E1 - 0.2 * (np.trace(D[0]) - np.trace(D[0] @ D[0]))) < 1e-14


def check_hubbard_derivative(kpt, seed=11):
    """dE_U/deps along a perturbation delta = 2 Re sum_n f_n <delta_n|V_U[D(X)]|x_n>
    (Sec. II.A.2: dE_U/dpsi_n^* = f_n V_U psi_n).  Returns (finite difference, analytic)."""
    wl = w.small_test_system(n=(12, 12, 12), natoms=2, kpt=kpt)
    g = o.Grid(wl.n, wl.L, kpt)
    H = o.Hamiltonian(g, wl.veff, wl.atoms)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((g.Nd, 6)) * 0.3
    dX = rng.standard_normal((g.Nd, 6))
    if g.is_complex:
        X = X + 0.3j * rng.standard_normal((g.Nd, 6))
        dX = dX + 1j * rng.standard_normal((g.Nd, 6))
    f = rng.uniform(0.2, 1.0, 6)
    U = [h[2] for h in H.hub]

    def EU(Xe):
        return o.hubbard_energy(o.occupation_matrices(H, Xe, f), U)

    eps = 1e-5
    fd = (EU(X + eps * dX) - EU(X - eps * dX)) / (2 * eps)
    H.set_occupation(o.occupation_matrices(H, X, f))
    VX = H.hubbard(X)
    an = 2.0 * g.dV * float(np.real(np.sum(f[None, :] * dX.conj() * VX)))
    return fd, an


@pytest.mark.parametrize("kpt", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.25)])
def test_hubbard_potential_is_derivative_of_hubbard_energy(kpt):
    fd, an = check_hubbard_derivative(kpt)
    print("finite difference", fd, "analytic", an)
    assert abs(fd - an) < 1e-7 * max(1.0, abs(an))
