"""Pins for the oracle's Chebyshev filter, Lanczos bounds, Rayleigh-Ritz, occupations and
SCF (Sec. II.B, last paragraph), against dense diagonalisation and closed forms."""
import numpy as np
import pytest

from oracle import hubbard as o
import workloads as w


def _dense_system(kpt=(0.0, 0.0, 0.0), n=(10, 11, 12)):
    wl = w.small_test_system(n=n, natoms=3, kpt=kpt, hub_rc=3.0, kb_rc=2.0)
    g = o.Grid(wl.n, wl.L, kpt)
    H = o.Hamiltonian(g, wl.veff, wl.atoms, wl.D0[0])
    return wl, g, H


@pytest.mark.parametrize("kpt", [(0.0, 0.0, 0.0), (0.2, 0.1, -0.3)])
def test_filter_equals_chebyshev_polynomial_of_dense_H(kpt):
    wl, g, H = _dense_system(kpt)
    A = H.dense()
    lam, V = np.linalg.eigh(A)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((g.Nd, 5))
    if g.is_complex:
        X = X + 1j * rng.standard_normal((g.Nd, 5))
    m, a_low, a, b = 12, lam[0] - 0.05, lam[40], lam[-1] + 0.5
    Y = o.chebyshev_filter(H, X, m, a, b, a_low)
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    p = o.chebyshev_T(m, (lam - c) / e) / o.chebyshev_T(m, np.array([(a_low - c) / e]))[0]
    ref = V @ (p[:, None] * (V.conj().T @ X))
    assert np.linalg.norm(Y - ref) <= 1e-10 * np.linalg.norm(ref)
    # on an exact eigenvector the filter is the scalar p_m(lambda)
    v = V[:, 3:4]
    np.testing.assert_allclose(o.chebyshev_filter(H, v, m, a, b, a_low), p[3] * v, atol=1e-10 * abs(p[3]))


def test_chebyshev_T_matches_recurrence():
    t = np.linspace(-3.0, 3.0, 61)
    T0, T1 = np.ones_like(t), t.copy()
    for m in range(2, 15):
        T0, T1 = T1, 2 * t * T1 - T0
        np.testing.assert_allclose(o.chebyshev_T(m, t), T1, rtol=1e-11, atol=1e-11)


def test_lanczos_bounds_bracket_spectrum():
    wl, g, H = _dense_system()
    lam = np.linalg.eigvalsh(H.dense())
    lo, up = o.lanczos_bounds(H, wl.lanczos_start(), 10)
    assert up >= lam[-1] - 1e-9           # the estimate is an upper bound here
    assert lo >= lam[0] - 1e-9            # a Ritz value never goes below the minimum
    assert up - lam[-1] < 0.35 * (lam[-1] - lam[0])     # and not a wild overestimate


@pytest.mark.parametrize("kpt", [(0.0, 0.0, 0.0), (0.15, -0.25, 0.05)])
def test_chefsi_converges_to_dense_eigenvalues(kpt):
    wl, g, H = _dense_system(kpt)
    lam_exact = np.linalg.eigvalsh(H.dense())
    ncol = 16
    rng = np.random.default_rng(7)
    X = rng.standard_normal((g.Nd, ncol))
    if g.is_complex:
        X = X + 1j * rng.standard_normal((g.Nd, ncol))
    lo, up = o.lanczos_bounds(H, wl.lanczos_start(complex_=g.is_complex), 10)
    a_low, a, b = lo, lo + 0.1 * (up - lo), up
    for it in range(30):
        Y = o.chebyshev_filter(H, X, 14, a, b, a_low)
        lam, X = o.rayleigh_ritz(H, Y)
        # Cauchy interlacing: Ritz values never fall below the true eigenvalues
        assert np.all(lam >= lam_exact[:ncol] - 1e-9)
        a_low, a = lam[0], lam[-1]
    np.testing.assert_allclose(lam[:12], lam_exact[:12], atol=1e-10)
    np.testing.assert_allclose(g.inner(X, X), np.eye(ncol), atol=1e-11)


def test_free_particle_spectrum():
    # U = 0, no projectors, constant V0: eigenvalues are the FD symbol of plane waves
    n, L = (8, 9, 10), (2.4, 2.8, 3.3)
    g = o.Grid(n, L)
    V0 = -0.7
    H = o.Hamiltonian(g, np.full(g.Nd, V0), [])
    c0, c = o.fd_laplacian_weights(6)
    ev = []
    for m1 in range(n[0]):
        for m2 in range(n[1]):
            for m3 in range(n[2]):
                q = 2 * np.pi * np.array([m1, m2, m3]) / g.L
                s = sum((c0 + 2 * sum(c[p - 1] * np.cos(p * q[a] * g.h[a]) for p in range(1, 7))) / g.h[a] ** 2
                        for a in range(3))
                ev.append(-0.5 * s + V0)
    ev = np.sort(ev)
    # 7 lowest: 1 + 2 + 2 + 2 (degenerate pairs +-G along each axis)
    ncol = 7
    assert ev[ncol] - ev[ncol - 1] > 1e-3
    X = np.random.default_rng(2).standard_normal((g.Nd, ncol + 3))
    a_low, a, b = ev[0] - 1.0, ev[20], 2 * ev[-1]
    for _ in range(25):
        lam, X = o.rayleigh_ritz(H, o.chebyshev_filter(H, X, 12, a, b, a_low))
        a_low, a = lam[0], lam[-1]
    np.testing.assert_allclose(lam[:ncol], ev[:ncol], atol=1e-10)
    # and the dense matrix agrees with the symbol everywhere
    np.testing.assert_allclose(np.linalg.eigvalsh(H.dense()), ev, atol=1e-10)


def test_fermi_dirac_counts_and_limits():
    e = [np.linspace(-1, 1, 40), np.linspace(-0.9, 1.2, 40)]
    f, mu = o.fermi_dirac(e, [1.0, 1.0], 0.01, 30.0, 1.0)
    assert abs(sum(np.sum(x) for x in f) - 30.0) < 1e-10
    assert all(np.all(np.diff(x) <= 0) for x in f)
    f0, _ = o.fermi_dirac([np.arange(10.0)], [1.0], 0.0, 8.0, 2.0)
    np.testing.assert_array_equal(f0[0], [1, 1, 1, 1, 0, 0, 0, 0, 0, 0])


def test_pulay_solves_linear_fixed_point():
    # Pulay/DIIS on a linear contraction reaches its fixed point
    rng = np.random.default_rng(0)
    A = rng.uniform(-0.2, 0.2, (6, 6))
    bvec = rng.standard_normal(6)
    x_star = np.linalg.solve(np.eye(6) - A, bvec)
    mix = o.Pulay(7, 0.3)
    x = np.zeros(6)
    for _ in range(20):
        x = mix.mix(x, A @ x + bvec)
    np.testing.assert_allclose(x, x_star, atol=1e-9)


def test_scf_chefsi_matches_dense_scf():
    # the SCF with CheFSI reaches the same fixed point as the SCF with dense eigensolves
    wl = w.small_test_system(n=(10, 10, 12), natoms=2, ncol=14, hub_rc=3.0, kb_rc=2.0, nspin=2)
    grid_args = (wl.n, wl.L, (0, 0, 0), 6)
    X0s = [wl.orbitals(s).T for s in range(2)]
    v0s = [wl.lanczos_start(s) for s in range(2)]
    kw = dict(n_elec=16.0, kT=0.01, degree=12, lanczos_v0s=v0s, max_iter=80, tol_e_atom=1e-11,
              tol_D=1e-8, first_passes=4)
    r1 = o.scf_model_a(grid_args, wl.veff, wl.atoms, wl.D0, X0s, **kw)
    r2 = o.scf_model_a(grid_args, wl.veff, wl.atoms, wl.D0, X0s, eig_solver="dense", **kw)
    assert r1["converged"] and r2["converged"]
    assert abs(r1["E"] - r2["E"]) < 1e-9
    np.testing.assert_allclose(r1["D"], r2["D"], atol=1e-7)
    # a fixed point: D_out(D_in) = D_in
    assert np.max(np.abs(r1["D"] - r1["D_in"])) < 1e-8


def test_fermi_entropy_closed_forms():
    # S = -sum f ln f + (1 - f) ln(1 - f): ln 2 per half-filled state, 0 for f in {0, 1}, and
    # the derivative dS/df = ln((1 - f) / f) (the Fermi-Dirac stationarity condition)
    assert abs(o.fermi_entropy([0.5, 0.5, 0.5]) - 3 * np.log(2.0)) < 1e-14
    assert abs(o.fermi_entropy([0.0, 1.0, 1.0, 0.0])) < 1e-12
    f, eps = 0.3, 1e-6
    d = (o.fermi_entropy([f + eps]) - o.fermi_entropy([f - eps])) / (2 * eps)
    assert abs(d - np.log((1 - f) / f)) < 1e-8
