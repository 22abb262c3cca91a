"""Mutation checks: plant a plausible mistake in the oracle (on the CPU, by monkeypatching)
and confirm that one of the pins fails.  This shows that the pins discriminate, i.e. that
a dropped term, a wrong sign or a transposed operand in the oracle would not go unseen."""
import numpy as np
import pytest

from oracle import hubbard as o
import test_oracle_fd as tfd
import test_oracle_hamiltonian as th
import test_oracle_chefsi as tc


def test_wrong_laplacian_weight_is_caught(monkeypatch):
    good = o.fd_laplacian_weights

    def bad(n0):
        c0, c = good(n0)
        c = c.copy()
        c[1] = -c[1]                     # wrong sign of the p = 2 weight
        return c0, c
    monkeypatch.setattr(o, "fd_laplacian_weights", bad)
    with pytest.raises(AssertionError):
        tfd.test_weights_match_published_table()
    with pytest.raises(AssertionError):
        tfd.test_second_derivative_exact_on_polynomials(6)


def test_wrong_bloch_phase_is_caught(monkeypatch):
    good = o.bloch_shift

    def bad(F, grid, axis, p):
        grid2 = o.Grid(grid.n, grid.L, -grid.kpt, grid.n0)    # conjugated Bloch factor
        return good(F, grid2, axis, p)
    monkeypatch.setattr(o, "bloch_shift", bad)
    with pytest.raises(AssertionError):
        tfd.test_fourier_symbol_plane_and_bloch_waves((0.13, -0.27, 0.41))


def test_transposed_hubbard_coefficients_are_caught(monkeypatch):
    def bad_hubbard(self, X):
        Y = np.zeros(X.shape, dtype=np.result_type(X, self.hub[0][1]))
        for I, (idx, vals, U) in enumerate(self.hub):
            M = self.hubbard_coefficients(I)
            C = self.grid.dV * (vals.conj().T @ X[idx])
            Y[idx] += vals @ (M.T @ C)        # literal D_mm' slot: transposed coefficients
        return Y
    monkeypatch.setattr(o.Hamiltonian, "hubbard", bad_hubbard)
    fd, an = th.check_hubbard_derivative((0.3, -0.2, 0.25))
    assert abs(fd - an) > 1e-6 * max(1.0, abs(an))


def test_dropped_factor_two_in_hubbard_coefficients_is_caught(monkeypatch):
    def bad_coef(self, I):
        return 0.5 * self.hub[I][2] * (np.eye(5) - self.D[I])     # (delta - D), not (delta - 2D)
    monkeypatch.setattr(o.Hamiltonian, "hubbard_coefficients", bad_coef)
    fd, an = th.check_hubbard_derivative((0.0, 0.0, 0.0))
    assert abs(fd - an) > 1e-6 * max(1.0, abs(an))


def test_missing_volume_element_in_occupation_is_caught(monkeypatch):
    good = o.occupation_matrices

    def bad(ham, X, f, kweight=1.0):
        return good(ham, X, f, kweight) / ham.grid.dV
    monkeypatch.setattr(o, "occupation_matrices", bad)
    with pytest.raises(AssertionError):
        tc_kpt = (0.0, 0.0, 0.0)
        th.test_occupation_identities_for_orbital_built_states(tc_kpt)


def test_wrong_filter_recurrence_is_caught(monkeypatch):
    def bad_filter(ham, X, m, a, b, a_low):
        e, c = 0.5 * (b - a), 0.5 * (b + a)
        sigma = e / (a_low - c)
        tau = 2.0 / sigma
        Y = (sigma / e) * (ham.apply(X) - c * X)
        for _ in range(2, m + 1):
            sigma_new = 1.0 / (tau - sigma)
            Ynew = (2.0 * sigma_new / e) * (ham.apply(Y) - c * Y) - sigma_new * X   # dropped sigma
            X, Y, sigma = Y, Ynew, sigma_new
        return Y
    monkeypatch.setattr(o, "chebyshev_filter", bad_filter)
    with pytest.raises(AssertionError):
        tc.test_filter_equals_chebyshev_polynomial_of_dense_H((0.0, 0.0, 0.0))


def _force_variant(coef_fn, grad_sign=1.0):
    """A copy of the oracle's Hubbard force with one planted change: the coefficient of the
    (m, m') term and the sign of the orbital gradient."""
    def forces(ham, X, f, kweight=1.0, D=None):
        D = ham.D if D is None else np.asarray(D)
        f = np.asarray(f, dtype=np.float64)
        out = np.zeros((len(ham.hub), 3))
        for I, (idx, vals, U) in enumerate(ham.hub):
            C = ham.grid.dV * (vals.conj().T @ X[idx])
            for a in range(3):
                G = grad_sign * ham.grid.dV * (vals.conj().T @ o.gradient(X, ham.grid, a)[idx])
                s = np.einsum("n,pn,mn->mp", f, np.conj(G), C)        # s[m, m']
                out[I, a] = np.real(np.sum(coef_fn(U, D[I]) * kweight * s))
        return out
    return forces


@pytest.mark.parametrize("name,coef,sign", [
    ("dropped delta term", lambda U, D: U * 2.0 * D.T, 1.0),
    ("D_mm' in the chain-rule slot", lambda U, D: U * (2.0 * D - np.eye(5)), 1.0),
    ("U/2 instead of U", lambda U, D: 0.5 * U * (2.0 * D.T - np.eye(5)), 1.0),
    ("gradient sign", lambda U, D: U * (2.0 * D.T - np.eye(5)), -1.0)])
def test_planted_force_mistakes_are_caught(monkeypatch, name, coef, sign):
    import test_oracle_forces as tf
    monkeypatch.setattr(o, "hubbard_forces", _force_variant(coef, sign))
    F, Ffd = tf.fd_and_formula(tf.K_POINT, n=28)
    assert np.max(np.abs(F - Ffd)) / np.max(np.abs(Ffd)) > 1e-2, name


def test_unplanted_force_variant_passes(monkeypatch):
    # the einsum rewrite used by the mutations is itself the oracle's formula
    import test_oracle_forces as tf
    monkeypatch.setattr(o, "hubbard_forces", _force_variant(lambda U, D: U * (2.0 * D.T - np.eye(5))))
    F, Ffd = tf.fd_and_formula(tf.K_POINT, n=28)
    assert np.max(np.abs(F - Ffd)) / np.max(np.abs(Ffd)) < 1e-3


def test_planted_density_scf_mistakes_are_caught(monkeypatch):
    import test_oracle_density_scf as tds
    from oracle import density_scf as ds
    good_h = ds.hartree_potential
    good_x = ds.lda_exchange
    # Hartree with the wrong sign
    monkeypatch.setattr(ds, "hartree_potential", lambda rho, g: -good_h(rho, g))
    with pytest.raises(AssertionError):
        tds.test_hartree_solves_the_fd_poisson_problem()
    monkeypatch.setattr(ds, "hartree_potential", good_h)

    # exchange potential without the 4/3 of the derivative
    def bad_x(rhos, g):
        v, E = good_x(rhos, g)
        return [0.75 * vv for vv in v], E
    monkeypatch.setattr(ds, "lda_exchange", bad_x)
    with pytest.raises(AssertionError):
        tds.test_exchange_potential_is_the_derivative_of_the_energy(1)
    monkeypatch.setattr(ds, "lda_exchange", good_x)

    # two channels without the spin-scaling factor 2^(1/3)
    def bad_spin(rhos, g):
        v, E = good_x(rhos, g)
        if len(rhos) == 2:
            f = 2.0 ** (-1.0 / 3.0)
            return [f * vv for vv in v], f * E
        return v, E
    monkeypatch.setattr(ds, "lda_exchange", bad_spin)
    with pytest.raises(AssertionError):
        tds.test_spin_scaling_relation()
    monkeypatch.setattr(ds, "lda_exchange", good_x)

    # the band-structure energy without the Hubbard double counting: the identity with the
    # directly evaluated functional breaks
    monkeypatch.setattr(ds, "hubbard_double_counting", lambda ham, D: 0.0)
    with pytest.raises(AssertionError):
        tds.test_model_b_scf_spin_polarized()


def test_planted_stress_mistakes_are_caught(monkeypatch):
    import test_oracle_stress as ts
    good_table = o.atom_function_table

    # moments about the atom with in-cell coordinates instead of about each image
    def bad_table(grid, R, channels, rc, moments=False):
        idx, vals = good_table(grid, R, channels, rc)
        if not moments:
            return idx, vals
        x = grid.coords()[idx]
        mom = np.stack([vals * (x[:, b] - np.asarray(R)[b])[:, None] for b in range(3)])
        return idx, vals, mom
    monkeypatch.setattr(o, "atom_function_table", bad_table)
    with pytest.raises(AssertionError):
        ts.test_lattice_translation_of_an_atom_leaves_the_stress_unchanged()
    monkeypatch.setattr(o, "atom_function_table", good_table)

    # without the delta_ab term of the volume change, or without 1/|Omega|
    good_stress = o.hubbard_stress

    def no_delta(ham, atoms, X, f, kweight=1.0, D=None):
        sig = good_stress(ham, atoms, X, f, kweight, D)
        Dm = ham.D if D is None else np.asarray(D)
        omega = ham.grid.Nd * ham.grid.dV
        tr = sum(0.5 * a.hub_U * float(np.real(np.trace(Dm[J]) - 2 * np.trace(Dm[J] @ Dm[J])))
                 for J, a in enumerate([a for a in atoms if a.hub_l >= 0]))
        return sig + np.eye(3) * tr / omega            # removes the -delta_ab term
    monkeypatch.setattr(o, "hubbard_stress", no_delta)
    with pytest.raises(AssertionError):
        ts.test_diagonal_stress_is_the_strain_derivative_of_EU((0.0, 0.0, 0.0))
    monkeypatch.setattr(o, "hubbard_stress",
                        lambda ham, atoms, X, f, kweight=1.0, D=None:
                        good_stress(ham, atoms, X, f, kweight, D) * ham.grid.Nd * ham.grid.dV)
    with pytest.raises(AssertionError):
        ts.test_diagonal_stress_is_the_strain_derivative_of_EU((0.0, 0.0, 0.0))
