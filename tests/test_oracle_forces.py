"""Pins for the oracle's Hubbard atomic forces (Sec. II.A.3).

The force is the negative derivative of E_U with respect to an atom position at fixed
orbitals and occupations.  The pin is that derivative itself, taken by central differences
of the oracle's E_U(D(R)) with the atomic orbitals re-sampled at R +- delta: it shares no
step with the force formula (no gradient of the orbitals, no chain rule), so a dropped
term, a wrong sign, a transposed D or a wrong Bloch phase in the formula fails it.  The two
differ by the discretisation of the transferred derivative (the FD gradient acting on the
orbitals instead of the analytic gradient of the atomic orbitals); on the grids below that
is below 1e-6 of the largest force, and it shrinks with h (checked by the coarser grid).
"""
import numpy as np
import pytest

from oracle import hubbard as o
import workloads as w

K_POINT = (0.21, -0.13, 0.34)


def _system(k=(0.0, 0.0, 0.0), n=36, L=9.0, rs=1.0, seed=0, ncol=5):
    """Two d shells (different U and widths) in a small orthorhombic cell, random orbitals.
    rc = 8 rs makes the hard cutoff negligible (the radial function is ~1e-12 there)."""
    rng = np.random.default_rng(seed)
    g = o.Grid((n, n + 2, n - 2), (L, L * (n + 2) / n, L * (n - 2) / n), k)
    atoms = [w.Atom("Ti", np.array([2.1, 3.3, 4.05]), hub_l=2, hub_rs=rs, hub_rc=8 * rs, hub_U=0.18),
             w.Atom("Ti", np.array([6.7, 5.2, 1.3]), hub_l=2, hub_rs=1.1 * rs, hub_rc=8.8 * rs,
                    hub_U=0.25)]
    X = rng.standard_normal((g.Nd, ncol))
    if g.is_complex:
        X = X + 1j * rng.standard_normal((g.Nd, ncol))
    f = rng.uniform(0.2, 1.0, ncol)
    return g, atoms, X, f


def _moved(atoms, J, a, d):
    out = [w.Atom(x.species, x.pos.copy(), hub_l=x.hub_l, hub_rs=x.hub_rs, hub_rc=x.hub_rc,
                  hub_U=x.hub_U) for x in atoms]
    out[J].pos[a] += d
    return out


def _energy_and_D(g, atoms, X, f, kweight):
    ham = o.Hamiltonian(g, np.zeros(g.Nd), atoms)
    D = o.occupation_matrices(ham, X, f, kweight)
    return o.hubbard_energy(D, [x.hub_U for x in atoms]), D, ham


def fd_and_formula(k, n=36, rs=1.0, kweight=0.7, delta=1e-4):
    g, atoms, X, f = _system(k, n=n, rs=rs)
    _, D, ham = _energy_and_D(g, atoms, X, f, kweight)
    F = o.hubbard_forces(ham, X, f, kweight, D)
    Ffd = np.zeros_like(F)
    for J in range(len(atoms)):
        for a in range(3):
            Ep = _energy_and_D(g, _moved(atoms, J, a, delta), X, f, kweight)[0]
            Em = _energy_and_D(g, _moved(atoms, J, a, -delta), X, f, kweight)[0]
            Ffd[J, a] = -(Ep - Em) / (2 * delta)
    return F, Ffd


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), K_POINT], ids=["gamma", "bloch"])
def test_force_is_minus_the_derivative_of_EU(k):
    F, Ffd = fd_and_formula(k)
    err = np.max(np.abs(F - Ffd)) / np.max(np.abs(Ffd))
    print({"max_force": float(np.max(np.abs(F))), "rel_err": float(err)})
    assert np.max(np.abs(Ffd)) > 1e-3          # the pin is not vacuous
    assert err < 3e-6


def test_discretisation_gap_shrinks_with_h():
    # same cell on a coarser grid: the transferred-derivative error grows, so the agreement
    # above is resolution, not coincidence
    F, Ffd = fd_and_formula(K_POINT, n=28)
    err = np.max(np.abs(F - Ffd)) / np.max(np.abs(Ffd))
    assert 3e-6 < err < 1e-3


def test_half_filled_shell_has_no_hubbard_force():
    # D = I/2 makes U (2D - I) vanish: no force, whatever the orbitals
    g, atoms, X, f = _system(K_POINT, n=24, L=8.0)
    ham = o.Hamiltonian(g, np.zeros(g.Nd), atoms)
    D = np.array([0.5 * np.eye(5)] * 2)
    assert np.max(np.abs(o.hubbard_forces(ham, X, f, 1.0, D))) < 1e-15


def test_kweight_and_occupations_scale_linearly():
    g, atoms, X, f = _system((0.0, 0.0, 0.0), n=24, L=8.0)
    ham = o.Hamiltonian(g, np.zeros(g.Nd), atoms)
    D = np.real(o.occupation_matrices(ham, X, f, 1.0))
    F1 = o.hubbard_forces(ham, X, f, 1.0, D)
    np.testing.assert_allclose(o.hubbard_forces(ham, X, f, 0.25, D), 0.25 * F1, rtol=1e-13, atol=1e-18)
    # splitting the states into two calls sums to the one call
    F_a = o.hubbard_forces(ham, X[:, :2], f[:2], 1.0, D)
    F_b = o.hubbard_forces(ham, X[:, 2:], f[2:], 1.0, D)
    np.testing.assert_allclose(F_a + F_b, F1, rtol=1e-12, atol=1e-17)
