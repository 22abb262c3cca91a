"""Pins for the oracle's Hubbard stress tensor (Sec. II.A.4).

The stress is (1/|Omega|) dE_U/dF at fixed orbitals carried along by the deformation
psi'(x) = psi(F^-1 x) / sqrt(det F).  For a diagonal strain of the orthorhombic cell the
deformed problem is again a grid problem: the same nodes with h_a (1 + eps), atoms at F R,
orbital values divided by sqrt(1 + eps), and the Bloch vector k_a / (1 + eps) (the same
phase per cell).  The diagonal components are pinned to central differences of the oracle's
E_U there (no gradient, no moments, no chain rule in common with the formula).  The other
pins: invariance under moving an atom by a lattice vector (which catches a moment taken
about the atom rather than each image), zero stress for D = I/2, and the symmetry of the
off-diagonal components to discretisation accuracy."""
import numpy as np
import pytest

from oracle import hubbard as o
import workloads as w

K_POINT = (0.21, -0.13, 0.34)


def _system(k=(0.0, 0.0, 0.0), n=36, L=9.0, rs=1.0, seed=0, ncol=5):
    rng = np.random.default_rng(seed)
    Ls = (L, L * (n + 2) / n, L * (n - 2) / n)
    ns = (n, n + 2, n - 2)
    atoms = [w.Atom("Ti", np.array([2.1, 3.3, 4.05]), hub_l=2, hub_rs=rs, hub_rc=8 * rs, hub_U=0.18),
             w.Atom("Ti", np.array([6.7, 5.2, 1.3]), hub_l=2, hub_rs=1.1 * rs, hub_rc=8.8 * rs,
                    hub_U=0.25)]
    Nd = int(np.prod(ns))
    X = rng.standard_normal((Nd, ncol))
    if any(k):
        X = X + 1j * rng.standard_normal((Nd, ncol))
    f = rng.uniform(0.2, 1.0, ncol)
    return ns, Ls, atoms, X, f


def _strained_energy(ns, Ls, k, atoms, X, f, kweight, axis, eps):
    s = np.ones(3)
    s[axis] += eps
    g = o.Grid(ns, tuple(np.asarray(Ls) * s), tuple(np.asarray(k) / s))
    at = [w.Atom(a.species, a.pos * s, hub_l=a.hub_l, hub_rs=a.hub_rs, hub_rc=a.hub_rc, hub_U=a.hub_U)
          for a in atoms]
    ham = o.Hamiltonian(g, np.zeros(g.Nd), at)
    D = o.occupation_matrices(ham, X / np.sqrt(1.0 + eps), f, kweight)
    return o.hubbard_energy(D, [a.hub_U for a in at])


def stress_and_fd(k, n=36, kweight=0.7, delta=1e-5):
    ns, Ls, atoms, X, f = _system(k, n=n)
    g = o.Grid(ns, Ls, k)
    ham = o.Hamiltonian(g, np.zeros(g.Nd), atoms)
    D = o.occupation_matrices(ham, X, f, kweight)
    sig = o.hubbard_stress(ham, atoms, X, f, kweight, D)
    omega = g.Nd * g.dV
    fd = np.array([(_strained_energy(ns, Ls, k, atoms, X, f, kweight, a, delta)
                    - _strained_energy(ns, Ls, k, atoms, X, f, kweight, a, -delta)) / (2 * delta * omega)
                   for a in range(3)])
    return sig, fd


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), K_POINT], ids=["gamma", "bloch"])
def test_diagonal_stress_is_the_strain_derivative_of_EU(k):
    sig, fd = stress_and_fd(k)
    err = np.max(np.abs(np.diag(sig) - fd)) / np.max(np.abs(fd))
    print({"diag": np.diag(sig).tolist(), "fd": fd.tolist(), "rel_err": float(err)})
    assert np.max(np.abs(fd)) > 1e-6
    assert err < 1e-5


def test_lattice_translation_of_an_atom_leaves_the_stress_unchanged():
    ns, Ls, atoms, X, f = _system(K_POINT, n=24, L=8.0)
    g = o.Grid(ns, Ls, K_POINT)
    ham = o.Hamiltonian(g, np.zeros(g.Nd), atoms)
    D = o.occupation_matrices(ham, X, f, 1.0)
    sig = o.hubbard_stress(ham, atoms, X, f, 1.0, D)
    moved = [w.Atom(a.species, a.pos + np.array([Ls[0], -Ls[1], 0.0]) * (i == 0), hub_l=a.hub_l,
                    hub_rs=a.hub_rs, hub_rc=a.hub_rc, hub_U=a.hub_U) for i, a in enumerate(atoms)]
    ham2 = o.Hamiltonian(g, np.zeros(g.Nd), moved)
    sig2 = o.hubbard_stress(ham2, moved, X, f, 1.0, D)
    np.testing.assert_allclose(sig2, sig, atol=1e-12 * np.max(np.abs(sig)))


def test_half_filled_shell_has_no_hubbard_stress():
    ns, Ls, atoms, X, f = _system(K_POINT, n=24, L=8.0)
    g = o.Grid(ns, Ls, K_POINT)
    ham = o.Hamiltonian(g, np.zeros(g.Nd), atoms)
    D = np.array([0.5 * np.eye(5)] * 2)
    assert np.max(np.abs(o.hubbard_stress(ham, atoms, X, f, 1.0, D))) < 1e-16


def test_off_diagonal_components_are_symmetric_to_discretisation_accuracy():
    # E_U is invariant under rigid rotations of atoms and orbitals together, so the
    # antisymmetric part of dE/dF vanishes in the continuum; on the grid it is small
    sig, _ = stress_and_fd((0.0, 0.0, 0.0))
    off = [(0, 1), (0, 2), (1, 2)]
    asym = max(abs(sig[a, b] - sig[b, a]) for a, b in off)
    scale = max(abs(sig[a, b]) for a, b in off)
    print({"offdiag": [sig[a, b] for a, b in off], "asym": asym})
    assert scale > 1e-7 and asym < 1e-5 * np.max(np.abs(sig))


def test_blocks_sum_to_the_whole():
    # with the prefactor D fixed, the stress is additive over blocks of states (spins,
    # k-points, or a split of the states), the delta term included
    ns, Ls, atoms, X, f = _system(K_POINT, n=24, L=8.0)
    g = o.Grid(ns, Ls, K_POINT)
    ham = o.Hamiltonian(g, np.zeros(g.Nd), atoms)
    D = o.occupation_matrices(ham, X, f, 0.6)
    whole = o.hubbard_stress(ham, atoms, X, f, 0.6, D)
    parts = o.hubbard_stress(ham, atoms, X[:, :2], f[:2], 0.6, D) + \
        o.hubbard_stress(ham, atoms, X[:, 2:], f[2:], 0.6, D)
    np.testing.assert_allclose(parts, whole, atol=1e-13 * np.max(np.abs(whole)))
