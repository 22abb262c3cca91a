"""Pins for the value-threshold truncation of the radial orbitals (Sec. II.B) and the
convergence of E_U with the threshold (the paper's truncation study, on a small synthetic
cell): the cutoff radius of an s function in closed form, the defining equation for l > 0,
the library's host implementation against the oracle, and E_U(tau) approaching its
converged value as tau decreases."""
import ctypes as C
from math import log, sqrt

import numpy as np
import pytest

from oracle import hubbard as o
import workloads as w


def test_s_function_cutoff_in_closed_form():
    rs, tau = 0.9, 1e-3
    N = o.radial_norm(0, rs)
    assert abs(o.cutoff_for_threshold(0, rs, tau) - rs * sqrt(2 * log(N / tau))) < 1e-12


@pytest.mark.parametrize("l,rs,tau", [(1, 0.8, 1e-2), (2, 1.0, 5e-3), (2, 1.0, 1e-4), (2, 1.3, 1e-6)])
def test_cutoff_solves_the_threshold_equation_beyond_the_maximum(l, rs, tau):
    rc = o.cutoff_for_threshold(l, rs, tau)
    N = o.radial_norm(l, rs)
    f = lambda r: N * r ** l * np.exp(-r * r / (2 * rs * rs))      # noqa: E731
    assert rc > rs * sqrt(l)
    assert abs(f(rc) - tau) < 1e-12 * max(tau, 1e-300) + 1e-15
    assert f(rc * 1.01) < tau < f(rc * 0.99)


def test_threshold_above_the_maximum_gives_no_support():
    assert o.cutoff_for_threshold(2, 1.0, 10.0) == 0.0


@pytest.fixture(scope="module")
def lib():
    from paper_2507_23612_gb300 import build as b
    b.build()
    from paper_2507_23612_gb300 import binding
    return binding.load_library()


@pytest.mark.parametrize("l,rs,tau", [(0, 0.8, 1e-3), (1, 0.8, 1e-2), (2, 1.0, 5e-3), (2, 1.0, 1e-8), (2, 1.0, 10.0)])
def test_library_cutoff_matches_the_oracle(lib, l, rs, tau):
    rc = C.c_double()
    assert lib.hub_cutoff_radius(l, C.c_double(rs), C.c_double(tau), C.byref(rc)) == 0
    assert abs(rc.value - o.cutoff_for_threshold(l, rs, tau)) < 1e-10


def test_hubbard_energy_converges_with_the_threshold():
    # one seeded set of orbitals, D and E_U from orbitals truncated at rc(tau): the error
    # against a tight threshold falls as tau falls (Sec. III's truncation study, in spirit)
    wl = w.small_test_system(n=(20, 20, 20), L=(8.0, 8.0, 8.0), ncol=10, natoms=2, hub_rc=6.0, seed=4)
    g = o.Grid(wl.n, wl.L)
    X = wl.orbitals().T
    f = np.linspace(1.0, 0.2, X.shape[1])

    def eu(tau):
        atoms = [w.Atom(a.species, a.pos, hub_l=a.hub_l, hub_rs=a.hub_rs,
                        hub_rc=o.cutoff_for_threshold(2, a.hub_rs, tau), hub_U=a.hub_U)
                 for a in wl.atoms if a.hub_l >= 0]
        ham = o.Hamiltonian(g, np.zeros(g.Nd), atoms)
        return o.hubbard_energy(o.occupation_matrices(ham, X, f), [a.hub_U for a in atoms])
    ref = eu(1e-9)
    # (a very coarse threshold can land near zero error by cancellation; from 1e-2 on the
    # error falls steadily)
    errs = [abs(eu(t) - ref) for t in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6)]
    print(errs)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3 * errs[0]
