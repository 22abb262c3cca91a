"""Pins for the MD extrapolation of the occupation matrices (Sec. II.B, last paragraph):
the fitted coefficients of constant-velocity and constant-acceleration trajectories, exact
extrapolation when D depends linearly on the positions along such trajectories, the atomic
guess without history, and the library's host implementation against the oracle."""
import ctypes as C

import numpy as np
import pytest

from oracle import hubbard as o


def _traj(kind, n=4, natoms=5, seed=0):
    rng = np.random.default_rng(seed)
    a, b, c = (rng.standard_normal((natoms, 3)) for _ in range(3))
    t = np.arange(n, dtype=np.float64)
    if kind == "linear":
        return [a + b * ti for ti in t]
    return [a + b * ti + 0.3 * c * ti * ti for ti in t]


def test_constant_velocity_gives_alpha_one_beta_zero():
    al, be = o.alfe_coefficients(_traj("linear"))
    # d1 = d2 = target: the two-coefficient system is singular; the one-coefficient fit
    assert abs(al - 1.0) < 1e-12 and be == 0.0
    al3, be3 = o.alfe_coefficients(_traj("linear")[1:])
    assert abs(al3 - 1.0) < 1e-12 and be3 == 0.0


def test_constant_acceleration_gives_two_and_minus_one():
    al, be = o.alfe_coefficients(_traj("quadratic"))
    assert abs(al - 2.0) < 1e-10 and abs(be + 1.0) < 1e-10


def test_linear_response_along_a_quadratic_trajectory_is_extrapolated_exactly():
    R = _traj("quadratic", n=4, natoms=3, seed=2)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((2 * 2 * 25, 9))                   # D depends linearly on R
    Da = np.tile(0.2 * np.eye(5), (2, 2, 1, 1))
    D_of = [Da + (A @ r.ravel()).reshape(2, 2, 5, 5) for r in R]
    al, be = o.alfe_coefficients(R)
    D_next = o.extrapolate_occupations(D_of[:3], Da, al, be)
    np.testing.assert_allclose(D_next, D_of[3], atol=1e-10)


def test_history_shorter_than_the_scheme():
    Da = 0.2 * np.eye(5)[None]
    np.testing.assert_array_equal(o.extrapolate_occupations([], Da, 2.0, -1.0), Da)
    D1 = Da + 0.01
    np.testing.assert_allclose(o.extrapolate_occupations([D1], Da, 2.0, -1.0), D1)
    assert o.alfe_coefficients(_traj("linear")[:2]) == (0.0, 0.0)


@pytest.fixture(scope="module")
def lib():
    from paper_2507_23612_gb300 import build as b
    b.build()
    from paper_2507_23612_gb300 import binding
    return binding.load_library()


@pytest.mark.parametrize("nhist", [0, 1, 2, 3])
def test_library_extrapolation_matches_the_oracle(lib, nhist):
    from paper_2507_23612_gb300.binding import extrapolate_occupations
    rng = np.random.default_rng(7 + nhist)
    R = _traj("quadratic", n=nhist + 1, natoms=4, seed=nhist)
    R = [r + 0.01 * rng.standard_normal(r.shape) for r in R]    # not exactly quadratic
    Da = np.tile(0.2 * np.eye(5), (2, 3, 1, 1))
    D_hist = [Da + 0.05 * rng.standard_normal(Da.shape) for _ in range(nhist)]
    al, be = o.alfe_coefficients(R)
    ref = o.extrapolate_occupations(D_hist, Da, al, be)
    D_next, (al2, be2) = extrapolate_occupations(D_hist, Da, R)
    assert abs(al2 - al) < 1e-12 and abs(be2 - be) < 1e-12
    np.testing.assert_allclose(D_next, ref, atol=1e-13)


def test_seeded_md_trajectory_is_a_sinusoid():
    # every coordinate follows a sinusoid of period 12 steps, so the two-step fit recovers
    # its recurrence x(t+1) = 2 cos(2 pi / 12) x(t) - x(t-1) about the rest position
    import workloads as w
    steps = w.rutile_trajectory((1, 1, 2), nsteps=5)
    R = [np.array([a.pos for a in s.atoms]) for s in steps]
    al, be = o.alfe_coefficients(R[:4])
    assert abs(al - 2 * np.cos(2 * np.pi / 12)) < 1e-9 and abs(be + 1.0) < 1e-9
    assert all(s.n == steps[0].n and s.ncol == steps[0].ncol for s in steps)


def test_trajectory_driver_orchestration_on_the_cpu(lib):
    # the MD driver with the oracle's SCF in place of the library's: each step starts from
    # the extrapolation of the previous converged D (checked against the oracle's formula)
    # and from the previous orbitals, and reaches the same fixed point as the atomic start
    import workloads as w
    from paper_2507_23612_gb300.md import trajectory_scf
    steps = w.rutile_trajectory((1, 1, 1), nsteps=4, amplitude=0.1, period=12.0, h_target=0.55,
                                occ_per_atom=2.0, nspin=1)

    def solve(wl, prec, D0=None, X0=None, tol_e_atom=1e-5, tol_D=1e-4):
        X = wl.orbitals(0).T if X0 is None else X0[0]
        r = o.scf_model_a((wl.n, wl.L, (0, 0, 0), wl.fd_half_order), wl.veff, wl.atoms, D0, [X],
                          n_elec=wl.n_elec, kT=0.01, degree=10, lanczos_v0s=[wl.lanczos_start(0)],
                          tol_e_atom=tol_e_atom, tol_D=tol_D, max_iter=80)
        return {"iterations": r["iterations"], "converged": r["converged"], "E": r["E"], "D": r["D"],
                "X": r["X"], "seconds": 0.0}
    atomic = trajectory_scf(steps, start="atomic", solve=solve, tol_e_atom=1e-7, tol_D=1e-6)
    extra = trajectory_scf(steps, start="extrapolated", solve=solve, tol_e_atom=1e-7, tol_D=1e-6)
    nat = len(steps[0].atoms)
    for t, (a, e) in enumerate(zip(atomic, extra)):
        assert a["converged"] and e["converged"]
        assert abs(a["E"] - e["E"]) / nat < 1e-5
        np.testing.assert_array_equal(a["D0"], steps[t].D0)
        if t >= 1:
            h = min(3, t)
            R = [np.array([x.pos for x in s.atoms]) for s in steps[t - h:t + 1]]
            al, be = o.alfe_coefficients(R)
            ref = o.extrapolate_occupations([extra[j]["D"] for j in range(t - h, t)], steps[t].D0, al, be)
            np.testing.assert_allclose(e["D0"], ref, atol=1e-12)
    print({"atomic": [a["iterations"] for a in atomic], "extrapolated": [e["iterations"] for e in extra]})
