"""Density warm start of the self-consistent density SCF, end to end on the GPU: the density
basis fit through the library's projector products against the oracle's fit, and a
per-species model trained on converged densities of displaced cells, whose predicted
starting density leads the SCF to the cold start's fixed point."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from oracle import density_scf as ds

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F32, HUB_F64  # noqa: E402
from paper_2507_23612_gb300.warmstart import DensityBasis, DensityModel, density_scf_solve  # noqa: E402

REPS = (1, 1, 2)


def test_density_basis_fit_matches_the_oracle():
    wl = w.rutile_snapshot(REPS, 0.1, seed=3)
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.0, 1.0, wl.Nd)
    basis = DensityBasis(wl)
    try:
        c = basis.fit(torch.tensor(rho, dtype=torch.float64, device="cuda").contiguous())
    finally:
        basis.close()
    g = o.Grid(wl.n, wl.L)
    c_ref = ds.fit_density_coefficients(g, ds.density_basis_atoms(wl.atoms), rho)
    assert np.max(np.abs(c - c_ref)) < 1e-8 * np.max(np.abs(c_ref))


def test_density_warm_start_reaches_the_cold_fixed_point():
    model = DensityModel(seed=0)
    for i in range(6):
        wl = w.rutile_snapshot(REPS, 0.1, seed=i)
        r = density_scf_solve(wl, HUB_F32, tol_e_atom=1e-6)
        assert r["converged"]
        basis = DensityBasis(wl)
        model.add_solution(wl.atoms, wl.L, basis.fit(r["rho"]))
        basis.close()
    model.fit(steps=1000)
    wl = w.rutile_snapshot(REPS, 0.1, seed=100)
    cold = density_scf_solve(wl, HUB_F64)
    basis = DensityBasis(wl)
    rho0 = basis.expand(model.predict(wl.atoms, wl.L), wl.n_elec)
    basis.close()
    warm = density_scf_solve(wl, HUB_F64, rho0=rho0)
    print({"cold_iterations": cold["iterations"], "warm_iterations": warm["iterations"]})
    assert cold["converged"] and warm["converged"]
    assert abs(warm["E"] - cold["E"]) / len(wl.atoms) < 1e-5
    # with the potential self-consistent the starting density matters: the predicted one
    # must not need more iterations than the uniform start
    assert warm["iterations"] <= cold["iterations"]
