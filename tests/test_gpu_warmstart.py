"""Warm start of the SCF from the trained occupation model, end to end on the GPU: SCF
solutions of displaced rutile-shaped cells (computed by the library), training by the
library's MLP kernels, prediction for a cell it has not seen, and the SCF started from the
prediction.  The SCF stays the arbiter: it must reach the cold start's fixed point.

What the network gains: along an MD trajectory, where each step's SCF starts from the
previous step's converged orbitals (Sec. II.B, last paragraph), the SCFs started from the
model's D need fewer iterations than those started from the atomic guess of D (the method
without the network); the paper's own second-order extrapolation is run beside them."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F32, HUB_F64  # noqa: E402
from paper_2507_23612_gb300.md import trajectory_scf  # noqa: E402
from paper_2507_23612_gb300.warmstart import (OccupationModel, pack_occupations,  # noqa: E402
                                              scf_solve, unpack_occupations)

REPS = (1, 1, 2)      # 12 atoms (4 Ti), 44x44x56 grid, 58 orbitals per spin


@pytest.fixture(scope="module")
def trained():
    model = OccupationModel(nspin=2, seed=0)
    train = []
    for i in range(16):
        wl = w.rutile_snapshot(REPS, 0.1, seed=i)
        r = scf_solve(wl, HUB_F32, tol_e_atom=1e-6, tol_D=1e-5)
        assert r["converged"]
        model.add_solution(wl.atoms, wl.L, r["D"])
        train.append(pack_occupations(r["D"]))
    losses = model.fit(steps=1500)
    return model, train, losses


def test_warm_start_reaches_the_cold_fixed_point_from_a_better_guess(trained):
    model, train, losses = trained
    assert losses[-1] < 1e-2 * losses[0]
    mean_guess = np.mean(np.concatenate(train), axis=0, keepdims=True)

    wl = w.rutile_snapshot(REPS, 0.1, seed=100)
    cold = scf_solve(wl, HUB_F64)
    D_pred = model.predict(wl.atoms, wl.L)
    warm = scf_solve(wl, HUB_F64, D0=D_pred)
    exact = scf_solve(wl, HUB_F64, D0=cold["D"])     # the best any guess of D can do
    assert cold["converged"] and warm["converged"] and exact["converged"]
    nat = len(wl.atoms)
    err_atomic = np.abs(wl.D0 - cold["D"])
    err_pred = np.abs(D_pred - cold["D"])
    err_mean = np.abs(unpack_occupations(np.repeat(mean_guess, D_pred.shape[1], 0), 2) - cold["D"])
    print({"cold_iterations": cold["iterations"], "warm_iterations": warm["iterations"],
           "exact_D_iterations": exact["iterations"],
           "max_err_atomic": err_atomic.max(), "max_err_model": err_pred.max(),
           "rms_err_model": np.sqrt(np.mean(err_pred ** 2)), "rms_err_mean": np.sqrt(np.mean(err_mean ** 2))})
    # the model's guess is far closer to the fixed point than the atomic guess, and closer
    # than the training set's mean occupation matrix
    assert err_pred.max() < 0.05 * err_atomic.max()
    assert np.sqrt(np.mean(err_pred ** 2)) < np.sqrt(np.mean(err_mean ** 2))
    # same fixed point (both runs stop at |dE| < 1e-5 Ha/atom and max|dD| < 1e-4)
    assert abs(warm["E"] - cold["E"]) / nat < 1e-6
    assert np.max(np.abs(warm["D"] - cold["D"])) < 5e-4


def test_trained_model_saves_scf_iterations_along_a_trajectory(trained):
    """From random orbitals the iteration count is set by the convergence of the orbital
    subspace, whatever the starting D; once the orbitals of the previous MD step start each
    SCF, the starting D decides it.  Seeded sinusoidal trajectory of the 12-atom cell
    (0.1 bohr, period 12 steps), six steps; the first step starts from random orbitals in
    every run, the later ones from the previous step's orbitals."""
    model = trained[0]
    steps = w.rutile_trajectory(REPS, nsteps=6, amplitude=0.1, period=12.0)
    runs = {start: trajectory_scf(steps, HUB_F32, start=start, model=model, tol_e_atom=1e-6)
            for start in ("atomic", "extrapolated", "mlp")}
    its = {k: [r["iterations"] for r in v] for k, v in runs.items()}
    print(its)
    nat = len(steps[0].atoms)
    for k in ("extrapolated", "mlp"):
        for a, b in zip(runs["atomic"], runs[k]):
            assert a["converged"] and b["converged"]
            assert abs(a["E"] - b["E"]) / nat < 1e-5
    # the network's gain over the method without it (atomic-guess D), over the steps that
    # reuse orbitals
    assert sum(its["mlp"][1:]) < sum(its["atomic"][1:])
