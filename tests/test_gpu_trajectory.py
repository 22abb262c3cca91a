"""SCF along a seeded MD trajectory (Sec. II.B, last paragraph): starting D from the atomic
guess or from the second-order extrapolation of the previous steps, the previous orbitals
reused.  Both reach the same fixed point at every step; the iteration counts are reported."""
import pytest

import workloads as w

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F32  # noqa: E402
from paper_2507_23612_gb300.md import trajectory_scf  # noqa: E402


def test_extrapolated_and_atomic_starts_reach_the_same_fixed_points():
    steps = w.rutile_trajectory((1, 1, 2), nsteps=5, amplitude=0.1, period=12.0)
    atomic = trajectory_scf(steps, HUB_F32, start="atomic", tol_e_atom=1e-6)
    extra = trajectory_scf(steps, HUB_F32, start="extrapolated", tol_e_atom=1e-6)
    print({"atomic": [s["iterations"] for s in atomic], "extrapolated": [s["iterations"] for s in extra],
           "alpha_beta": [s["alpha_beta"] for s in extra]})
    nat = len(steps[0].atoms)
    for a, e in zip(atomic, extra):
        assert a["converged"] and e["converged"]
        assert abs(a["E"] - e["E"]) / nat < 1e-5
    # from the fourth step on the fit sees two position steps of a sinusoid of period 12:
    # alpha = 2 cos(2 pi / 12), beta = -1
    al, be = extra[3]["alpha_beta"]
    assert abs(al - 3 ** 0.5) < 1e-6 and abs(be + 1.0) < 1e-6


def test_resume_from_a_checkpoint_reaches_the_same_fixed_point(tmp_path):
    from paper_2507_23612_gb300.md import load_scf_checkpoint, save_scf_checkpoint
    from paper_2507_23612_gb300.warmstart import scf_solve
    wl = w.rutile_snapshot((1, 1, 2), 0.1, seed=5)
    full = scf_solve(wl, HUB_F32, tol_e_atom=1e-6)
    part = scf_solve(wl, HUB_F32, tol_e_atom=1e-6, max_iter=4, keep_orbitals=True)
    assert not part["converged"]
    save_scf_checkpoint(tmp_path / "scf.npz", part["X"], part["D"], {"iter": part["iterations"]})
    Xs, D, meta = load_scf_checkpoint(tmp_path / "scf.npz", device="cuda", dtype=torch.float32)
    resumed = scf_solve(wl, HUB_F32, D0=D, X0=Xs, tol_e_atom=1e-6)
    print({"full": full["iterations"], "resumed": meta["iter"] + resumed["iterations"]})
    assert full["converged"] and resumed["converged"]
    assert abs(full["E"] - resumed["E"]) / len(wl.atoms) < 1e-6
