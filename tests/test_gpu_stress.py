"""Parity of the Hubbard stress tensor (Sec. II.A.4) through the C ABI with the CPU oracle:
real and Bloch orbitals, FP64 and float handles, a cell small enough that periodic images
of one atom overlap, and the sum over blocks.

Tolerance: FP64 1e-10 relative (norm of the difference over the norm of the
oracle's tensor); float handles 1e-4 (float gradient and products)."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import make_hub, oracle_ham, to_dev, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F32, HUB_F64  # noqa: E402

KPT = (0.21, -0.13, 0.34)


def systems():
    return {
        "ragged": w.small_test_system(n=(20, 24, 28), ncol=37, natoms=3),
        "images-overlap": w.small_test_system(n=(12, 10, 14), ncol=6, natoms=2, hub_rc=3.0),
        "bloch": w.small_test_system(n=(12, 10, 14), ncol=6, natoms=3, kpt=KPT),
    }


def _case(name, prec):
    wl = systems()[name]
    cplx = name == "bloch"
    X = wl.orbitals(complex_=cplx)
    if prec != HUB_F64:
        X = X.astype(np.complex64 if cplx else np.float32).astype(np.complex128 if cplx else np.float64)
    f = np.linspace(1.0, 0.1, X.shape[0])
    D = wl.D0[0]
    H = oracle_ham(wl, D=D)
    ref = o.hubbard_stress(H, wl.atoms, X.T, f, 0.7)
    hb = make_hub(wl, prec)
    hb.set_occupation_matrix(0, D)
    sig = hb.hubbard_stress(0, to_dev(X, hb.dtype), f, 0.7)
    return sig, ref


@pytest.mark.parametrize("name", list(systems()))
def test_hubbard_stress_fp64(name):
    sig, ref = _case(name, HUB_F64)
    print(name, "max |sigma|", np.max(np.abs(ref)), "rel err", rel(sig, ref))
    assert np.max(np.abs(ref)) > 0
    assert rel(sig, ref) < 1e-10


@pytest.mark.parametrize("name", ["ragged", "bloch"])
def test_hubbard_stress_float(name):
    sig, ref = _case(name, HUB_F32)
    assert rel(sig, ref) < 1e-4


def test_stress_blocks_add_up():
    wl = systems()["ragged"]
    X = wl.orbitals()
    f = np.linspace(1.0, 0.1, X.shape[0])
    hb = make_hub(wl, HUB_F64)
    hb.set_occupation_matrix(0, wl.D0[0])
    Xd = to_dev(X, hb.dtype)
    whole = hb.hubbard_stress(0, Xd, f, 1.0)
    parts = hb.hubbard_stress(0, Xd[:20].contiguous(), f[:20], 1.0) + \
        hb.hubbard_stress(0, Xd[20:].contiguous(), f[20:], 1.0)
    assert rel(parts, whole) < 1e-12


def test_scf_forces_and_stress_of_the_converged_state():
    # hub_scf_forces sums the channels of the SCF's last iteration with D_out; the oracle
    # evaluates the same sums from the downloaded orbitals, occupations and D_out
    from paper_2507_23612_gb300 import scf_params
    wl = w.small_test_system(n=(16, 14, 18), natoms=2, ncol=14, hub_rc=3.0, kb_rc=2.0, nspin=2)
    hb = make_hub(wl, HUB_F64)
    p = scf_params(nspin=2, ncol=wl.ncol, ld=wl.Nd, degree=12, max_iter=80, first_passes=4,
                   lanczos_steps=10, pulay_history=7, natoms=len(wl.atoms), pulay_beta=0.3,
                   kT=0.01, n_elec=16.0, tol_e_atom=1e-8, tol_D=1e-6)
    Xs = [to_dev(wl.orbitals(s), torch.float64) for s in range(2)]
    vs = [to_dev(wl.lanczos_start(s), torch.float64) for s in range(2)]
    hb.scf_begin(p, Xs, vs, wl.D0)
    res = hb.scf_run()
    assert res["converged"] == 1
    eig, occ, D = hb.scf_get()
    F, sig = hb.scf_forces(stress=True)
    F_ref = np.zeros((len(wl.atoms), 3))
    sig_ref = np.zeros((3, 3))
    hub_atoms = [i for i, a in enumerate(wl.atoms) if a.hub_l >= 0]
    for s in range(2):
        X = Xs[s].cpu().numpy().T
        H = oracle_ham(wl, D=D[s])
        F_ref[hub_atoms] += o.hubbard_forces(H, X, occ[s], 1.0)
        sig_ref += o.hubbard_stress(H, wl.atoms, X, occ[s], 1.0)
    assert rel(F, F_ref) < 1e-10
    assert rel(sig, sig_ref) < 1e-10


def test_full_size_rutile_forces_on_sampled_orbitals():
    # the benchmarked rutile 2x2x3 grid (88x88x84, 24 Hubbard Ti): forces of a few orbitals
    # against the oracle on the same orbitals (FP64)
    wl = w.rutile()
    cols = 6
    X = w.random_orbitals(wl.Nd, cols, 321).T                  # (Nd, cols)
    X = X / np.sqrt(wl.dV * np.sum(X * X, axis=0))
    f = np.linspace(1.0, 0.3, cols)
    H = oracle_ham(wl, D=wl.D0[0])
    ref_hub = o.hubbard_forces(H, X, f, 1.0)
    hub_atoms = [i for i, a in enumerate(wl.atoms) if a.hub_l >= 0]
    ref = np.zeros((len(wl.atoms), 3))
    ref[hub_atoms] = ref_hub
    hb = make_hub(wl, HUB_F64)
    hb.set_occupation_matrix(0, wl.D0[0])
    F = hb.hubbard_forces(0, to_dev(X.T, hb.dtype), f, 1.0)
    assert rel(F, ref) < 1e-10
