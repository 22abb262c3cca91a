"""Parity of the Hubbard atomic forces (Sec. II.A.3) through the C ABI with the CPU oracle:
real and Bloch orbitals, FP64 and float handles, both gather forms, grids smaller than the
stencil (the gradient wraps several times), a ragged column count, and the empty cases.

Tolerance: FP64 forces agree with the FP64 oracle to 1e-10 relative (norm of the difference
over the norm of the oracle's forces).  Float handles take the gradient and the inner
products of float orbitals (24-bit significands, sums of a few thousand terms): 1e-4."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import make_hub, oracle_ham, to_dev, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F64, HUB_F32  # noqa: E402

TOL64 = 1e-10
TOL32 = 1e-4
KPT = (0.21, -0.13, 0.34)


def systems():
    return {
        "ragged": w.small_test_system(n=(20, 24, 28), ncol=37, natoms=3),
        "tiny-grid-wraps": w.small_test_system(n=(5, 7, 4), ncol=3, natoms=2, hub_rc=2.0, kb_rc=1.5),
        "odd": w.small_test_system(n=(33, 9, 17), ncol=5, natoms=4, seed=3),
        "bloch": w.small_test_system(n=(12, 10, 14), ncol=6, natoms=3, kpt=KPT),
    }


def _hermitian_D(wl, cplx, seed=5):
    """The workload's D, with a small antisymmetric imaginary part at a Bloch wavevector so
    that the index order of D in the force matters."""
    D = wl.D0[0].astype(np.complex128 if cplx else np.float64)
    if cplx:
        rng = np.random.default_rng(seed)
        A = rng.uniform(-0.03, 0.03, D.shape)
        D = D + 1j * (A - np.swapaxes(A, -1, -2))
    return D


def _case(name, prec, gather_form=-1):
    wl = systems()[name]
    cplx = name == "bloch"
    X = wl.orbitals(complex_=cplx)
    if prec != HUB_F64:
        X = X.astype(np.complex64 if cplx else np.float32).astype(np.complex128 if cplx else np.float64)
    f = np.linspace(1.0, 0.1, X.shape[0])
    D = _hermitian_D(wl, cplx)
    H = oracle_ham(wl, D=D)
    ref_hub = o.hubbard_forces(H, X.T, f, 0.7)
    hub_atoms = [i for i, a in enumerate(wl.atoms) if a.hub_l >= 0]
    ref = np.zeros((len(wl.atoms), 3))
    ref[hub_atoms] = ref_hub
    hb = make_hub(wl, prec)
    if gather_form >= 0:
        hb.set_tuning(gather_form=gather_form)
    hb.set_occupation_matrix(0, D)
    F = hb.hubbard_forces(0, to_dev(X, hb.dtype), f, 0.7)
    return F, ref


@pytest.mark.parametrize("name", list(systems()))
def test_hubbard_forces_fp64(name):
    F, ref = _case(name, HUB_F64)
    err = rel(F, ref)
    print(name, "max |F|", np.max(np.abs(ref)), "rel err", err)
    assert np.max(np.abs(ref)) > 0
    assert err < TOL64


@pytest.mark.parametrize("name", ["ragged", "bloch", "odd"])
def test_hubbard_forces_float(name):
    F, ref = _case(name, HUB_F32)
    err = rel(F, ref)
    print(name, "rel err", err)
    assert err < TOL32


def test_hubbard_forces_float_brick_gather():
    # real float with the gather in the brick form
    F, ref = _case("ragged", HUB_F32, gather_form=1)
    assert rel(F, ref) < TOL32


def test_forces_sum_over_calls_and_caller_workspace():
    # two column halves sum to the whole; a caller-owned gradient buffer gives the same result
    wl = systems()["ragged"]
    X = wl.orbitals()
    f = np.linspace(1.0, 0.1, X.shape[0])
    hb = make_hub(wl, HUB_F64)
    hb.set_occupation_matrix(0, wl.D0[0])
    Xd = to_dev(X, hb.dtype)
    F = hb.hubbard_forces(0, Xd, f, 1.0)
    Fa = hb.hubbard_forces(0, Xd[:20].contiguous(), f[:20], 1.0)
    Fb = hb.hubbard_forces(0, Xd[20:].contiguous(), f[20:], 1.0)
    assert rel(Fa + Fb, F) < 1e-12
    work = torch.empty_like(Xd)
    assert rel(hb.hubbard_forces(0, Xd, f, 1.0, work=work), F) < 1e-15


def test_forces_empty_cases():
    wl = systems()["odd"]
    hb = make_hub(wl, HUB_F64)
    Xd = to_dev(wl.orbitals(), hb.dtype)
    F = hb.hubbard_forces(0, Xd[:0], np.zeros(0), 1.0)
    assert F.shape == (len(wl.atoms), 3) and not np.any(F)
    # atoms without Hubbard shells only: no force
    atoms = [w.Atom(a.species, a.pos, kb_l=a.kb_l, kb_rs=a.kb_rs, kb_gamma=a.kb_gamma, kb_rc=a.kb_rc)
             for a in wl.atoms]
    hb.set_atoms(atoms)
    F = hb.hubbard_forces(0, Xd, np.ones(Xd.shape[0]), 1.0)
    assert not np.any(F)
