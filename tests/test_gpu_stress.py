"""Parity of the Hubbard stress tensor (Sec. II.A.4) through the C ABI with the CPU oracle:
real and Bloch orbitals, FP64 and float handles, a cell small enough that periodic images
of one atom overlap, and the sum over blocks.

Marked gpu_pending: this code has not run on a GPU yet; the marker moves to gpu after its
first GPU run.  Tolerance: FP64 1e-10 relative (norm of the difference over the norm of the
oracle's tensor); float handles 1e-4 (float gradient and products)."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import make_hub, oracle_ham, to_dev, rel

pytestmark = pytest.mark.gpu_pending
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
