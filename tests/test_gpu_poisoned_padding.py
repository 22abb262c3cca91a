"""Poisoned padding: blocks with a leading dimension larger than the grid carry NaN in the
rows past Nd; no kernel may read them.  H application, the filter, Rayleigh-Ritz, the
occupation matrices, the forces and the Gram products must match the unpadded results (and
leave the padding of their outputs as it was).

Marked gpu_pending: this test has not run on a GPU yet; the marker moves to gpu after its
first GPU run."""
import numpy as np
import pytest

import workloads as w
from hubtest import make_hub, to_dev, rel

pytestmark = pytest.mark.gpu_pending
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F32, HUB_F64, HUB_MIXED_BF16  # noqa: E402

PAD = 37


def _padded(X, dtype, fill=float("nan")):
    ld = X.shape[1] + PAD
    Xp = np.full((X.shape[0], ld), fill)
    Xp[:, :X.shape[1]] = X
    return to_dev(Xp, dtype)


@pytest.mark.parametrize("prec", [HUB_F64, HUB_F32, HUB_MIXED_BF16])
def test_nan_padding_is_never_read(prec):
    wl = w.small_test_system(n=(20, 24, 28), ncol=12, natoms=3)
    X = wl.orbitals()
    f = np.linspace(1.0, 0.2, X.shape[0])
    runs = []
    for pad in (False, True):
        hb = make_hub(wl, prec)
        hb.set_occupation_matrix(0, wl.D0[0])
        Xd = _padded(X, hb.dtype) if pad else to_dev(X, hb.dtype)
        Yd = torch.full_like(Xd, 3.0)
        hb.apply_H(0, Xd, Yd)
        y = Yd[:, :wl.Nd].cpu().numpy().copy()
        if pad:
            assert torch.all(Yd[:, wl.Nd:] == 3.0)
        hb.chefsi_filter(0, Xd, 8, a=-0.5, b=40.0, a_low=-3.0)
        eig = hb.rayleigh_ritz(0, Xd)
        Dr, _, eu = hb.occupation(0, Xd, f, 1.0)
        F = hb.hubbard_forces(0, Xd, f, 1.0)
        if pad:
            assert torch.isnan(Xd[:, wl.Nd:]).all()        # the padding stayed as it was
        runs.append((y, eig, Dr, eu, F, Xd[:, :wl.Nd].cpu().numpy()))
    (y0, e0, D0, u0, F0, X0), (y1, e1, D1, u1, F1, X1) = runs
    for a in (y1, e1, D1, F1, X1):
        assert np.all(np.isfinite(a))
    # identical inputs through the same kernels: equal up to reduction order
    tol = 1e-12 if prec == HUB_F64 else 1e-5
    assert rel(y1, y0) < tol and rel(e1, e0) < tol and rel(D1, D0) < tol and rel(F1, F0) < max(tol, 1e-9)
    assert abs(u1 - u0) < tol * max(1.0, abs(u0))
