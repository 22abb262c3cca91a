"""Poisoned padding: blocks with a leading dimension larger than the grid carry NaN in the
rows past Nd; no kernel may read them.  H application, the filter, Rayleigh-Ritz, the
occupation matrices, the forces and the Gram products must match the unpadded results (and
leave the padding of their outputs as it was).

Tolerances: FP64 1e-12 relative (the same kernels on the same values, up to reduction
order).  Float handles: H X and the Ritz values 1e-5 relative; D, E_U and the forces by an
absolute bound, because the padded and unpadded launches may take kernel forms of different
vector width (the padded ld is odd) whose rounding differs, and D of a filtered block is a
sum of products of coefficients far smaller than the float unit in the last place of the
terms they cancel from.  With dV-orthonormal orbitals and normalised Hubbard orbitals every
coefficient |c| <= 1, so each D entry (and each force component, up to the gradient norm
of the orbitals, below 2 bohr^-1 here) is bounded by sum_n f_n, and float rounding of the
coefficients (~1e-7 each) moves it by less than 1e-6 sum_n f_n."""
import numpy as np
import pytest

import workloads as w
from hubtest import make_hub, to_dev, rel

pytestmark = pytest.mark.gpu
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
        G = torch.empty((X.shape[0], X.shape[0]), dtype=torch.float64, device=Xd.device)
        hb.gram(Xd, Yd, 1.0, G)
        g = G.cpu().numpy()
        hb.chefsi_filter(0, Xd, 8, a=-0.5, b=40.0, a_low=-3.0)
        eig = hb.rayleigh_ritz(0, Xd)
        Dr, _, eu = hb.occupation(0, Xd, f, 1.0)
        F = hb.hubbard_forces(0, Xd, f, 1.0)
        if pad:
            assert torch.isnan(Xd[:, wl.Nd:]).all()        # the padding stayed as it was
        runs.append((y, eig, Dr, eu, F, Xd[:, :wl.Nd].cpu().numpy(), g))
    (y0, e0, D0, u0, F0, X0, g0), (y1, e1, D1, u1, F1, X1, g1) = runs
    for a in (y1, e1, D1, F1, X1, g1):
        assert np.all(np.isfinite(a))
    # identical inputs through the same kernels: equal up to reduction order
    if prec == HUB_F64:
        tol = 1e-12
        assert rel(y1, y0) < tol and rel(e1, e0) < tol and rel(D1, D0) < tol and rel(F1, F0) < 1e-9
        assert abs(u1 - u0) < tol * max(1.0, abs(u0))
        assert rel(g1, g0) < tol
    else:
        assert rel(y1, y0) < 1e-5 and rel(e1, e0) < 1e-5 and rel(g1, g0) < 1e-5
        bound = 1e-6 * float(np.sum(f))
        assert np.max(np.abs(D1 - D0)) < bound
        assert np.max(np.abs(F1 - F0)) < 2.0 * bound
        assert abs(u1 - u0) < bound
