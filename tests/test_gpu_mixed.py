"""The mixed-precision forms (HUB_MIXED_BF16, HUB_MIXED_F16): 16-bit tensor-core block
products (tcgen05, FP32 accumulation) against the FP64 oracle.  Tolerances follow from the
operand rounding: one BF16 product rounds each operand to 8 significand bits (relative error
<= 2^-9 per factor, ~3e-3 on a product of sums with cancellation-free diagonals); the hi/lo
split keeps ~16 bits (2^-17 ~ 8e-6 per factor) plus float accumulation over the grid.  FP16
keeps 11 bits in one product (each product within 2^-11 of |a_i b_i|, so the sum within
2^-11 |a||b| ~ 4.9e-4) and ~22 in the split, where the float accumulation over the grid
(~sqrt(K) 2^-24 of |a||b|) dominates."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import make_hub, oracle_ham, to_dev, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_MIXED_BF16, HUB_MIXED_F16  # noqa: E402


@pytest.mark.parametrize("prec,terms,tol", [(HUB_MIXED_BF16, 1, 1e-2), (HUB_MIXED_BF16, 3, 5e-5),
                                            (HUB_MIXED_F16, 1, 5e-4), (HUB_MIXED_F16, 3, 1e-5)])
@pytest.mark.parametrize("shape", [(37, 29), (130, 257)])
def test_tensor_core_block_product(prec, terms, tol, shape):
    wl = w.small_test_system(n=(20, 24, 28), ncol=8, natoms=1)
    g = o.Grid(wl.n, wl.L)
    na, nb = shape
    A = w.random_orbitals(wl.Nd, na, 5).astype(np.float32)
    B = w.random_orbitals(wl.Nd, nb, 6).astype(np.float32)
    hb = make_hub(wl, prec)
    hb.set_bf16_terms(terms)
    Ad, Bd = to_dev(A, torch.float32), to_dev(B, torch.float32)
    G = torch.empty(na, nb, dtype=torch.float64, device="cuda")
    hb.gram(Ad, Bd, g.dV, G)
    ref = g.inner(A.astype(np.float64).T, B.astype(np.float64).T)
    # random blocks: |G| is dominated by cancellation, so scale by the norms of the factors
    scale = g.dV * np.linalg.norm(A, axis=1)[:, None] * np.linalg.norm(B, axis=1)[None, :]
    err = np.max(np.abs(G.cpu().numpy() - ref) / scale)
    print(prec, terms, shape, "max error / (|a||b| dV)", err)
    assert err < tol
    # symmetric call A^T A
    S = torch.empty(na, na, dtype=torch.float64, device="cuda")
    hb.gram(Ad, Ad, g.dV, S)
    refS = g.inner(A.astype(np.float64).T, A.astype(np.float64).T)
    assert rel(S.cpu().numpy(), refS) < tol


@pytest.mark.parametrize("prec,terms,tol", [(HUB_MIXED_BF16, 1, 3e-3), (HUB_MIXED_BF16, 3, 2e-5),
                                            (HUB_MIXED_F16, 1, 5e-4), (HUB_MIXED_F16, 3, 2e-5)])
def test_mixed_rayleigh_ritz_eigenvalues(prec, terms, tol):
    wl = w.small_test_system(n=(20, 24, 28), ncol=37, natoms=3)
    H = oracle_ham(wl, D=wl.D0[0])
    lo, up = o.lanczos_bounds(H, wl.lanczos_start(), 10)
    Y = o.chebyshev_filter(H, wl.orbitals().T, 10, lo + 0.1 * (up - lo), up, lo)
    Y = Y / np.linalg.norm(Y, axis=0)
    lam_ref, _ = o.rayleigh_ritz(H, Y.astype(np.float32).astype(np.float64))
    hb = make_hub(wl, prec)
    hb.set_bf16_terms(terms)
    hb.set_occupation_matrix(0, wl.D0[0])
    Xd = to_dev(Y.T, torch.float32)
    lam = hb.rayleigh_ritz(0, Xd)
    err = np.max(np.abs(lam - lam_ref)) / np.max(np.abs(lam_ref))
    print(prec, "terms", terms, "max rel eigenvalue error", err)
    assert err < tol
    X = Xd.double().cpu().numpy().T
    ortho = np.max(np.abs(wl.dV * X.T @ X - np.eye(X.shape[1])))
    print("orthonormality", ortho)
    assert ortho < (3e-2 if terms == 1 else 1e-4)


@pytest.mark.parametrize("terms,tol", [(1, 5e-4), (3, 1e-5)])
def test_f16_operand_scaling_covers_any_magnitude(terms, tol):
    """FP16 overflows above 65504 and loses bits below 2^-14: blocks far outside that range
    (|A| ~ 1e-7, |B| ~ 1e6) must still give the product to the FP16 tolerance, and the
    rotation X Q must come back at its own scale."""
    wl = w.small_test_system(n=(20, 24, 28), ncol=8, natoms=1)
    g = o.Grid(wl.n, wl.L)
    A = (3e-7 * w.random_orbitals(wl.Nd, 33, 7)).astype(np.float32)
    B = (2e5 * w.random_orbitals(wl.Nd, 40, 8)).astype(np.float32)
    hb = make_hub(wl, HUB_MIXED_F16)
    hb.set_bf16_terms(terms)
    G = torch.empty(33, 40, dtype=torch.float64, device="cuda")
    hb.gram(to_dev(A, torch.float32), to_dev(B, torch.float32), g.dV, G)
    ref = g.inner(A.astype(np.float64).T, B.astype(np.float64).T)
    scale = g.dV * np.linalg.norm(A, axis=1)[:, None] * np.linalg.norm(B, axis=1)[None, :]
    err = np.max(np.abs(G.cpu().numpy() - ref) / scale)
    print("scaled blocks: max error / (|a||b| dV)", err)
    assert np.all(np.isfinite(G.cpu().numpy())) and err < tol
    # Rayleigh-Ritz of a block scaled by 1e-6: S ~ 1e-12, so the rotation X L^-T V multiplies
    # a tiny X by a large Q; eigenvalues and orthonormality must match the unscaled block's
    H = oracle_ham(wl, D=wl.D0[0])
    lo, up = o.lanczos_bounds(H, wl.lanczos_start(), 10)
    Y0 = o.chebyshev_filter(H, wl.orbitals().T, 10, lo + 0.1 * (up - lo), up, lo)
    Y0 = (Y0 / np.linalg.norm(Y0, axis=0)).T.astype(np.float32)
    hb.set_occupation_matrix(0, wl.D0[0])
    lam = {}
    for f in (1.0, 1e-6):
        Xd = to_dev(np.float32(f) * Y0, torch.float32)
        lam[f] = hb.rayleigh_ritz(0, Xd)
        X = Xd.double().cpu().numpy().T
        ortho = np.max(np.abs(wl.dV * X.T @ X - np.eye(X.shape[1])))
        print("block scale", f, "orthonormality", ortho)
        assert ortho < (3e-2 if terms == 1 else 1e-4)
    err = np.max(np.abs(lam[1e-6] - lam[1.0])) / np.max(np.abs(lam[1.0]))
    print("Ritz values of the scaled block against the unscaled one", err)
    assert err < (5e-4 if terms == 1 else 2e-5)
