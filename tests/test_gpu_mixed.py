"""The mixed-precision form (HUB_MIXED_BF16): BF16 tensor-core block products (tcgen05,
FP32 accumulation) against the FP64 oracle.  Tolerances follow from the operand rounding:
one BF16 product rounds each operand to 8 significand bits (relative error <= 2^-9 per
factor, ~3e-3 on a product of sums with cancellation-free diagonals); the hi/lo split keeps
~16 bits (2^-17 ~ 8e-6 per factor) plus float accumulation over the grid."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import make_hub, oracle_ham, to_dev, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_MIXED_BF16  # noqa: E402


@pytest.mark.parametrize("terms,tol", [(1, 1e-2), (3, 5e-5)])
@pytest.mark.parametrize("shape", [(37, 29), (130, 257)])
def test_tensor_core_block_product(terms, tol, shape):
    wl = w.small_test_system(n=(20, 24, 28), ncol=8, natoms=1)
    g = o.Grid(wl.n, wl.L)
    na, nb = shape
    A = w.random_orbitals(wl.Nd, na, 5).astype(np.float32)
    B = w.random_orbitals(wl.Nd, nb, 6).astype(np.float32)
    hb = make_hub(wl, HUB_MIXED_BF16)
    hb.set_bf16_terms(terms)
    Ad, Bd = to_dev(A, torch.float32), to_dev(B, torch.float32)
    G = torch.empty(na, nb, dtype=torch.float64, device="cuda")
    hb.gram(Ad, Bd, g.dV, G)
    ref = g.inner(A.astype(np.float64).T, B.astype(np.float64).T)
    # random blocks: |G| is dominated by cancellation, so scale by the norms of the factors
    scale = g.dV * np.linalg.norm(A, axis=1)[:, None] * np.linalg.norm(B, axis=1)[None, :]
    err = np.max(np.abs(G.cpu().numpy() - ref) / scale)
    print(terms, shape, "max error / (|a||b| dV)", err)
    assert err < tol
    # symmetric call A^T A
    S = torch.empty(na, na, dtype=torch.float64, device="cuda")
    hb.gram(Ad, Ad, g.dV, S)
    refS = g.inner(A.astype(np.float64).T, A.astype(np.float64).T)
    assert rel(S.cpu().numpy(), refS) < tol


@pytest.mark.parametrize("terms,tol", [(1, 3e-3), (3, 2e-5)])
def test_mixed_rayleigh_ritz_eigenvalues(terms, tol):
    wl = w.small_test_system(n=(20, 24, 28), ncol=37, natoms=3)
    H = oracle_ham(wl, D=wl.D0[0])
    lo, up = o.lanczos_bounds(H, wl.lanczos_start(), 10)
    Y = o.chebyshev_filter(H, wl.orbitals().T, 10, lo + 0.1 * (up - lo), up, lo)
    Y = Y / np.linalg.norm(Y, axis=0)
    lam_ref, _ = o.rayleigh_ritz(H, Y.astype(np.float32).astype(np.float64))
    hb = make_hub(wl, HUB_MIXED_BF16)
    hb.set_bf16_terms(terms)
    hb.set_occupation_matrix(0, wl.D0[0])
    Xd = to_dev(Y.T, torch.float32)
    lam = hb.rayleigh_ritz(0, Xd)
    err = np.max(np.abs(lam - lam_ref)) / np.max(np.abs(lam_ref))
    print("terms", terms, "max rel eigenvalue error", err)
    assert err < tol
    X = Xd.double().cpu().numpy().T
    ortho = np.max(np.abs(wl.dV * X.T @ X - np.eye(X.shape[1])))
    print("orthonormality", ortho)
    assert ortho < (3e-2 if terms == 1 else 1e-4)
