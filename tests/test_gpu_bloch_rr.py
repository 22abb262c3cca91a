"""Rayleigh-Ritz of complex Bloch blocks (CheFSI, Sec. II.B, at k != 0) through the C ABI
against the CPU oracle: the Hermitian block product <A|B>, the Cholesky Rayleigh-Ritz
projection with a complex Hermitian occupation matrix in H, and CheFSI iterations whose Ritz
values reach the lowest eigenvalues of the dense Bloch Hamiltonian (a spectrum with
degenerate pairs, so the complex Jacobi solver meets degenerate clusters).

Comparisons are element by element: a block's error is the largest elementwise difference
over the RMS magnitude of the reference orbital (or row) it belongs to.  FP64: 1e-10 (the
FP64 tolerance of the method); float: the bound stated at each test."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import make_hub, oracle_ham, to_dev, rel, rel_elem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F32, HUB_F64, HUB_MIXED_BF16  # noqa: E402

TOL64 = 1e-10
KPT = (0.21, -0.13, 0.34)


def _hermitian_D(nhub, seed):
    """A seeded complex Hermitian occupation matrix per Hubbard atom (entries ~0.1)."""
    rng = np.random.default_rng(seed)
    D = np.empty((nhub, 5, 5), dtype=np.complex128)
    for i in range(nhub):
        A = 0.05 * rng.standard_normal((5, 5)) + 0.05j * rng.standard_normal((5, 5))
        D[i] = 0.2 * np.eye(5) + A + A.conj().T
    return D


def _system(ncol=24, seed=7):
    return w.small_test_system(n=(12, 10, 14), ncol=ncol, natoms=3, kpt=KPT, seed=seed)


@pytest.mark.parametrize("prec,tol", [(HUB_F64, TOL64), (HUB_F32, 2e-6)])
def test_bloch_gram_block_product(prec, tol):
    """hub_gram on complex blocks against the oracle's grid inner product dV A^H B."""
    wl = _system()
    g = o.Grid(wl.n, wl.L, KPT)
    A = wl.orbitals(complex_=True)
    B = w.random_orbitals(wl.Nd, 17, 5, complex_=True)
    hb = make_hub(wl, prec)
    Ad, Bd = to_dev(A, hb.dtype), to_dev(B, hb.dtype)
    Ah, Bh = Ad.to(torch.complex128).cpu().numpy().T, Bd.to(torch.complex128).cpu().numpy().T
    G = torch.empty(A.shape[0], 17, dtype=torch.complex128, device="cuda")
    hb.gram(Ad, Bd, g.dV, G)
    err = rel_elem(G.cpu().numpy(), g.inner(Ah, Bh))
    print("rectangular", err)
    assert err < tol
    S = torch.empty(A.shape[0], A.shape[0], dtype=torch.complex128, device="cuda")
    hb.gram(Ad, Ad, g.dV, S)                    # Hermitian path: upper tiles mirrored
    Sh = S.cpu().numpy()
    err = rel_elem(Sh, g.inner(Ah, Ah))
    print("hermitian", err)
    assert err < tol
    # tiles off the diagonal are mirrored exactly; elements inside a diagonal tile are summed
    # separately for (i, j) and (j, i), so Hermiticity holds to rounding
    assert np.max(np.abs(Sh - Sh.conj().T)) <= tol * np.max(np.abs(Sh))


@pytest.mark.parametrize("prec", [HUB_F64, HUB_F32, HUB_MIXED_BF16])
def test_bloch_rayleigh_ritz(prec):
    """Eigenvalues, dV-orthonormality and the spectral projector sum_j lam_j x_j x_j^H (unique
    even where Ritz values are degenerate) against oracle.rayleigh_ritz, with a complex
    Hermitian D in the Hamiltonian."""
    wl = _system()
    D = _hermitian_D(len(wl.hub_atoms), 3)
    H = oracle_ham(wl, D=D)
    lo, up = o.lanczos_bounds(H, wl.lanczos_start(complex_=True), 10)
    Y = o.chebyshev_filter(H, wl.orbitals(complex_=True).T, 10, lo + 0.1 * (up - lo), up, lo)
    lam_ref, X_ref = o.rayleigh_ritz(H, Y)
    hb = make_hub(wl, prec)
    hb.set_occupation_matrix(0, D)
    Xd = to_dev(Y.T, hb.dtype)
    lam = hb.rayleigh_ritz(0, Xd)
    X = Xd.to(torch.complex128).cpu().numpy().T
    g = H.grid
    Pr = X_ref @ np.diag(lam_ref) @ X_ref.conj().T * g.dV
    P = X @ np.diag(lam) @ X.conj().T * g.dV
    e_lam = np.max(np.abs(lam - lam_ref)) / np.max(np.abs(lam_ref))
    e_orth = np.max(np.abs(g.dV * X.conj().T @ X - np.eye(X.shape[1])))
    e_P = rel_elem(P, Pr)
    print(prec, "eig", e_lam, "orth", e_orth, "projector", e_P)
    if prec == HUB_F64:
        assert e_lam < TOL64 and e_orth < 1e-10 and e_P < TOL64
    else:
        # float block products: ~1e-7 relative rounding of the Gram and projected-H entries,
        # amplified by the condition number of the filtered block (its Gram matrix spans
        # ~1e3 here) in the Cholesky factor
        assert e_lam < 1e-5 and e_orth < 1e-4 and e_P < 1e-4


def test_bloch_chefsi_reaches_the_dense_spectrum():
    """CheFSI (filter + Rayleigh-Ritz) on a tiny Bloch grid: the Ritz values converge to the
    lowest eigenvalues of the dense Hamiltonian built by the oracle (numpy eigh), and never
    fall below them (Cauchy interlacing)."""
    wl = w.small_test_system(n=(8, 8, 8), ncol=10, natoms=1, kpt=(0.3, 0.0, 0.0), seed=5)
    D = _hermitian_D(len(wl.hub_atoms), 9)
    H = oracle_ham(wl, D=D)
    Nd = wl.Nd
    Hd = H.apply(np.eye(Nd, dtype=np.complex128))
    ev = np.linalg.eigvalsh(0.5 * (Hd + Hd.conj().T))
    hb = make_hub(wl, HUB_F64)
    hb.set_occupation_matrix(0, D)
    v0 = wl.lanczos_start(complex_=True)
    lo, up = hb.lanczos_bound(0, 10, to_dev(v0, torch.complex128))
    Xd = to_dev(wl.orbitals(complex_=True), torch.complex128)
    a_low, a, b = lo, lo + 0.1 * (up - lo), up
    for _ in range(40):
        hb.chefsi_filter(0, Xd, 12, a, b, a_low)
        lam = hb.rayleigh_ritz(0, Xd)
        a_low, a = lam[0], lam[-1]
    nconv = 6           # the top Ritz values of a block converge last
    print("Ritz", lam[:nconv], "dense", ev[:nconv])
    assert np.all(lam >= ev[:len(lam)] - 1e-10)
    assert np.max(np.abs(lam[:nconv] - ev[:nconv])) < 1e-9 * np.max(np.abs(ev))
