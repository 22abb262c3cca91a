"""Parity of the CUDA library (through the C ABI) with the CPU oracle, element by element,
on seeded synthetic inputs: H application, Chebyshev filter, Lanczos bounds, Rayleigh-Ritz,
occupation matrices and E_U, and one full filter + Rayleigh-Ritz pass of the 24^3 tiny cell.

Comparisons are element by element: the largest elementwise difference over the RMS
magnitude of the reference row it belongs to (one orbital of a block, one row of a matrix,
a whole vector of eigenvalues), so one wrong element at a tile edge stands out against its
own orbital's scale.  Tolerance: FP64 results agree with the FP64 oracle to 1e-10; float
results to the float bound stated at each test."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import make_hub, oracle_ham, to_dev, rel_elem as rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F64, HUB_F32, HubError  # noqa: E402

TOL64 = 1e-10


def systems():
    return {
        "ragged": w.small_test_system(n=(20, 24, 28), ncol=37, natoms=3),
        "tiny-grid-wraps": w.small_test_system(n=(5, 7, 4), ncol=3, natoms=2, hub_rc=2.0, kb_rc=1.5),
        "odd": w.small_test_system(n=(33, 9, 17), ncol=5, natoms=4, seed=3),
        "bloch": w.small_test_system(n=(12, 10, 14), ncol=6, natoms=3, kpt=(0.21, -0.13, 0.34)),
    }


@pytest.mark.parametrize("name", list(systems()))
def test_apply_H_fp64(name):
    wl = systems()[name]
    cplx = name == "bloch"
    X = wl.orbitals(complex_=cplx)
    H = oracle_ham(wl, D=wl.D0[0])
    ref = H.apply(X.T).T
    hb = make_hub(wl, HUB_F64)
    hb.set_occupation_matrix(0, wl.D0[0])
    Xd = to_dev(X, hb.dtype)
    Yd = torch.empty_like(Xd)
    hb.apply_H(0, Xd, Yd)
    err = rel(Yd.cpu().numpy(), ref)
    print(name, "rel err", err)
    assert err < TOL64


def test_apply_H_padded_leading_dimension_and_spin_channels():
    wl = w.small_test_system(n=(16, 12, 10), ncol=4, natoms=2, nspin=2)
    hb = make_hub(wl, HUB_F64)
    for s in range(2):
        hb.set_occupation_matrix(s, wl.D0[s])
    X = wl.orbitals()
    ld = wl.Nd + 37
    Xp = np.zeros((4, ld))
    Xp[:, :wl.Nd] = X
    Xd = to_dev(Xp, torch.float64)
    Yd = torch.full_like(Xd, 7.0)
    for s in range(2):
        hb.apply_H(s, Xd, Yd)
        ref = oracle_ham(wl, D=wl.D0[s]).apply(X.T).T
        assert rel(Yd[:, :wl.Nd].cpu().numpy(), ref) < TOL64
        assert torch.all(Yd[:, wl.Nd:] == 7.0)            # padding untouched


@pytest.mark.parametrize("prec", [HUB_F32, HUB_F64])
def test_apply_H_every_stencil_variant(prec):
    """Every tile shape the autotuner may choose, on a ragged grid with chunked z, on a grid
    thinner in z than the stencil's half-width (each plane wraps several times), and on a
    grid with an odd number of y-rows (the last row pair of the two-row float tiles has one
    row outside the cell)."""
    cases = [systems()["ragged"],
             w.small_test_system(n=(8, 12, 3), ncol=5, natoms=2, hub_rc=2.0, kb_rc=1.5, seed=5),
             w.small_test_system(n=(12, 9, 10), ncol=6, natoms=2, hub_rc=2.0, kb_rc=1.5, seed=6),
             # a ragged second x-tile (8 columns), ragged y-tiles of 14 and 6 rows, z thinner
             # than the queue
             w.small_test_system(n=(40, 30, 12), ncol=5, natoms=2, hub_rc=2.5, kb_rc=1.5, seed=8)]
    # Bloch (complex) blocks: a ragged grid, and one thinner in z than the half-width with
    # wraps on every face (the halo and queue planes carry their Bloch factors)
    cases += [w.small_test_system(n=(12, 10, 14), ncol=6, natoms=3, kpt=(0.21, -0.13, 0.34)),
              w.small_test_system(n=(8, 12, 3), ncol=5, natoms=2, hub_rc=2.0, kb_rc=1.5, seed=5,
                                  kpt=(0.31, 0.17, -0.45))]
    for wl in cases:
        cplx = bool(np.any(np.asarray(wl.kpts[0]) != 0))
        X = wl.orbitals(complex_=cplx)
        ref = oracle_ham(wl, D=wl.D0[0]).apply(X.T).T
        hb = make_hub(wl, prec)
        hb.set_occupation_matrix(0, wl.D0[0])
        Xd = to_dev(X, hb.dtype)
        for v in range(hb.get_tuning()["n_variants"]):
            hb.set_tuning(v)
            Yd = torch.empty_like(Xd)
            hb.apply_H(0, Xd, Yd)
            err = rel(Yd.cpu().numpy().astype(np.complex128 if cplx else np.float64), ref)
            assert err < (5e-6 if prec == HUB_F32 else TOL64), (wl.name, v, err)
        with pytest.raises(HubError):
            hb.set_tuning(hb.get_tuning()["n_variants"])


@pytest.mark.parametrize("n,natoms", [((12, 10, 9), 3), ((16, 16, 16), 12)])
def test_apply_H_fp32_brick_edges_and_crowded_bricks(n, natoms):
    """Real float blocks use the 8x8x4 brick form of the projectors: a grid that ends inside
    bricks in x, y and z, and a cell so crowded that bricks carry more than 64 functions
    (several entries per brick)."""
    wl = w.small_test_system(n=n, ncol=19, natoms=natoms, seed=21, hub_rc=2.5, kb_rc=2.5)
    X = wl.orbitals()
    ref = oracle_ham(wl, D=wl.D0[0]).apply(X.T).T
    hb = make_hub(wl, HUB_F32)
    hb.set_occupation_matrix(0, wl.D0[0])
    Xd = to_dev(X, torch.float32)
    for form in (0, 1):                     # point-major and brick-form gather
        hb.set_tuning(gather_form=form)
        Yd = torch.empty_like(Xd)
        hb.apply_H(0, Xd, Yd)
        err = rel(Yd.cpu().numpy().astype(np.float64), ref)
        print(n, natoms, form, "fp32 rel err", err)
        assert err < 5e-6


@pytest.mark.parametrize("name", ["ragged", "bloch"])
def test_apply_H_fp32(name):
    wl = systems()[name]
    cplx = name == "bloch"
    X = wl.orbitals(complex_=cplx)
    ref = oracle_ham(wl, D=wl.D0[0]).apply(X.T).T
    hb = make_hub(wl, HUB_F32)
    hb.set_occupation_matrix(0, wl.D0[0])
    Xd = to_dev(X, hb.dtype)
    Yd = torch.empty_like(Xd)
    hb.apply_H(0, Xd, Yd)
    err = rel(Yd.cpu().numpy().astype(np.complex128 if cplx else np.float64), ref)
    print(name, "fp32 rel err", err)
    # float rounding of inputs and weights: ~1e-7 relative per term, stencil sums of ~40 terms
    assert err < 5e-6


@pytest.mark.parametrize("name,degree", [("ragged", 8), ("bloch", 7), ("tiny-grid-wraps", 5)])
def test_chebyshev_filter_fp64(name, degree):
    wl = systems()[name]
    cplx = name == "bloch"
    H = oracle_ham(wl, D=wl.D0[0])
    lo, up = o.lanczos_bounds(H, wl.lanczos_start(complex_=cplx), 10)
    a_low, a, b = lo, lo + 0.1 * (up - lo), up
    X = wl.orbitals(complex_=cplx)
    ref = o.chebyshev_filter(H, X.T, degree, a, b, a_low).T
    hb = make_hub(wl, HUB_F64)
    hb.set_occupation_matrix(0, wl.D0[0])
    Xd = to_dev(X, hb.dtype)
    hb.chefsi_filter(0, Xd, degree, a, b, a_low)
    err = rel(Xd.cpu().numpy(), ref)
    print(name, "filter rel err", err)
    assert err < TOL64
    # user-provided work buffer gives the same result
    Xd2 = to_dev(X, hb.dtype)
    work = torch.empty_like(Xd2)
    hb.chefsi_filter(0, Xd2, degree, a, b, a_low, work=work)
    assert rel(Xd2.cpu().numpy(), ref) < TOL64


def test_lanczos_bounds_fp64():
    wl = systems()["ragged"]
    H = oracle_ham(wl, D=wl.D0[0])
    v0 = wl.lanczos_start()
    lo, up = o.lanczos_bounds(H, v0, 12)
    hb = make_hub(wl, HUB_F64)
    hb.set_occupation_matrix(0, wl.D0[0])
    glo, gup = hb.lanczos_bound(0, 12, to_dev(v0, torch.float64))
    assert abs(glo - lo) < 1e-9 * max(1.0, abs(lo))
    assert abs(gup - up) < 1e-9 * abs(up)


def test_rayleigh_ritz_fp64():
    wl = systems()["ragged"]
    H = oracle_ham(wl, D=wl.D0[0])
    lo, up = o.lanczos_bounds(H, wl.lanczos_start(), 10)
    Y = o.chebyshev_filter(H, wl.orbitals().T, 10, lo + 0.1 * (up - lo), up, lo)   # input block
    lam_ref, X_ref = o.rayleigh_ritz(H, Y)
    hb = make_hub(wl, HUB_F64)
    hb.set_occupation_matrix(0, wl.D0[0])
    Xd = to_dev(Y.T, torch.float64)
    lam = hb.rayleigh_ritz(0, Xd)
    assert rel(lam, lam_ref) < TOL64
    X = Xd.cpu().numpy().T
    g = H.grid
    np.testing.assert_allclose(g.dV * X.T @ X, np.eye(X.shape[1]), atol=1e-10)
    # Ritz vectors are unique up to sign where the Ritz values are simple: compare the
    # spectral projector sum_j lam_j x_j x_j^T, which is unique in any case
    P = X @ np.diag(lam) @ X.T * g.dV
    P_ref = X_ref @ np.diag(lam_ref) @ X_ref.T * g.dV
    assert rel(P, P_ref) < TOL64


def test_rayleigh_ritz_rejects_rank_deficient_block():
    wl = systems()["odd"]
    hb = make_hub(wl, HUB_F64)
    X = wl.orbitals()
    X[1] = X[0]
    with pytest.raises(HubError) as e:
        hb.rayleigh_ritz(0, to_dev(X, torch.float64))
    assert e.value.code == -4                 # HUB_ENOTSPD
    # the handle stays usable afterwards
    X2 = wl.orbitals()
    lam = hb.rayleigh_ritz(0, to_dev(X2, torch.float64))
    assert np.all(np.isfinite(lam))


@pytest.mark.parametrize("name", ["ragged", "bloch"])
def test_occupation_matrices_and_EU_fp64(name):
    wl = systems()[name]
    cplx = name == "bloch"
    H = oracle_ham(wl)
    X = wl.orbitals(complex_=cplx) * 0.05
    f = np.linspace(1.0, 0.1, X.shape[0])
    D_ref = o.occupation_matrices(H, X.T, f, 0.7)
    U = [h[2] for h in H.hub]
    hb = make_hub(wl, HUB_F64)
    Dr, Di, eu = hb.occupation(0, to_dev(X, hb.dtype), f, 0.7)
    D = Dr + 1j * Di if cplx else Dr
    assert rel(D, D_ref) < TOL64
    eu_ref = o.hubbard_energy(np.real(D_ref) if not cplx else D_ref, U)
    assert abs(eu - eu_ref) < 1e-10 * max(1.0, abs(eu_ref))


def test_bad_arguments_are_rejected():
    wl = systems()["odd"]
    hb = make_hub(wl, HUB_F64)
    Xd = to_dev(wl.orbitals(), torch.float64)
    with pytest.raises(HubError) as e:
        hb.chefsi_filter(0, Xd, 5, a=1.0, b=0.5, a_low=-1.0)      # a > b
    assert e.value.code == -1
    with pytest.raises(HubError):
        hb.chefsi_filter(0, Xd, 0, a=1.0, b=2.0, a_low=0.0)      # degree 0
    with pytest.raises(HubError):
        hb.apply_H(2, Xd, torch.empty_like(Xd))                   # spin 2
    # ncol = 0 is a no-op
    hb.apply_H(0, Xd[:0], torch.empty_like(Xd[:0]))


def test_tiny_cell_one_pass():
    """The 24^3 tiny cell: Lanczos bounds, degree-20 filter, Rayleigh-Ritz, D and E_U."""
    wl = w.tiny()
    H = oracle_ham(wl, D=wl.D0[0])
    v0 = wl.lanczos_start()
    lo, up = o.lanczos_bounds(H, v0, 10)
    a_low, a, b = lo, lo + 0.1 * (up - lo), up
    X0 = wl.orbitals()
    Y = o.chebyshev_filter(H, X0.T, wl.degree, a, b, a_low)
    lam_ref, X_ref = o.rayleigh_ritz(H, Y)
    f = np.zeros(wl.ncol)
    f[:16] = 1.0
    D_ref = o.occupation_matrices(H, X_ref, f)
    U = [hh[2] for hh in H.hub]
    EU_ref = 2 * o.hubbard_energy(D_ref, U)          # both spin channels

    hb = make_hub(wl, HUB_F64)
    hb.set_occupation_matrix(0, wl.D0[0])
    glo, gup = hb.lanczos_bound(0, 10, to_dev(v0, torch.float64))
    assert abs(glo - lo) < 1e-9 * max(1, abs(lo)) and abs(gup - up) < 1e-9 * abs(up)
    Xd = to_dev(X0, torch.float64)
    hb.chefsi_filter(0, Xd, wl.degree, a, b, a_low)
    assert rel(Xd.cpu().numpy(), Y.T) < TOL64
    lam = hb.rayleigh_ritz(0, Xd)
    assert rel(lam, lam_ref) < TOL64
    Dr, _, eu = hb.occupation(0, Xd, f)
    assert rel(Dr, D_ref) < TOL64
    assert abs(2 * eu - EU_ref) < 1e-10 * abs(EU_ref)


@pytest.mark.parametrize("prec,tol", [(HUB_F64, TOL64), (HUB_F32, 2e-6)])
def test_gram_block_product(prec, tol):
    """hub_gram against the oracle's grid inner product <A|B> = dV A^T B."""
    wl = w.small_test_system(n=(20, 24, 28), ncol=37, natoms=1)
    g = o.Grid(wl.n, wl.L)
    A = wl.orbitals()
    B = w.random_orbitals(wl.Nd, 29, 5)
    hb = make_hub(wl, prec)
    Ad, Bd = to_dev(A, hb.dtype), to_dev(B, hb.dtype)
    G = torch.empty(37, 29, dtype=torch.float64, device="cuda")
    hb.gram(Ad, Bd, g.dV, G)
    ref = g.inner(Ad.double().cpu().numpy().T, Bd.double().cpu().numpy().T)
    assert rel(G.cpu().numpy(), ref) < tol
    S = torch.empty(37, 37, dtype=torch.float64, device="cuda")
    hb.gram(Ad, Ad, g.dV, S)                    # symmetric path: upper tiles mirrored
    refS = g.inner(Ad.double().cpu().numpy().T, Ad.double().cpu().numpy().T)
    assert rel(S.cpu().numpy(), refS) < tol
