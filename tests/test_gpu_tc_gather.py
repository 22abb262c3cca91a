"""The projector gather and scatter as tcgen05 tensor-core products (brick form, TF32 with
both operands split hi + lo, FP32 accumulation; gather form 2 takes the tensor-core gather,
form 3 the tensor-core gather and scatter) against the oracle, through the C ABI.

The projector coefficients C = dV Phi^T X (hub_project) are compared with the oracle's own
tables element by element (the largest difference over the RMS magnitude of each function's
row of C), for every gather form of a real float handle: a ragged grid, a grid whose bricks
end inside the cell in x, y and z (n1 = 12: the last brick holds one 4-point half in x), two
tiles of 128 orbitals with a ragged last tile, and a cell so crowded that bricks carry more
than 64 functions (several entries per brick).  The scatter Y += alpha Phi W (hub_expand)
is compared with the oracle's Phi W on the same cases.  Then H X, a Chebyshev filter and
Lanczos bounds with the tensor-core gather and scatter against the oracle.

Tolerance: the three-term TF32 product carries about 21 significant bits per term and
accumulates 256 brick points in FP32 before the partial rows are summed in double, the same
order of accuracy as the float SIMT gather: 1e-5 on C (the float bound of the other
projector tests), 5e-6 on H X (the float H bound)."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import make_hub, oracle_ham, to_dev, rel_elem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F32  # noqa: E402

CASES = {
    "ragged": dict(n=(20, 24, 28), ncol=9, natoms=3, seed=7),
    "brick-edges-two-tiles": dict(n=(12, 10, 9), ncol=150, natoms=3, seed=21, hub_rc=2.5, kb_rc=2.5),
    "crowded": dict(n=(16, 16, 16), ncol=19, natoms=12, seed=21, hub_rc=2.5, kb_rc=2.5),
}


def _oracle_projectors(wl):
    """The oracle's functions as columns, in the library's row order: per atom its KB
    channels, then its Hubbard shell."""
    g = o.Grid(wl.n, wl.L, wl.kpts[0])
    cols = []
    for a in wl.atoms:
        tabs = []
        if len(a.kb_l):
            tabs.append(o.atom_function_table(g, a.pos, list(zip(a.kb_l, a.kb_rs)), a.kb_rc))
        if a.hub_l >= 0:
            tabs.append(o.atom_function_table(g, a.pos, [(a.hub_l, a.hub_rs)], a.hub_rc))
        for idx, vals in tabs:
            B = np.zeros((wl.Nd, vals.shape[1]))
            B[idx] = vals
            cols.append(B)
    return g, np.concatenate(cols, axis=1)


@pytest.mark.parametrize("name", list(CASES))
def test_projector_coefficients_every_gather_form(name):
    wl = w.small_test_system(**CASES[name])
    g, P = _oracle_projectors(wl)
    X = wl.orbitals().astype(np.float32).astype(np.float64)      # the block as the GPU holds it
    C_ref = g.dV * (P.T @ X.T)
    hb = make_hub(wl, HUB_F32)
    assert hb.num_projectors() == P.shape[1]
    Xd = to_dev(X, torch.float32)
    got = {}
    for form in (0, 1, 2, 3):
        hb.set_tuning(gather_form=form)
        got[form] = hb.project(Xd)
        err = rel_elem(got[form], C_ref)
        print(name, "form", form, "elementwise err", err)
        assert err < 1e-5, (name, form, err)
    # the tensor-core form agrees with the float brick form on CUDA cores to float rounding
    assert rel_elem(got[2], got[1]) < 1e-5
    assert rel_elem(got[3], got[2]) == 0.0      # the same gather kernel


@pytest.mark.parametrize("name", list(CASES))
def test_projector_expansion_every_scatter_form(name):
    wl = w.small_test_system(**CASES[name])
    g, P = _oracle_projectors(wl)
    rng = np.random.default_rng(4)
    Wc = rng.standard_normal((P.shape[1], wl.ncol)).astype(np.float32).astype(np.float64)
    Y0 = rng.standard_normal((wl.ncol, wl.Nd)).astype(np.float32).astype(np.float64)
    ref = Y0 + 0.5 * (P @ Wc).T
    hb = make_hub(wl, HUB_F32)
    for form in (1, 3):                  # the brick scatter on CUDA cores and on tensor cores
        hb.set_tuning(gather_form=form)
        Y = to_dev(Y0, torch.float32)
        hb.expand(Wc, Y, 0.5)
        err = rel_elem(Y.cpu().numpy().astype(np.float64), ref)
        print(name, "scatter form", form, "elementwise err", err)
        assert err < 1e-5, (name, form, err)


@pytest.mark.parametrize("name,form", [("ragged", 3), ("crowded", 3), ("crowded", 2)])
def test_apply_H_and_filter_with_the_tensor_core_gather(name, form):
    wl = w.small_test_system(**CASES[name])
    H = oracle_ham(wl, D=wl.D0[0])
    X = wl.orbitals().astype(np.float32).astype(np.float64)
    hb = make_hub(wl, HUB_F32)
    hb.set_occupation_matrix(0, wl.D0[0])
    hb.set_tuning(gather_form=form)
    Xd = to_dev(X, torch.float32)
    Yd = torch.empty_like(Xd)
    hb.apply_H(0, Xd, Yd)
    err = rel_elem(Yd.cpu().numpy().astype(np.float64), H.apply(X.T).T)
    print(name, "H X elementwise err", err)
    assert err < 5e-6
    lo, up = o.lanczos_bounds(H, wl.lanczos_start(), 10)
    glo, gup = hb.lanczos_bound(0, 10, to_dev(wl.lanczos_start(), torch.float32))
    assert abs(glo - lo) < 1e-4 * abs(up) and abs(gup - up) < 1e-4 * abs(up)
    a_low, a, b = lo, lo + 0.1 * (up - lo), up
    ref = o.chebyshev_filter(H, X.T, 6, a, b, a_low).T
    hb.chefsi_filter(0, Xd, 6, a, b, a_low)
    err = rel_elem(Xd.cpu().numpy().astype(np.float64), ref)
    print(name, "degree-6 filter elementwise err", err)
    # six recurrence steps of the per-application float bound
    assert err < 6 * 5e-6
