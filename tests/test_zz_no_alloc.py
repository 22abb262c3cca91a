"""hub_gram_noalloc, the allocation-free form of the Gram block product.

Some callers cannot allocate device memory when they need this product: code that runs
during CUDA graph capture, services whose memory is owned by a pooling allocator, callers
without a hub handle.  hub_gram_noalloc keeps its split-K partial sums in a static device
array instead of handle-owned scratch.  This test calls it twice in a row, with different
shapes (the second call also takes the symmetric path), in double and in float, and checks
each result element by element against hub_gram, which computes the same product with
handle-owned scratch, and against the oracle's grid inner product dV A^T B of the same
values: FP64 to the 1e-10 tolerance of the other parity tests; float to 1e-5 against
hub_gram (the two use different tile shapes, so their float partial sums round differently)
and 2e-6 against the oracle (the float Gram bound of the other tests).  It also checks
that a product whose partial tile would not fit the static array is rejected before any
GPU work.  This file is collected last so that a failure here cannot hide another test's
result."""
import ctypes

import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import make_hub, to_dev, rel_elem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F32, HUB_F64, load_library  # noqa: E402

TOL = {HUB_F64: (1e-10, 1e-10), HUB_F32: (1e-5, 2e-6)}     # (against hub_gram, against the oracle)


def _noalloc(lib, A, B, alpha, G, prec=HUB_F64):
    na, ld = A.shape
    nb = B.shape[0]
    rc = lib.hub_gram_noalloc(ctypes.c_void_p(A.data_ptr()), na, ctypes.c_void_p(B.data_ptr()), nb,
                              A.shape[1], ld, prec, alpha, ctypes.c_void_p(G.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


@pytest.mark.parametrize("prec", [HUB_F64, HUB_F32])
def test_noalloc_gram_matches_hub_gram_on_two_calls(prec):
    lib = load_library()
    wl = w.small_test_system(n=(20, 24, 28), ncol=37, natoms=1)
    hb = make_hub(wl, prec)
    g = o.Grid(wl.n, wl.L)
    dV = wl.dV
    tol_hub, tol_oracle = TOL[prec]
    cases = [("A B^T", 37, 29, False), ("A A^T (symmetric path)", 23, 23, True)]
    for k, (name, na, nb, same) in enumerate(cases):
        A = to_dev(w.random_orbitals(wl.Nd, na, 50 + k), hb.dtype)
        B = A if same else to_dev(w.random_orbitals(wl.Nd, nb, 60 + k), hb.dtype)
        G_ref = torch.empty(na, nb, dtype=torch.float64, device="cuda")
        hb.gram(A, B, dV, G_ref)
        G = torch.full((na, nb), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(lib, A, B, dV, G, prec) == 0, name
        torch.cuda.synchronize()
        got = G.cpu().numpy()
        err_hub = rel_elem(got, G_ref.cpu().numpy())
        oracle = g.inner(A.double().cpu().numpy().T, B.double().cpu().numpy().T)
        err_oracle = rel_elem(got, oracle)
        print(name, prec, "vs hub_gram", err_hub, "vs oracle", err_oracle)
        assert err_hub < tol_hub and err_oracle < tol_oracle, name


def test_noalloc_gram_rejects_tiles_beyond_the_static_array():
    lib = load_library()
    nrows = 1024
    A = torch.zeros(2100, nrows, dtype=torch.float64, device="cuda")   # 2100^2 > 4 Mi doubles
    G = torch.zeros(2100, 2100, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, A, A, 1.0, G) == -1                          # HUB_EINVAL, no launch
    assert torch.count_nonzero(G).item() == 0
