"""The SCF driver of the library (hub_scf_*) against the oracle's SCF with the same
algorithm (Sec. II.B last paragraph: D updated every iteration, Pulay mixing of D).
Both start from the same seeded orbitals, Lanczos vectors and D0, so they must reach the
same fixed point with the same iteration count."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import make_hub, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F64, scf_params  # noqa: E402


def test_scf_spin_polarised_matches_oracle():
    wl = w.small_test_system(n=(16, 14, 18), natoms=2, ncol=14, hub_rc=3.0, kb_rc=2.0, nspin=2)
    kw = dict(n_elec=16.0, kT=0.01, degree=12, max_iter=80, tol_e_atom=1e-10, tol_D=1e-7,
              first_passes=4, hist=7, beta=0.3, lanczos_steps=10)
    X0s = [wl.orbitals(s) for s in range(2)]
    v0s = [wl.lanczos_start(s) for s in range(2)]
    ref = o.scf_model_a((wl.n, wl.L, (0, 0, 0), 6), wl.veff, wl.atoms, wl.D0, [x.T for x in X0s],
                        lanczos_v0s=v0s, **kw)
    assert ref["converged"]

    hb = make_hub(wl, HUB_F64)
    p = scf_params(nspin=2, ncol=wl.ncol, ld=wl.Nd, degree=kw["degree"], max_iter=kw["max_iter"],
                   first_passes=kw["first_passes"], lanczos_steps=10, pulay_history=7,
                   natoms=len(wl.atoms), pulay_beta=0.3, kT=kw["kT"], n_elec=kw["n_elec"],
                   tol_e_atom=kw["tol_e_atom"], tol_D=kw["tol_D"])
    Xs = [to_dev(x, torch.float64) for x in X0s]
    vs = [to_dev(v, torch.float64) for v in v0s]
    hb.scf_begin(p, Xs, vs, wl.D0)
    res = hb.scf_run()
    eig, occ, D = hb.scf_get()
    print("gpu", res, "oracle", ref["iterations"], ref["E"])
    assert res["converged"] == 1
    # near the fixed point the Pulay system is ill-conditioned: the oracle's least-squares
    # solve and the library's pivoted elimination may take a few different iterations
    assert abs(res["iter"] - ref["iterations"]) <= 5
    assert abs(res["E"] - ref["E"]) < 1e-9 * max(1.0, abs(ref["E"]))
    assert abs(res["E_U"] - ref["E_U"]) < 1e-9
    np.testing.assert_allclose(D, ref["D"], atol=1e-7)
    # the top Ritz values of the block are unconverged buffer states (their value depends on
    # how many iterations ran); the occupied part and a margin above it are converged
    np.testing.assert_allclose(eig[:, :10], np.array(ref["eig"])[:, :10], atol=1e-8)
    np.testing.assert_allclose(occ, np.array(ref["f"]), atol=1e-8)


@pytest.mark.parametrize("prec,ladder", [("f32", 0), ("mixed", 1), ("mixed16", 1), ("mixed16", 0)])
def test_reduced_precision_scf_reaches_the_fp64_fixed_point(prec, ladder):
    """FP32 filter (and BF16 or FP16 tensor-core products, with or without the precision
    ladder) reach the oracle's FP64 SCF fixed point within 1e-5 Ha/atom in energy and band
    energy."""
    from paper_2507_23612_gb300 import HUB_F32, HUB_MIXED_BF16, HUB_MIXED_F16
    wl = w.small_test_system(n=(16, 16, 20), natoms=2, ncol=14, hub_rc=3.0, kb_rc=2.0, nspin=2)
    kw = dict(n_elec=16.0, kT=0.01, degree=12, max_iter=80, tol_e_atom=1e-7, tol_D=1e-5,
              first_passes=4, hist=7, beta=0.3, lanczos_steps=10)
    X0s = [wl.orbitals(s) for s in range(2)]
    v0s = [wl.lanczos_start(s) for s in range(2)]
    ref = o.scf_model_a((wl.n, wl.L, (0, 0, 0), 6), wl.veff, wl.atoms, wl.D0, [x.T for x in X0s],
                        lanczos_v0s=v0s, **kw)
    assert ref["converged"]
    P = {"f32": HUB_F32, "mixed": HUB_MIXED_BF16, "mixed16": HUB_MIXED_F16}[prec]
    hb = make_hub(wl, P)
    p = scf_params(nspin=2, ncol=wl.ncol, ld=wl.Nd, degree=kw["degree"], max_iter=kw["max_iter"],
                   first_passes=kw["first_passes"], lanczos_steps=10, pulay_history=7,
                   natoms=len(wl.atoms), pulay_beta=0.3, kT=kw["kT"], n_elec=kw["n_elec"],
                   tol_e_atom=kw["tol_e_atom"], tol_D=kw["tol_D"], ladder=ladder, ladder_tol=1e-4)
    Xs = [to_dev(x, torch.float32) for x in X0s]
    vs = [to_dev(v, torch.float32) for v in v0s]
    hb.scf_begin(p, Xs, vs, wl.D0)
    res = hb.scf_run()
    eig, occ, D = hb.scf_get()
    nat = len(wl.atoms)
    e_err = abs(res["E"] - ref["E"]) / nat
    eu_err = abs(res["E_U"] - ref["E_U"]) / nat
    band = sum(float(np.dot(ref["f"][s], ref["eig"][s])) for s in range(2))
    band_gpu = float(np.sum(occ * eig))
    print(prec, "iters", res["iter"], "E err/atom", e_err, "E_U err/atom", eu_err,
          "band err/atom", abs(band_gpu - band) / nat, "max dD", np.max(np.abs(D - ref["D"])),
          "terms", res["bf16_terms"])
    assert res["converged"] == 1
    assert e_err < 1e-5 and eu_err < 1e-5 and abs(band_gpu - band) / nat < 1e-5
    assert np.max(np.abs(D - ref["D"])) < 1e-3
    if ladder:
        assert res["bf16_terms"] == 0          # finished on float products
