"""The SCF with Brillouin-zone sampling over one library handle per k-point against the
oracle's k-point SCF: the Gamma point alone, a pair k, -k (real D), and one Bloch point
(complex Hermitian D).  Both sides start from the same orbitals, Lanczos vectors and D0 and
must reach the same fixed point.  The whole driver (Fermi level over the k-weighted states,
the Brillouin-zone average of D, the energy terms and Pulay) runs in the library
(hub_kscf_*); the Python class only marshals handles and arrays.  Tolerances: E to 1e-9
relative and D to 1e-6 (the SCF tolerances tol_e_atom = 1e-8 and tol_D = 1e-6)."""
import numpy as np
import pytest

import workloads as w
from oracle import hubbard as o
from hubtest import to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import HUB_F64  # noqa: E402
from paper_2507_23612_gb300.kpoint_scf import KpointSCF, run_batched  # noqa: E402

K = (0.3, -0.2, 0.25)


@pytest.mark.parametrize("kpts,kw", [([(0.0, 0.0, 0.0)], [1.0]),
                                     ([K, tuple(-np.asarray(K))], [0.5, 0.5]),
                                     ([K], [1.0])], ids=["gamma", "pair", "bloch"])
def test_kpoint_scf_matches_the_oracle(kpts, kw):
    wl = w.small_test_system(n=(12, 10, 14), ncol=8, natoms=2, seed=11)
    nk = len(kpts)
    X0 = [[wl.orbitals(complex_=any(kpts[k])) for k in range(nk)]]
    v0 = [[wl.lanczos_start(complex_=any(kpts[k])) for k in range(nk)]]
    if nk == 2:
        X0[0][1], v0[0][1] = np.conj(X0[0][0]), np.conj(v0[0][0])
    kwargs = dict(n_elec=6.0, kT=0.01, degree=12, max_iter=80, tol_e_atom=1e-8, tol_D=1e-6)
    ref = o.scf_model_a_kpoints(wl.n, wl.L, kpts, kw, wl.veff, wl.atoms, wl.D0,
                                [[x.T for x in X0[0]]], lanczos_v0s=v0, **kwargs)
    assert ref["converged"]
    scf = KpointSCF(wl, kpts, kw, HUB_F64)
    try:
        Xd = [[to_dev(X0[0][k], scf.hubs[k].dtype) for k in range(nk)]]
        vd = [[to_dev(v0[0][k], scf.hubs[k].dtype) for k in range(nk)]]
        res = scf.run(Xd, vd, wl.D0, **kwargs)
    finally:
        scf.close()
    print({"gpu": (res["iterations"], res["E"]), "oracle": (ref["iterations"], ref["E"])})
    assert res["converged"]
    assert abs(res["E"] - ref["E"]) < 1e-9 * max(1.0, abs(ref["E"]))
    np.testing.assert_allclose(res["D"], ref["D"], atol=1e-6)


def test_batched_kpoint_scfs_match_the_oracle():
    """The three k-sets above as three SCFs run batched (hub_kscf_run_batch: the filters of
    all four channels in one CUDA graph per pass); each reaches the oracle's fixed point."""
    wl = w.small_test_system(n=(12, 10, 14), ncol=8, natoms=2, seed=11)
    sets = [([(0.0, 0.0, 0.0)], [1.0]), ([K, tuple(-np.asarray(K))], [0.5, 0.5]), ([K], [1.0])]
    kwargs = dict(n_elec=6.0, kT=0.01, degree=12, max_iter=80, tol_e_atom=1e-8, tol_D=1e-6)
    scfs, refs = [], []
    try:
        for kpts, kw in sets:
            nk = len(kpts)
            X0 = [[wl.orbitals(complex_=any(kpts[k])) for k in range(nk)]]
            v0 = [[wl.lanczos_start(complex_=any(kpts[k])) for k in range(nk)]]
            if nk == 2:
                X0[0][1], v0[0][1] = np.conj(X0[0][0]), np.conj(v0[0][0])
            refs.append(o.scf_model_a_kpoints(wl.n, wl.L, kpts, kw, wl.veff, wl.atoms, wl.D0,
                                              [[x.T for x in X0[0]]], lanczos_v0s=v0, **kwargs))
            scf = KpointSCF(wl, kpts, kw, HUB_F64)
            scfs.append(scf)
            Xd = [[to_dev(X0[0][k], scf.hubs[k].dtype) for k in range(nk)]]
            vd = [[to_dev(v0[0][k], scf.hubs[k].dtype) for k in range(nk)]]
            scf.begin(Xd, vd, wl.D0, **kwargs)
        out = run_batched(scfs)
    finally:
        for scf in scfs:
            scf.close()
    for res, ref in zip(out, refs):
        print({"gpu": (res["iterations"], res["E"]), "oracle": (ref["iterations"], ref["E"])})
        assert res["converged"]
        assert abs(res["E"] - ref["E"]) < 1e-9 * max(1.0, abs(ref["E"]))
        np.testing.assert_allclose(res["D"], ref["D"], atol=1e-6)
