"""Argument checks of the C ABI that happen on the host, before any device work: bad sizes,
orders, precisions and NULL handles come back as HUB_EINVAL (no GPU needed, no launch)."""
import ctypes as C

import numpy as np
import pytest

EINVAL = -1


@pytest.fixture(scope="module")
def lib():
    from paper_2507_23612_gb300 import build as b
    b.build()
    from paper_2507_23612_gb300 import binding
    return binding.load_library()


def _create(lib, n=(8, 8, 8), L=(2.0, 2.0, 2.0), order=6, prec=0):
    h = C.c_void_p()
    k = (C.c_double * 3)(0.0, 0.0, 0.0)
    rc = lib.hub_create_grid(C.byref(h), n[0], n[1], n[2], L[0], L[1], L[2], order, 0, k, prec, None)
    return rc, h


@pytest.mark.parametrize("kw", [dict(n=(0, 8, 8)), dict(n=(8, -1, 8)), dict(L=(2.0, 0.0, 2.0)),
                                dict(L=(float("nan"), 2.0, 2.0)), dict(order=0), dict(order=7),
                                dict(prec=4), dict(prec=-1), dict(n=(2000, 2000, 1000))])
def test_create_grid_rejects_bad_arguments(lib, kw):
    rc, h = _create(lib, **kw)
    assert rc == EINVAL and not h.value


def test_null_handles(lib):
    assert lib.hub_destroy(None) == 0
    assert lib.hub_last_error(None)                         # a message, not a crash
    assert lib.hub_set_tuning(None, 0, 1, 0) == EINVAL
    n = C.c_int()
    assert lib.hub_get_tuning(None, C.byref(n), None, None, None) == EINVAL
    assert lib.hub_mlp_destroy(None) == 0


def test_batch_filter_rejects_empty_batch(lib):
    assert lib.hub_batch_filter(0, None, None, None, None, None, 24, None, None, None, None) == EINVAL


def test_mlp_create_rejects_bad_shapes(lib):
    m = C.c_void_p()
    for args in [(0, 256, 3, 30), (48, 0, 3, 30), (48, 256, 0, 30), (48, 256, 3, 0)]:
        assert lib.hub_mlp_create(C.byref(m), *args, 1, 0, None) == EINVAL


def test_descriptors_reject_bad_inputs(lib):
    pos = np.zeros(6)
    L = np.array([10.0, 10.0, 10.0])
    out = C.c_void_p(0)

    def call(species, centers, nspecies=2, nrad=16, rc=6.0, eta=0.4):
        sp = np.ascontiguousarray(species, dtype=np.int32)
        ce = np.ascontiguousarray(centers, dtype=np.int32)
        return lib.hub_descriptors(2, pos.ctypes.data_as(C.POINTER(C.c_double)),
                                   sp.ctypes.data_as(C.POINTER(C.c_int)),
                                   L.ctypes.data_as(C.POINTER(C.c_double)), len(ce),
                                   ce.ctypes.data_as(C.POINTER(C.c_int)), nspecies, rc, nrad, eta,
                                   out, None)
    assert call([0, 2], [0]) == EINVAL                     # species out of range
    assert call([0, 1], [2]) == EINVAL                     # centre out of range
    assert call([0, 1], [0], nspecies=3) == EINVAL          # at most two species
    assert call([0, 1], [0], nrad=33) == EINVAL             # at most 32 radial values
    assert call([0, 1], [0], rc=0.0) == EINVAL
    assert call([0, 1], [0], eta=-1.0) == EINVAL


def test_gram_noalloc_rejects_bad_arguments_before_any_device_work(lib):
    assert lib.hub_gram_noalloc(None, 4, None, 4, 1024, 1024, 0, 1.0, None, None) == EINVAL   # NULL operands
    assert lib.hub_gram_noalloc(None, 4, None, 4, 1024, 1000, 0, 1.0, None, None) == EINVAL   # ld < nrows
    assert lib.hub_gram_noalloc(None, 4, None, 4, 1024, 1024, 2, 1.0, None, None) == EINVAL   # precision
    assert lib.hub_gram_noalloc(None, 0, None, 4, 1024, 1024, 0, 1.0, None, None) == 0        # empty: no work


def test_hubbard_forces_rejects_a_null_handle(lib):
    F = (C.c_double * 3)()
    assert lib.hub_hubbard_forces(None, 0, None, 0, 0, None, 1.0, F, None) == EINVAL


def test_density_steps_reject_a_null_handle(lib):
    assert lib.hub_density(None, None, 0, 0, None, 1.0, None) == EINVAL
    assert lib.hub_hartree(None, None, None, 1e-10, 10, None, None) == EINVAL
    assert lib.hub_lda_exchange(None, 1, None, None, None, None, None) == EINVAL
    assert lib.hub_kerker(None, None, None, 0.5, 1e-10, 10, None) == EINVAL
    assert lib.hub_scf_density(None, None) == EINVAL


def test_scf_structs_match_the_header(lib):
    # the binding's ctypes layouts carry every field the header declares, in order
    import re
    from paper_2507_23612_gb300.binding import scf_params, scf_result
    import os
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hub.h")).read()
    for struct, name in ((scf_params, "hub_scf_params"), (scf_result, "hub_scf_result")):
        body = hdr[:hdr.index("} " + name + ";")]
        body = body[body.rindex("typedef struct {"):]
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = []
        for decl in body.split(";")[:-1]:
            decl = decl.replace("typedef struct {", "").strip()
            names = decl.split(None, 1)[1]
            fields += [n.strip() for n in names.split(",")]
        assert [f for f, _ in struct._fields_] == fields, name


def test_hubbard_stress_rejects_a_null_handle(lib):
    sig = (C.c_double * 9)()
    assert lib.hub_hubbard_stress(None, 0, None, 0, 0, None, 1.0, sig, None) == EINVAL


def test_extrapolation_rejects_bad_history(lib):
    D = (C.c_double * 25)()
    out = (C.c_double * 25)()
    assert lib.hub_extrapolate_occupations(25, 4, D, D, 0, None, None, out) == EINVAL    # nhist > 3
    assert lib.hub_extrapolate_occupations(25, 1, None, D, 0, None, None, out) == EINVAL  # no history array
    assert lib.hub_extrapolate_occupations(25, 2, D, D, 1, None, None, out) == EINVAL     # no positions
    assert lib.hub_extrapolate_occupations(25, 0, None, D, 0, None, None, out) == 0       # atomic guess


def test_scf_forces_rejects_a_null_handle(lib):
    F = (C.c_double * 3)()
    assert lib.hub_scf_forces(None, F, None) == EINVAL


def test_projector_entry_points_reject_a_null_handle(lib):
    n = C.c_int()
    assert lib.hub_num_projectors(None, C.byref(n)) == EINVAL
    assert lib.hub_project(None, None, 0, 0, None) == EINVAL
    assert lib.hub_expand(None, None, 0, None, 0, 1.0) == EINVAL
    assert lib.hub_scf_set_density(None, None) == EINVAL


def test_binding_rejects_blocks_of_the_wrong_type_before_any_call():
    # the checks run on the host before the library is called, so a handle-less object
    # with the handle's type fields is enough (no GPU)
    torch = pytest.importorskip("torch")
    from paper_2507_23612_gb300.binding import Hub, HUB_F64, HUB_F32
    hb = Hub.__new__(Hub)
    hb.n, hb.Nd, hb.complex = (4, 4, 4), 64, False
    hb.prec = HUB_F64
    with pytest.raises(ValueError):
        hb._blk(torch.zeros((3, 64), dtype=torch.float32), "X")          # float block, FP64 handle
    with pytest.raises(ValueError):
        hb._blk(torch.zeros((3, 60), dtype=torch.float64), "X")          # ld < Nd
    assert hb._blk(torch.zeros((3, 70), dtype=torch.float64), "X") == (3, 70)
    assert hb._blk(torch.zeros((0, 64), dtype=torch.float64), "X") == (0, 64)
    hb.prec = HUB_F32
    hb.complex = True
    with pytest.raises(ValueError):
        hb._blk(torch.zeros((3, 64), dtype=torch.float64), "X")          # same size, not complex
    hb._blk(torch.zeros((3, 64), dtype=torch.complex64), "X")
    with pytest.raises(ValueError):
        hb._vec(torch.zeros(63, dtype=torch.float64), torch.float64, "v")  # too short
    hb.h = None                                                         # nothing to release


def test_kpoint_scf_rejects_bad_arguments(lib):
    from paper_2507_23612_gb300.binding import scf_params, scf_result
    obj = C.c_void_p()
    p = scf_params(nspin=1, ncol=4, ld=512, degree=8, max_iter=5, first_passes=1, lanczos_steps=10,
                   pulay_history=7, natoms=1, pulay_beta=0.3, kT=0.01, n_elec=2.0, tol_e_atom=1e-5, tol_D=1e-4)
    w = (C.c_double * 1)(1.0)
    hs = (C.c_void_p * 1)(None)
    xs = (C.c_void_p * 1)(None)
    assert lib.hub_kscf_create(None, 1, hs, w, C.byref(p), xs, xs, None, None) == EINVAL
    assert lib.hub_kscf_create(C.byref(obj), 0, hs, w, C.byref(p), xs, xs, None, None) == EINVAL
    assert lib.hub_kscf_create(C.byref(obj), 1, hs, w, C.byref(p), xs, xs, None, None) == EINVAL   # NULL handle
    assert lib.hub_kscf_create(C.byref(obj), 1, None, w, C.byref(p), xs, xs, None, None) == EINVAL
    assert not obj.value
    r = scf_result()
    assert lib.hub_kscf_iterate(None, C.byref(r)) == EINVAL
    assert lib.hub_kscf_run(None, C.byref(r)) == EINVAL
    assert lib.hub_kscf_get(None, None, None, None, None) == EINVAL
    assert lib.hub_kscf_destroy(None) == 0
    assert lib.hub_kscf_last_error(None)
