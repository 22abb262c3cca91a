"""Host-side logic of the warm start (no GPU): packing of occupation matrices into the
model's targets and back, and the displaced-cell workloads it trains on."""
import numpy as np

import workloads as w
from paper_2507_23612_gb300.warmstart import N_IN, pack_occupations, unpack_occupations


def test_pack_roundtrip_and_layout():
    g = np.random.Generator(np.random.PCG64(0))
    A = g.normal(size=(2, 3, 5, 5))
    D = A + A.transpose(0, 1, 3, 2)
    Y = pack_occupations(D)
    assert Y.shape == (3, 30)
    # upper triangle row by row, spin 0 then spin 1
    assert Y[1, 0] == D[0, 1, 0, 0] and Y[1, 1] == D[0, 1, 0, 1] and Y[1, 5] == D[0, 1, 1, 1]
    assert Y[2, 15] == D[1, 2, 0, 0]
    np.testing.assert_array_equal(unpack_occupations(Y, 2), D)


def test_descriptor_width():
    assert N_IN == 2 * (16 + 8)


def test_rutile_snapshots_are_seeded_and_displaced():
    a = w.rutile_snapshot((1, 1, 2), 0.1, seed=3)
    b = w.rutile_snapshot((1, 1, 2), 0.1, seed=3)
    c = w.rutile_snapshot((1, 1, 2), 0.1, seed=4)
    pa = np.array([x.pos for x in a.atoms])
    assert np.array_equal(pa, np.array([x.pos for x in b.atoms]))
    assert not np.allclose(pa, np.array([x.pos for x in c.atoms]))
    # one pseudopotential per species
    gam = {x.species: x.kb_gamma for x in a.atoms}
    assert all(x.kb_gamma == gam[x.species] for x in a.atoms)
    big = w.rutile_snapshot((3, 3, 4))
    assert big.n == (132, 132, 112) and big.ncol == 1044 and len(big.atoms) == 216


def test_scf_checkpoint_roundtrip(tmp_path):
    from paper_2507_23612_gb300.md import load_scf_checkpoint, save_scf_checkpoint
    rng = np.random.default_rng(0)
    Xs = [rng.standard_normal((4, 30)) for _ in range(2)]
    D = rng.standard_normal((2, 3, 5, 5))
    save_scf_checkpoint(tmp_path / "c.npz", Xs, D, {"iter": 7, "E": -1.25, "seed": 3})
    X2, D2, meta = load_scf_checkpoint(tmp_path / "c.npz")
    assert len(X2) == 2 and all(np.array_equal(a, b) for a, b in zip(Xs, X2))
    assert np.array_equal(D, D2) and meta == {"iter": 7, "E": -1.25, "seed": 3}
