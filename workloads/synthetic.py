"""Seeded synthetic stand-ins for the paper's TiO2 workloads.

The paper's own inputs (ONCV pseudopotentials, Materials-Project geometries, the spectral
atomic solver's radial orbitals) are not available, so every workload here is synthetic:

* the local potential is a periodic sum of Gaussians (seeded depths and widths, or one
  Gaussian per atom for the crystal cells);
* nonlocal projectors and Hubbard orbitals are Gaussian-type radial functions
  ``r^l exp(-r^2 / (2 rs^2))`` times real spherical harmonics, with hard cutoffs;
* geometries are ideal rutile / anatase-shaped cells (textbook lattice constants), optionally
  with seeded Gaussian displacements;
* starting orbitals and the Lanczos start vector are standard normal draws.

Every random draw uses ``numpy.random.Generator(PCG64(seed))``.  Arrays on the grid are
flattened x-fastest: ``index = i1 + n1 * (i2 + n2 * i3)``.  A block of orbitals is stored
column-major (numpy shape ``(ncol, Nd)``, C order), i.e. column ``j`` is ``X[j]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

HARTREE_EV = 27.211386245988          # CODATA 2018, eV per hartree
BOHR_PER_ANGSTROM = 1.0 / 0.529177210903


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Atom:
    """One atom: position plus the parameters of its localized functions.

    KB-type nonlocal projectors come in channels (one per angular momentum ``l``, with
    ``2l+1`` projectors each); every channel has a Gaussian width ``rs`` and an energy
    ``gamma`` (Ha).  ``hub_l`` is -1 for atoms without Hubbard orbitals and 2 for d shells.
    """
    species: str
    pos: np.ndarray
    kb_l: tuple = ()
    kb_rs: tuple = ()
    kb_gamma: tuple = ()
    kb_rc: float = 0.0
    hub_l: int = -1
    hub_rs: float = 1.0
    hub_rc: float = 0.0
    hub_U: float = 0.0

    @property
    def n_kb(self) -> int:
        return int(sum(2 * l + 1 for l in self.kb_l))

    @property
    def n_hub(self) -> int:
        return 0 if self.hub_l < 0 else 2 * self.hub_l + 1


@dataclass
class Workload:
    name: str
    n: tuple
    L: tuple
    veff: np.ndarray                # (Nd,) float64, Ha
    atoms: list
    ncol: int
    degree: int
    nspin: int = 1
    kpts: tuple = ((0.0, 0.0, 0.0),)  # Cartesian Bloch wavevectors (bohr^-1)
    kweights: tuple = (1.0,)
    n_elec: float = 0.0             # electrons in the cell; with nspin == 1 every state
                                    # holds two electrons, with nspin == 2 one
    kT: float = 0.005
    D0: np.ndarray = None           # (nspin, nhub_atoms, 5, 5) starting occupation matrices
    fd_half_order: int = 6
    seed_orbitals: int = 2
    seed_lanczos: int = 3
    meta: dict = field(default_factory=dict)

    @property
    def Nd(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def h(self) -> tuple:
        return tuple(self.L[a] / self.n[a] for a in range(3))

    @property
    def dV(self) -> float:
        h = self.h
        return h[0] * h[1] * h[2]

    @property
    def hub_atoms(self) -> list:
        return [a for a in self.atoms if a.hub_l >= 0]

    def orbitals(self, spin: int = 0, kidx: int = 0, complex_: bool = False,
                 dtype=np.float64) -> np.ndarray:
        """Starting block, shape (ncol, Nd): column j is X[j].  Seeded per (spin, k)."""
        return random_orbitals(self.Nd, self.ncol,
                               self.seed_orbitals + 1000 * spin + 100 * kidx,
                               complex_=complex_, dtype=dtype)

    def lanczos_start(self, spin: int = 0, kidx: int = 0, complex_: bool = False) -> np.ndarray:
        return random_orbitals(self.Nd, 1, self.seed_lanczos + 1000 * spin + 100 * kidx,
                               complex_=complex_)[0]


def random_orbitals(Nd: int, ncol: int, seed: int, complex_: bool = False,
                    dtype=np.float64) -> np.ndarray:
    g = _rng(seed)
    if complex_:
        re = g.standard_normal((ncol, Nd))
        im = g.standard_normal((ncol, Nd))
        out = (re + 1j * im) / np.sqrt(2.0)
        return out.astype(np.complex128 if dtype in (np.float64, np.complex128) else np.complex64)
    return g.standard_normal((ncol, Nd)).astype(dtype, copy=False)


def gaussian_potential(n, L, centres, depths, widths) -> np.ndarray:
    """Periodic sum of Gaussians on the grid, summed over enough lattice images."""
    n = tuple(int(v) for v in n)
    L = np.asarray(L, dtype=np.float64)
    h = L / np.asarray(n)
    axes = [np.arange(n[a]) * h[a] for a in range(3)]
    V = np.zeros((n[2], n[1], n[0]))
    for c, A, w in zip(np.asarray(centres, dtype=np.float64), depths, widths):
        reach = 7.0 * w
        comp = []
        for a in range(3):
            tmax = int(np.ceil(reach / L[a])) + 1
            acc = np.zeros(n[a])
            for t in range(-tmax, tmax + 1):
                d = axes[a] - c[a] - t * L[a]
                acc += np.exp(-d * d / (2.0 * w * w))
            comp.append(acc)
        # a Gaussian factorises over the three axes, and so does its image sum
        V += A * comp[2][:, None, None] * comp[1][None, :, None] * comp[0][None, None, :]
    return V.reshape(-1)


# ----------------------------------------------------------------------------- geometry

def rutile_cell(a_ang: float = 4.594, c_ang: float = 2.959, u: float = 0.305):
    a = a_ang * BOHR_PER_ANGSTROM
    c = c_ang * BOHR_PER_ANGSTROM
    ti = [(0.0, 0.0, 0.0), (0.5, 0.5, 0.5)]
    o = [(u, u, 0.0), (1 - u, 1 - u, 0.0), (0.5 + u, 0.5 - u, 0.5), (0.5 - u, 0.5 + u, 0.5)]
    return np.array([a, a, c]), ti, o


def anatase_cell(a_ang: float = 3.785, c_ang: float = 9.514, z: float = 0.208):
    a = a_ang * BOHR_PER_ANGSTROM
    c = c_ang * BOHR_PER_ANGSTROM
    ti = [(0.0, 0.0, 0.0), (0.0, 0.5, 0.25), (0.5, 0.5, 0.5), (0.5, 0.0, 0.75)]
    o = []
    for t in ti:
        o.append((t[0], t[1], (t[2] + z) % 1.0))
        o.append((t[0], t[1], (t[2] - z) % 1.0))
    return np.array([a, a, c]), ti, o


def _supercell(cell, reps):
    lat, ti, o = cell
    reps = tuple(int(r) for r in reps)
    L = lat * np.asarray(reps)
    pos_ti, pos_o = [], []
    for i in range(reps[0]):
        for j in range(reps[1]):
            for k in range(reps[2]):
                shift = np.array([i, j, k], dtype=np.float64)
                for f in ti:
                    pos_ti.append((np.asarray(f) + shift) * lat)
                for f in o:
                    pos_o.append((np.asarray(f) + shift) * lat)
    return L, pos_ti, pos_o


def scaled_grid_for(L, h_target: float = 0.2, multiple: int = 4):
    return tuple(int(multiple * max(1, round(Lx / h_target / multiple))) for Lx in L)


def displaced(positions, sigma: float, seed: int):
    g = _rng(seed)
    return [np.asarray(p) + sigma * g.standard_normal(3) for p in positions]


def _tio2_atoms(pos_ti, pos_o, U_ev: float, seed_gamma: int, kb_rc: float = 2.5,
                hub_rc: float = 5.0, species_gamma: bool = False):
    """Ti (KB s/p/d + Hubbard d) and O (KB s/p/d) atoms.  KB strengths are drawn per atom,
    or, with species_gamma, once per species (the same pseudopotential for every atom of a
    species, as transferable models across cells need)."""
    g = _rng(seed_gamma)
    if species_gamma:
        g_ti, g_o = tuple(g.uniform(0.5, 2.0, 3)), tuple(g.uniform(0.5, 2.0, 3))
    atoms = []
    for p in pos_ti:
        atoms.append(Atom("Ti", np.asarray(p, dtype=np.float64), kb_l=(0, 1, 2),
                          kb_rs=(0.8, 0.8, 1.0),
                          kb_gamma=g_ti if species_gamma else tuple(g.uniform(0.5, 2.0, 3)),
                          kb_rc=kb_rc, hub_l=2, hub_rs=1.0, hub_rc=hub_rc,
                          hub_U=U_ev / HARTREE_EV))
    for p in pos_o:
        atoms.append(Atom("O", np.asarray(p, dtype=np.float64), kb_l=(0, 1, 2),
                          kb_rs=(0.8, 0.8, 1.0),
                          kb_gamma=g_o if species_gamma else tuple(g.uniform(0.5, 2.0, 3)),
                          kb_rc=kb_rc))
    return atoms


def _tio2_potential(n, L, atoms):
    centres = [a.pos for a in atoms]
    depths = [-3.0 if a.species == "Ti" else -2.0 for a in atoms]
    widths = [1.2 if a.species == "Ti" else 0.9 for a in atoms]
    return gaussian_potential(n, L, centres, depths, widths)


def _spin_split_D0(nhub: int, nspin: int, base: float = 0.2, split: float = 0.05):
    D0 = np.zeros((nspin, nhub, 5, 5))
    for s in range(nspin):
        occ = base if nspin == 1 else base + (split if s == 0 else -split)
        D0[s] = occ * np.eye(5)[None]
    return D0


# ----------------------------------------------------------------------------- workloads

def tiny() -> Workload:
    """24^3 periodic cube at h = 0.3 bohr, 2 Ti-like atoms, 32 real orbitals, degree 20."""
    n = (24, 24, 24)
    L = (7.2, 7.2, 7.2)
    g = _rng(0)
    depths = g.uniform(-2.0, 0.0, 8)
    widths = g.uniform(0.5, 1.5, 8)
    centres = g.uniform(0.0, 1.0, (8, 3)) * np.asarray(L)
    veff = gaussian_potential(n, L, centres, depths, widths)
    ga = _rng(1)
    atoms = []
    for _ in range(2):
        pos = ga.uniform(0.0, 1.0, 3) * np.asarray(L)
        atoms.append(Atom("Ti", pos, kb_l=(0, 1), kb_rs=(0.8, 0.8),
                          kb_gamma=tuple(ga.uniform(0.5, 2.0, 2)), kb_rc=3.0,
                          hub_l=2, hub_rs=1.0, hub_rc=5.0, hub_U=4.0 / HARTREE_EV))
    return Workload("tiny-24^3-2atoms-32orb", n, L, veff, atoms, ncol=32, degree=20, nspin=1,
                    n_elec=32.0, kT=0.0, D0=_spin_split_D0(2, 1),
                    seed_orbitals=2, seed_lanczos=3,
                    meta={"occupations": "f=1 for the lowest 16 states, else 0"})


def rutile(reps=(2, 2, 3), grid=(88, 88, 84), n_occ=290, n_extra=58, degree=24,
           U_ev: float = 3.5, nspin: int = 2, seed_gamma: int = 4) -> Workload:
    """Rutile-shaped supercell (default 2x2x3: 24 Ti + 48 O, 88x88x84 grid, 348 orbitals)."""
    L, pti, po = _supercell(rutile_cell(), reps)
    atoms = _tio2_atoms(pti, po, U_ev, seed_gamma)
    veff = _tio2_potential(grid, L, atoms)
    nhub = len(pti)
    return Workload(f"rutile-{reps[0]}x{reps[1]}x{reps[2]}-{len(atoms)}atoms-"
                    f"{grid[0]}x{grid[1]}x{grid[2]}-{n_occ + n_extra}orb",
                    tuple(grid), tuple(L), veff, atoms, ncol=n_occ + n_extra, degree=degree,
                    nspin=nspin, n_elec=float(2 * n_occ), kT=0.005,
                    D0=_spin_split_D0(nhub, nspin), seed_orbitals=20, seed_lanczos=30)


def rutile_snapshot(reps=(2, 2, 3), sigma: float = 0.1, seed: int = 0, h_target: float = 0.2,
                    degree: int = 24, U_ev: float = 3.5, nspin: int = 2,
                    occ_per_atom: float = 290 / 72, extra: float = 0.2) -> Workload:
    """A displaced rutile-shaped supercell (atoms moved by N(0, sigma) bohr) with one KB
    pseudopotential per species, grid spacing about h_target, occ_per_atom occupied orbitals
    per atom plus a fraction `extra` of buffer orbitals, spin-polarised: a member of the
    family whose SCF solutions train the warm-start model (3x3x4: 216 atoms, 132x132x112
    grid, 1044 orbitals)."""
    L, pti, po = _supercell(rutile_cell(), reps)
    pti = displaced(pti, sigma, 50_000 + seed)
    po = displaced(po, sigma, 60_000 + seed)
    atoms = _tio2_atoms(pti, po, U_ev, 4, species_gamma=True)
    grid = scaled_grid_for(L, h_target)
    veff = _tio2_potential(grid, L, atoms)
    n_occ = int(round(occ_per_atom * len(atoms)))
    ncol = n_occ + int(round(extra * n_occ))
    return Workload(f"rutile-snap{seed}-{reps[0]}x{reps[1]}x{reps[2]}-{len(atoms)}atoms-"
                    f"{grid[0]}x{grid[1]}x{grid[2]}-{ncol}orb",
                    tuple(grid), tuple(L), veff, atoms, ncol=ncol, degree=degree, nspin=nspin,
                    n_elec=float(2 * n_occ), kT=0.005, D0=_spin_split_D0(len(pti), nspin),
                    seed_orbitals=70_000 + seed, seed_lanczos=80_000 + seed)


def rutile_trajectory(reps=(1, 1, 2), nsteps: int = 6, amplitude: float = 0.1, period: float = 12.0,
                      seed: int = 0, **kw) -> list:
    """A smooth seeded trajectory of a rutile-shaped supercell: atom i at step t sits at
    R_i + a_i sin(2 pi t / period + phi_i), a_i ~ N(0, amplitude) per component and phi_i
    uniform, one Workload per step on the same grid (the local potential follows the atoms;
    the orbital and Lanczos seeds stay fixed).  Keyword arguments go to rutile_snapshot."""
    base = rutile_snapshot(reps, 0.0, seed, **kw)
    g = _rng(90_000 + seed)
    R0 = np.array([a.pos for a in base.atoms])
    amp = amplitude * g.standard_normal(R0.shape)
    phase = g.uniform(0.0, 2 * np.pi, (len(R0), 1))
    out = []
    for t in range(nsteps):
        R = R0 + amp * np.sin(2 * np.pi * t / period + phase)
        atoms = [Atom(a.species, R[i].copy(), kb_l=a.kb_l, kb_rs=a.kb_rs, kb_gamma=a.kb_gamma,
                      kb_rc=a.kb_rc, hub_l=a.hub_l, hub_rs=a.hub_rs, hub_rc=a.hub_rc, hub_U=a.hub_U)
                 for i, a in enumerate(base.atoms)]
        veff = _tio2_potential(base.n, base.L, atoms)
        out.append(Workload(f"{base.name}-md{t}", base.n, base.L, veff, atoms, ncol=base.ncol,
                            degree=base.degree, nspin=base.nspin, n_elec=base.n_elec, kT=base.kT,
                            D0=base.D0.copy(), seed_orbitals=base.seed_orbitals,
                            seed_lanczos=base.seed_lanczos))
    return out


def small_test_system(n=(20, 24, 28), L=None, ncol=37, natoms=3, nspin=1, seed=7,
                      kpt=(0.0, 0.0, 0.0), hub_rc=4.0, kb_rc=2.5) -> Workload:
    """A ragged, anisotropic grid with a few atoms: sizes that span several kernel tiles
    plus ragged tails, for parity tests that the oracle finishes in seconds."""
    if L is None:
        L = tuple(0.3 * v for v in n)
    g = _rng(seed)
    depths = g.uniform(-2.0, 0.0, 6)
    widths = g.uniform(0.5, 1.5, 6)
    centres = g.uniform(0.0, 1.0, (6, 3)) * np.asarray(L)
    veff = gaussian_potential(n, L, centres, depths, widths)
    atoms = []
    for i in range(natoms):
        pos = g.uniform(0.0, 1.0, 3) * np.asarray(L)
        hub = (i % 3) != 2
        atoms.append(Atom("Ti" if hub else "O", pos, kb_l=(0, 1, 2), kb_rs=(0.8, 0.8, 1.0),
                          kb_gamma=tuple(g.uniform(0.5, 2.0, 3)), kb_rc=kb_rc,
                          hub_l=2 if hub else -1, hub_rs=1.0, hub_rc=hub_rc,
                          hub_U=4.0 / HARTREE_EV if hub else 0.0))
    nhub = sum(1 for a in atoms if a.hub_l >= 0)
    D0 = np.zeros((nspin, nhub, 5, 5))
    for s in range(nspin):
        for i in range(nhub):
            A = g.uniform(-0.05, 0.05, (5, 5))
            D0[s, i] = 0.2 * np.eye(5) + 0.5 * (A + A.T)
    return Workload(f"test-{n[0]}x{n[1]}x{n[2]}-{natoms}atoms-{ncol}orb", tuple(n), tuple(L),
                    veff, atoms, ncol=ncol, degree=8, nspin=nspin, kpts=(tuple(kpt),),
                    n_elec=float(ncol if nspin == 1 else ncol // 2 * 2) * 0.5 * (2 if nspin == 1 else 1),
                    kT=0.005, D0=D0, seed_orbitals=seed + 100,
                    seed_lanczos=seed + 200)


def snapshot_batch(n_snap: int = 16, h_target: float = 0.2, seed0: int = 10,
                   sigma: float = 0.1, max_kpts: int = 4):
    """Perturbed rutile / anatase-shaped cells of 24-96 atoms with 1-4 k-points each."""
    sizes = [24, 36, 48, 72, 96]
    rut_reps = {24: (2, 2, 1), 36: (3, 2, 1), 48: (2, 2, 2), 72: (2, 2, 3), 96: (2, 2, 4)}
    ana_reps = {24: (2, 1, 1), 36: (3, 1, 1), 48: (2, 2, 1), 72: (3, 2, 1), 96: (2, 2, 2)}
    out = []
    for i in range(n_snap):
        nat = sizes[i % len(sizes)]
        is_rutile = (i % 2) == 0
        cell = rutile_cell() if is_rutile else anatase_cell()
        reps = rut_reps[nat] if is_rutile else ana_reps[nat]
        L, pti, po = _supercell(cell, reps)
        pti = displaced(pti, sigma, seed0 + i)
        po = displaced(po, sigma, seed0 + 1000 + i)
        atoms = _tio2_atoms(pti, po, 3.5, seed0 + 2000 + i)
        grid = scaled_grid_for(L, h_target)
        veff = _tio2_potential(grid, L, atoms)
        nk = 1 + (i % max_kpts)
        mp = [(0.25, 0.25, 0.25), (-0.25, 0.25, 0.25), (0.25, -0.25, 0.25),
              (0.25, 0.25, -0.25)]
        kpts = tuple(tuple(2.0 * np.pi * np.asarray(f) / np.asarray(L)) for f in mp[:nk])
        ncol = int(round(1.2 * 4 * nat))
        out.append(Workload(f"snap{i}-{'rutile' if is_rutile else 'anatase'}-{nat}atoms-"
                            f"{grid[0]}x{grid[1]}x{grid[2]}-{ncol}orb-{nk}k",
                            grid, tuple(L), veff, atoms, ncol=ncol, degree=24, nspin=1,
                            kpts=kpts, kweights=tuple([1.0 / nk] * nk),
                            n_elec=float(8 * nat), kT=0.005,
                            D0=_spin_split_D0(len(pti), 1), seed_orbitals=seed0 + 3000 + i,
                            seed_lanczos=seed0 + 4000 + i))
    return out
