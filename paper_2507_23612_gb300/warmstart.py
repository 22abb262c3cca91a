"""Warm start of the DFT+U SCF from a learned guess of the Hubbard occupation matrices.

The SCF of Sec. II.B starts from an atomic guess of the occupation matrices D of every
Hubbard atom and updates and mixes D every iteration until it is self-consistent.  Here a
SiLU multilayer perceptron (hub_mlp_*: forward, backward and Adam in the library's own
kernels) maps descriptors of each Hubbard atom's neighbourhood (hub_descriptors) to the 15
unique entries of its 5x5 D per spin, and is trained on SCF solutions that the library
itself computes on displaced cells.  For the self-consistent density SCF a second model per
species maps every atom's descriptors to the coefficients of its s-type Gaussian density
basis (DensityBasis: the least-squares fit of a converged density, by the library's
projector products), whose expansion is the SCF's starting density.  The SCF started from
the predicted guess converges to its own fixed point: the models only save iterations, and
the plain SCF remains the fallback and the arbiter of their error.  (The paper has no
learned component.)

This module is argument marshalling and orchestration: descriptors, training, inference and
the SCF all run in the library's kernels.
"""
from __future__ import annotations

import time

import numpy as np

from .binding import HUB_F64, HUB_MIXED_BF16, HUB_MIXED_F16, MLP, Hub, descriptors, scf_params

SPECIES = {"Ti": 0, "O": 1}
NRAD = 16
RC = 6.0
ETA = 0.4
N_IN = len(SPECIES) * (NRAD + 8)
_IU = np.triu_indices(5)


def pack_occupations(D) -> np.ndarray:
    """(nspin, nhub, 5, 5) -> (nhub, 15 * nspin): upper triangles, row by row, spin by spin."""
    D = np.asarray(D, dtype=np.float64)
    return np.concatenate([D[s][:, _IU[0], _IU[1]] for s in range(D.shape[0])], axis=1)


def unpack_occupations(Y, nspin: int) -> np.ndarray:
    """Inverse of pack_occupations; the result is symmetric by construction."""
    Y = np.asarray(Y, dtype=np.float64)
    D = np.zeros((nspin, Y.shape[0], 5, 5))
    for s in range(nspin):
        D[s][:, _IU[0], _IU[1]] = Y[:, 15 * s:15 * (s + 1)]
        D[s][:, _IU[1], _IU[0]] = Y[:, 15 * s:15 * (s + 1)]
    return D


def atom_descriptors(atoms, L, centres, device):
    """Descriptors (device float [len(centres), N_IN]) of the given atoms' neighbourhoods."""
    import torch
    pos = np.asarray([a.pos for a in atoms], dtype=np.float64)
    sp = np.asarray([SPECIES[a.species] for a in atoms], dtype=np.int32)
    centres = np.asarray(centres, dtype=np.int32)
    out = torch.empty((len(centres), N_IN), dtype=torch.float32, device=device)
    descriptors(pos, sp, np.asarray(L, dtype=np.float64), centres, out, nspecies=len(SPECIES),
                rc=RC, nrad=NRAD, eta=ETA)
    return out


def hubbard_descriptors(atoms, L, device):
    """Descriptors (device float [nhub, N_IN]) of the Hubbard atoms, in the order in which
    the library numbers them (atoms with hub_l >= 0, in input order)."""
    return atom_descriptors(atoms, L, [i for i, a in enumerate(atoms) if a.hub_l >= 0], device)


def scf_solve(wl, prec: int = HUB_F64, D0=None, tol_e_atom: float = 1e-5, tol_D: float = 1e-4,
              max_iter: int = 200, first_passes: int = 3, ladder: int | None = None, device=None,
              X0=None, keep_orbitals: bool = False):
    """One SCF of a workload (Gamma point, real orbitals) from D0 (default: its atomic guess)
    and the starting orbitals X0 (device tensors, one [ncol, Nd] block per spin, updated in
    place; default: the workload's seeded random orbitals).  Returns iterations, energies, the
    converged D, the wall time and, with keep_orbitals, the converged orbital blocks."""
    import torch
    dev = device or torch.device("cuda", 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hub = Hub(wl.n, wl.L, wl.fd_half_order, prec=prec)
    try:
        hub.set_veff(torch.tensor(wl.veff, device=dev))
        hub.set_atoms(wl.atoms)
        if X0 is None:
            Xs = [torch.tensor(wl.orbitals(s), device=dev).to(hub.dtype).contiguous() for s in range(wl.nspin)]
        else:
            Xs = list(X0)
        v0s = [torch.tensor(wl.lanczos_start(s), device=dev).to(hub.dtype).contiguous()
               for s in range(wl.nspin)]
        if ladder is None:
            ladder = 1 if prec in (HUB_MIXED_BF16, HUB_MIXED_F16) else 0
        p = scf_params(nspin=wl.nspin, ncol=wl.ncol, ld=wl.Nd, degree=wl.degree, max_iter=max_iter,
                       first_passes=first_passes, lanczos_steps=10, pulay_history=7, natoms=len(wl.atoms),
                       pulay_beta=0.3, kT=wl.kT if wl.kT > 0 else 0.005, n_elec=wl.n_elec,
                       tol_e_atom=tol_e_atom, tol_D=tol_D, ladder=ladder, ladder_tol=1e-4)
        hub.scf_begin(p, Xs, v0s, wl.D0 if D0 is None else D0)
        res = hub.scf_run()
        eig, occ, D = hub.scf_get()
        torch.cuda.synchronize()
        out = {"iterations": res["iter"], "converged": bool(res["converged"]), "E": res["E"],
               "E_U": res["E_U"], "band": float(np.sum(occ * eig)), "D": D,
               "seconds": time.perf_counter() - t0}
        if keep_orbitals:
            out["X"] = Xs
        return out
    finally:
        hub.close()


class OccupationModel:
    """MLP from Hubbard-atom descriptors to packed occupation matrices (15 per spin)."""

    def __init__(self, nspin: int, hidden: int = 256, layers: int = 3, fp16: bool = True, seed: int = 0):
        self.nspin = nspin
        self.mlp = MLP(N_IN, hidden, layers, 15 * nspin, fp16=fp16, seed=seed)
        self._X, self._T = [], []

    def add_solution(self, atoms, L, D):
        """One SCF solution: descriptors of its Hubbard atoms and their converged D (kept on
        the host until fit)."""
        import torch
        X = hubbard_descriptors(atoms, L, torch.device("cuda", 0)).cpu().numpy()
        T = pack_occupations(D).astype(np.float32)
        if X.shape[0] != T.shape[0]:
            raise ValueError("D does not match the Hubbard atoms")
        self._X.append(X)
        self._T.append(T)

    @property
    def n_samples(self) -> int:
        return sum(x.shape[0] for x in self._X)

    def fit(self, steps: int = 2000, lr: float = 2e-3, lr_final: float = 2e-5, batch: int = 256,
            seed: int = 0):
        """Adam on mini-batches of a once-shuffled training set (contiguous slices of it), with
        a cosine learning-rate decay; standardisation fitted to the training set.
        Returns the losses of the steps (every 50th step read back)."""
        import torch
        Xh = np.concatenate(self._X)
        n = Xh.shape[0]
        perm = np.random.Generator(np.random.PCG64(seed)).permutation(n)
        dev = torch.device("cuda", 0)
        X = torch.tensor(Xh[perm], device=dev).contiguous()
        T = torch.tensor(np.concatenate(self._T)[perm], device=dev).contiguous()
        self.mlp.fit_normalization(X, T)
        batch = min(batch, n)
        nb = max(1, n // batch)
        losses = []
        for it in range(steps):
            j = it % nb
            xb, tb = X[j * batch:(j + 1) * batch], T[j * batch:(j + 1) * batch]
            lr_t = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * it / max(steps - 1, 1)))
            if it % 50 == 0 or it == steps - 1:
                losses.append(self.mlp.train_step(xb, tb, lr_t))
            else:
                self.mlp._check(self.mlp.lib.hub_mlp_train_step(
                    self.mlp.m, _ptr(xb), _ptr(tb), xb.shape[0], float(lr_t), None), "train_step")
        return losses

    def predict(self, atoms, L) -> np.ndarray:
        """Predicted D (nspin, nhub, 5, 5) for a new cell."""
        import torch
        X = hubbard_descriptors(atoms, L, torch.device("cuda", 0))
        Y = torch.empty((X.shape[0], 15 * self.nspin), dtype=torch.float32, device=X.device)
        self.mlp.forward(X, Y)
        return unpack_occupations(Y.cpu().numpy(), self.nspin)


def _ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------------------ density
DENSITY_WIDTHS = (0.5, 1.0, 2.0)     # bohr: s-type Gaussians per atom
DENSITY_RC_FACTOR = 3.0              # cutoff = factor * the widest Gaussian


class DensityBasis:
    """Atom-centred s-type Gaussian basis of the electron density on one grid and geometry,
    held as the projector tables of a separate library handle (three l = 0 channels per
    atom).  fit: least-squares coefficients of a density (normal equations with the basis
    Gram matrix; both sides from hub_project); expand: the density of given coefficients
    (hub_expand), scaled to carry n_elec electrons."""

    def __init__(self, wl, atoms=None, device=None, hub_factory=None):
        """hub_factory(basis_atoms) -> a handle whose tables hold the basis (default: an FP64
        library Hub on the workload's grid); any object with num_projectors / project /
        expand will do."""
        import torch
        from types import SimpleNamespace
        self.dev = device or torch.device("cuda", 0)
        self.atoms = wl.atoms if atoms is None else atoms
        K = len(DENSITY_WIDTHS)
        rc = DENSITY_RC_FACTOR * max(DENSITY_WIDTHS)
        basis = [SimpleNamespace(pos=np.asarray(a.pos, dtype=np.float64), kb_l=(0,) * K,
                                 kb_rs=DENSITY_WIDTHS, kb_gamma=(0.0,) * K, kb_rc=rc, hub_l=-1,
                                 hub_rs=1.0, hub_rc=0.0, hub_U=0.0) for a in self.atoms]
        self.K = K
        self.Nd, self.dV = wl.Nd, wl.dV
        if hub_factory is None:
            def hub_factory(atoms_):
                hb = Hub(wl.n, wl.L, wl.fd_half_order, prec=HUB_F64)
                hb.set_atoms(atoms_)
                return hb
        self.hub = hub_factory(basis)
        nb = self.hub.num_projectors()
        if nb != K * len(self.atoms):
            raise RuntimeError("density basis tables do not have K functions per atom")
        eye = torch.zeros((nb, self.Nd), dtype=torch.float64, device=self.dev)
        self.hub.expand(np.eye(nb), eye)                 # the basis functions, one per column
        self.G = self.hub.project(eye)                   # <g_i|g_j>
        del eye

    def fit(self, rho) -> np.ndarray:
        """Coefficients (natoms, K) of a device density [Nd]."""
        b = self.hub.project(rho.reshape(1, -1))[:, 0]
        return np.linalg.solve(self.G, b).reshape(len(self.atoms), self.K)

    def expand(self, coef, n_elec: float):
        """Device density [Nd] of the coefficients, scaled to integrate to n_elec."""
        import torch
        rho = torch.zeros((1, self.Nd), dtype=torch.float64, device=self.dev)
        self.hub.expand(np.asarray(coef, dtype=np.float64).reshape(-1, 1), rho)
        total = float(rho.sum()) * self.dV
        return (rho[0] * (n_elec / total)).contiguous()

    def close(self):
        self.hub.close()


def density_scf_solve(wl, prec: int = HUB_F64, D0=None, rho0=None, tol_e_atom: float = 1e-5,
                      tol_D: float = 1e-4, tol_rho: float = 1e-4, max_iter: int = 200, device=None):
    """Self-consistent density SCF of a workload (uniform starting density unless rho0, a
    device double [Nd] total density, is given).  Returns iterations, energies, D, the output
    density (device) and the wall time."""
    import torch
    dev = device or torch.device("cuda", 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hub = Hub(wl.n, wl.L, wl.fd_half_order, prec=prec)
    try:
        hub.set_veff(torch.tensor(wl.veff, device=dev))
        hub.set_atoms(wl.atoms)
        Xs = [torch.tensor(wl.orbitals(s), device=dev).to(hub.dtype).contiguous() for s in range(wl.nspin)]
        v0s = [torch.tensor(wl.lanczos_start(s), device=dev).to(hub.dtype).contiguous()
               for s in range(wl.nspin)]
        p = scf_params(nspin=wl.nspin, ncol=wl.ncol, ld=wl.Nd, degree=wl.degree, max_iter=max_iter,
                       first_passes=3, lanczos_steps=10, pulay_history=7, natoms=len(wl.atoms),
                       pulay_beta=0.3, kT=wl.kT if wl.kT > 0 else 0.005, n_elec=wl.n_elec,
                       tol_e_atom=tol_e_atom, tol_D=tol_D, ladder=1 if prec in (HUB_MIXED_BF16, HUB_MIXED_F16) else 0,
                       ladder_tol=1e-4, density=1, kerker_kappa=0.5, tol_rho=tol_rho, cg_tol=1e-10)
        hub.scf_begin(p, Xs, v0s, wl.D0 if D0 is None else D0)
        if rho0 is not None:
            hub.scf_set_density(rho0)
        res = hub.scf_run()
        eig, occ, D = hub.scf_get()
        rho = torch.empty(wl.Nd, dtype=torch.float64, device=dev)
        hub.scf_density(rho)
        torch.cuda.synchronize()
        return {"iterations": res["iter"], "converged": bool(res["converged"]), "E": res["E"],
                "E_U": res["E_U"], "D": D, "rho": rho, "seconds": time.perf_counter() - t0}
    finally:
        hub.close()


class DensityModel:
    """One MLP per species from an atom's descriptors to its K density coefficients."""

    def __init__(self, hidden: int = 256, layers: int = 3, fp16: bool = True, seed: int = 0):
        K = len(DENSITY_WIDTHS)
        self.K = K
        self.mlp = {sp: MLP(N_IN, hidden, layers, K, fp16=fp16, seed=seed + i)
                    for i, sp in enumerate(SPECIES)}
        self._X = {sp: [] for sp in SPECIES}
        self._T = {sp: [] for sp in SPECIES}

    def add_solution(self, atoms, L, coef):
        """Descriptors of every atom and its fitted coefficients (natoms, K)."""
        import torch
        X = atom_descriptors(atoms, L, range(len(atoms)), torch.device("cuda", 0)).cpu().numpy()
        coef = np.asarray(coef, dtype=np.float32)
        for sp in SPECIES:
            sel = [i for i, a in enumerate(atoms) if a.species == sp]
            if sel:
                self._X[sp].append(X[sel])
                self._T[sp].append(coef[sel])

    def fit(self, steps: int = 1500, lr: float = 2e-3, lr_final: float = 2e-5, batch: int = 256, seed: int = 0):
        """Adam with a cosine decay per species model; returns the last loss of each."""
        import torch
        dev = torch.device("cuda", 0)
        out = {}
        for sp, mlp in self.mlp.items():
            if not self._X[sp]:
                continue
            Xh, Th = np.concatenate(self._X[sp]), np.concatenate(self._T[sp])
            perm = np.random.Generator(np.random.PCG64(seed)).permutation(Xh.shape[0])
            X = torch.tensor(Xh[perm], device=dev).contiguous()
            T = torch.tensor(Th[perm], device=dev).contiguous()
            mlp.fit_normalization(X, T)
            b = min(batch, X.shape[0])
            nb = max(1, X.shape[0] // b)
            loss = None
            for it in range(steps):
                j = it % nb
                xb, tb = X[j * b:(j + 1) * b], T[j * b:(j + 1) * b]
                lr_t = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * it / max(steps - 1, 1)))
                if it == steps - 1:
                    loss = mlp.train_step(xb, tb, lr_t)
                else:
                    mlp._check(mlp.lib.hub_mlp_train_step(mlp.m, _ptr(xb), _ptr(tb), xb.shape[0],
                                                          float(lr_t), None), "train_step")
            out[sp] = loss
        return out

    def predict(self, atoms, L) -> np.ndarray:
        """Predicted coefficients (natoms, K)."""
        import torch
        dev = torch.device("cuda", 0)
        X = atom_descriptors(atoms, L, range(len(atoms)), dev)
        coef = np.zeros((len(atoms), self.K))
        for sp, mlp in self.mlp.items():
            sel = [i for i, a in enumerate(atoms) if a.species == sp]
            if not sel:
                continue
            Y = torch.empty((len(sel), self.K), dtype=torch.float32, device=dev)
            mlp.forward(X[sel].contiguous(), Y)
            coef[sel] = Y.cpu().numpy()
        return coef
