"""Warm start of the DFT+U SCF from a learned guess of the Hubbard occupation matrices.

The SCF of Sec. II.B starts from an atomic guess of the occupation matrices D of every
Hubbard atom and updates and mixes D every iteration until it is self-consistent.  Here a
SiLU multilayer perceptron (hub_mlp_*: forward, backward and Adam in the library's own
kernels) maps descriptors of each Hubbard atom's neighbourhood (hub_descriptors) to the 15
unique entries of its 5x5 D per spin, and is trained on SCF solutions that the library
itself computes on displaced cells.  The SCF started from the predicted D converges to its
own fixed point: the model only saves iterations, and the plain SCF remains the fallback
and the arbiter of its error.  (The paper has no learned component.)

This module is argument marshalling and orchestration: descriptors, training, inference and
the SCF all run in the library's kernels.
"""
from __future__ import annotations

import time

import numpy as np

from .binding import HUB_F64, HUB_MIXED_BF16, MLP, Hub, descriptors, scf_params

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


def hubbard_descriptors(atoms, L, device):
    """Descriptors (device float [nhub, N_IN]) of the Hubbard atoms, in the order in which
    the library numbers them (atoms with hub_l >= 0, in input order)."""
    import torch
    pos = np.asarray([a.pos for a in atoms], dtype=np.float64)
    sp = np.asarray([SPECIES[a.species] for a in atoms], dtype=np.int32)
    centres = np.asarray([i for i, a in enumerate(atoms) if a.hub_l >= 0], dtype=np.int32)
    out = torch.empty((len(centres), N_IN), dtype=torch.float32, device=device)
    descriptors(pos, sp, np.asarray(L, dtype=np.float64), centres, out, nspecies=len(SPECIES),
                rc=RC, nrad=NRAD, eta=ETA)
    return out


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
            ladder = 1 if prec == HUB_MIXED_BF16 else 0
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
