"""Fixed-potential DFT+U SCF with Brillouin-zone sampling, over one library handle per
k-point: a marshalling layer over the library's hub_kscf_* entry points.

Eq. (orbital_occup_ext) averages the occupation matrices over the Brillouin zone; the
library's driver takes D = sum_k w_k D_k over a set of Bloch wavevectors with weights summing
to one, one Fermi level over every (spin, k) channel, the same D in every k-point's
Hamiltonian (Sec. II.B: D updated every SCF iteration and Pulay-mixed), the energy sums and
the mixing.  D is complex Hermitian in general; a k-set holding the Gamma point (real
orbitals there) must be closed under k -> -k, which makes D real.  Several such SCFs (cells,
snapshots) can run batched: their filters go through one CUDA graph per pass
(hub_kscf_run_batch).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .binding import HUB_F64, Hub, HubError, _dptr, load_library, scf_params, scf_result


class KpointSCF:
    """The workload's cell on one handle per k-point (complex orbitals where k != 0)."""

    def __init__(self, wl, kpts, kweights, prec: int = HUB_F64, device=None):
        if abs(sum(kweights) - 1.0) > 1e-12 or len(kweights) != len(kpts):
            raise ValueError("one weight per k-point, summing to one")
        import torch
        dev = device or torch.device("cuda", 0)
        self.wl, self.kpts, self.kw = wl, [tuple(map(float, k)) for k in kpts], list(map(float, kweights))
        self.hubs = []
        for k in self.kpts:
            hb = Hub(wl.n, wl.L, wl.fd_half_order, kpt=k, complex_=any(k), prec=prec)
            hb.set_veff(torch.tensor(wl.veff, dtype=torch.float64, device=dev))
            hb.set_atoms(wl.atoms)
            self.hubs.append(hb)
        self.lib = load_library()
        self.obj = None

    def close(self):
        self._destroy()
        for hb in self.hubs:
            hb.close()

    def _destroy(self):
        if self.obj is not None:
            self.lib.hub_kscf_destroy(self.obj)
            self.obj = None

    def begin(self, X0s, v0s, D0, n_elec: float, kT: float, degree: int, max_iter: int = 60,
              first_passes: int = 3, lanczos_steps: int = 10, tol_e_atom: float = 1e-5,
              tol_D: float = 1e-4, hist: int = 7, beta: float = 0.3):
        """X0s[s][k], v0s[s][k]: device starting blocks [ncol, Nd] and Lanczos vectors of each
        channel (the handle's element type; updated in place by the iterations)."""
        self._destroy()
        nspin, nk = len(X0s), len(self.kpts)
        self.ncol, self.nspin = X0s[0][0].shape[0], nspin
        for s in range(nspin):
            for k, hb in enumerate(self.hubs):
                hb._blk(X0s[s][k], "k-point SCF X")
                hb._vec(v0s[s][k], hb.dtype, "k-point SCF v0")
        p = scf_params(nspin=nspin, ncol=self.ncol, ld=X0s[0][0].shape[1], degree=degree, max_iter=max_iter,
                       first_passes=first_passes, lanczos_steps=lanczos_steps, pulay_history=hist,
                       natoms=len(self.wl.atoms), pulay_beta=beta, kT=kT, n_elec=n_elec,
                       tol_e_atom=tol_e_atom, tol_D=tol_D)
        hs = (C.c_void_p * nk)(*[hb.h.value for hb in self.hubs])
        kw = np.ascontiguousarray(self.kw, dtype=np.float64)
        xa = (C.c_void_p * (nspin * nk))(*[X0s[s][k].data_ptr() for s in range(nspin) for k in range(nk)])
        va = (C.c_void_p * (nspin * nk))(*[v0s[s][k].data_ptr() for s in range(nspin) for k in range(nk)])
        D0 = np.asarray(D0, dtype=np.complex128)
        Dr = np.ascontiguousarray(D0.real, dtype=np.float64).reshape(-1)
        Di = np.ascontiguousarray(D0.imag, dtype=np.float64).reshape(-1)
        obj = C.c_void_p()
        rc = self.lib.hub_kscf_create(C.byref(obj), nk, hs, _dptr(kw), C.byref(p), xa, va, _dptr(Dr), _dptr(Di))
        if rc != 0:
            raise HubError(rc, "hub_kscf_create: handles or arguments disagree")
        self.obj = obj
        self._keep = (X0s, v0s)

    def _check(self, rc, what):
        if rc not in (0, -6):
            msg = self.lib.hub_kscf_last_error(self.obj)
            raise HubError(rc, f"{what}: {msg.decode() if msg else ''}")

    def result(self, r) -> dict:
        """E, E_U, D, eigenvalues, occupations, Fermi level, iterations and convergence of the
        last iteration (r: its scf_result)."""
        nspin, nk, ncol = self.nspin, len(self.kpts), self.ncol
        nh = self.hubs[0].nhub
        eig = np.zeros(nspin * nk * ncol)
        occ = np.zeros_like(eig)
        Dro = np.zeros(max(nspin * nh * 25, 1))
        Dio = np.zeros_like(Dro)
        self.lib.hub_kscf_get(self.obj, _dptr(eig), _dptr(occ), _dptr(Dro), _dptr(Dio))
        D = (Dro[:nspin * nh * 25] + 1j * Dio[:nspin * nh * 25]).reshape(nspin, nh, 5, 5)
        eig = eig.reshape(nspin, nk, ncol)
        occ = occ.reshape(nspin, nk, ncol)
        return {"E": r.E, "E_U": r.E_U, "D": D, "eig": [[eig[s, k] for k in range(nk)] for s in range(nspin)],
                "f": [[occ[s, k] for k in range(nk)] for s in range(nspin)], "mu": r.mu,
                "iterations": r.iter, "converged": bool(r.converged)}

    def run(self, X0s, v0s, D0, **kw) -> dict:
        """begin, then iterations until converged or max_iter (hub_kscf_run)."""
        self.begin(X0s, v0s, D0, **kw)
        try:
            r = scf_result()
            self._check(self.lib.hub_kscf_run(self.obj, C.byref(r)), "hub_kscf_run")
            return self.result(r)
        finally:
            self._destroy()


def run_batched(scfs, stream=None) -> list:
    """Run SCFs that have begun (KpointSCF.begin) together: per filter pass one CUDA graph over
    every channel of every SCF (hub_kscf_run_batch).  Returns each SCF's result."""
    import torch
    lib = load_library()
    n = len(scfs)
    objs = (C.c_void_p * n)(*[s.obj.value for s in scfs])
    res = (scf_result * n)()
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.hub_kscf_run_batch(n, objs, res, C.c_void_p(st.cuda_stream))
    if rc not in (0, -6):
        msgs = [lib.hub_kscf_last_error(s.obj) for s in scfs]
        raise HubError(rc, "hub_kscf_run_batch: " + "; ".join(m.decode() for m in msgs if m))
    return [s.result(res[i]) for i, s in enumerate(scfs)]
