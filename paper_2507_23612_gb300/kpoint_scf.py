"""Fixed-potential DFT+U SCF with Brillouin-zone sampling, over one library handle per
k-point.

Eq. (orbital_occup_ext) averages the occupation matrices over the Brillouin zone: here
D = sum_k w_k D_k over a set of Bloch wavevectors with weights summing to one, one Fermi
level spans every (spin, k) channel (hub_fermi_dirac), and every k-point's Hamiltonian
carries the same D (Sec. II.B: D updated every SCF iteration and Pulay-mixed).  D is complex
Hermitian in general; a k-set holding the Gamma point (real orbitals there) must be closed
under k -> -k, which makes D real.

Every grid-sized step (Lanczos bounds, Chebyshev filter, Rayleigh-Ritz, occupation
matrices) is a library call; the host does the scalar work of the driver: the energy sums
and Pulay mixing of the 25 numbers per Hubbard atom and spin (real and imaginary parts as
one vector).
"""
from __future__ import annotations

import numpy as np

from .binding import HUB_F64, Hub, fermi_dirac


def _pulay(xs, rs, beta):
    """DIIS on the stored inputs xs and residuals rs: minimise |sum c_i r_i| with
    sum c_i = 1, then sum c_i (x_i + beta r_i); linear mixing for one entry or a singular
    system."""
    k = len(rs)
    if k > 1:
        A = np.zeros((k + 1, k + 1))
        A[:k, :k] = [[np.dot(a, b) for b in rs] for a in rs]
        A[k, :k] = A[:k, k] = 1.0
        rhs = np.zeros(k + 1)
        rhs[k] = 1.0
        try:
            c = np.linalg.solve(A, rhs)[:k]
            return sum(ci * (x + beta * r) for ci, x, r in zip(c, xs, rs))
        except np.linalg.LinAlgError:
            pass
    return xs[-1] + beta * rs[-1]


def _entropy(f):
    f = np.clip(np.asarray(f, dtype=np.float64), 1e-300, 1.0 - 1e-16)
    g = np.clip(1.0 - f, 1e-300, None)
    return -float(np.sum(f * np.log(f) + g * np.log(g)))


class KpointSCF:
    """The workload's cell on one handle per k-point (complex orbitals where k != 0)."""

    def __init__(self, wl, kpts, kweights, prec: int = HUB_F64, device=None, hub_factory=None):
        """hub_factory(k) -> a handle with the potential and atoms set (default: a library
        Hub on `device`); any object with the Hub methods the driver calls will do."""
        if abs(sum(kweights) - 1.0) > 1e-12 or len(kweights) != len(kpts):
            raise ValueError("one weight per k-point, summing to one")
        self.wl, self.kpts, self.kw = wl, [tuple(map(float, k)) for k in kpts], list(map(float, kweights))
        self.real_k = [not any(k) for k in self.kpts]
        if hub_factory is None:
            import torch
            dev = device or torch.device("cuda", 0)

            def hub_factory(k):
                hb = Hub(wl.n, wl.L, wl.fd_half_order, kpt=k, complex_=any(k), prec=prec)
                hb.set_veff(torch.tensor(wl.veff, dtype=torch.float64, device=dev))
                hb.set_atoms(wl.atoms)
                return hb
        self.hubs = [hub_factory(k) for k in self.kpts]
        self.U = np.array([a.hub_U for a in wl.atoms if a.hub_l >= 0])

    def close(self):
        for hb in self.hubs:
            hb.close()

    def _set_D(self, D):
        if any(self.real_k) and np.max(np.abs(D.imag)) > 1e-10:
            raise ValueError("a real (Gamma) k-point needs a real D: use a k-set closed under k -> -k")
        for hb, real in zip(self.hubs, self.real_k):
            for s in range(D.shape[0]):
                if real:
                    hb.set_occupation_matrix(s, np.real(D[s]))
                else:
                    hb.set_occupation_matrix(s, np.real(D[s]), np.imag(D[s]))

    def run(self, X0s, v0s, D0, n_elec: float, kT: float, degree: int, max_iter: int = 60,
            first_passes: int = 3, lanczos_steps: int = 10, tol_e_atom: float = 1e-5,
            tol_D: float = 1e-4, hist: int = 7, beta: float = 0.3):
        """X0s[s][k], v0s[s][k]: device starting blocks [ncol, Nd] and Lanczos vectors of each
        channel (the handle's element type; updated in place).  Returns E, E_U, D, the
        eigenvalues, occupations, Fermi level, iterations and convergence."""
        nspin, nk = len(X0s), len(self.kpts)
        deg = 2.0 if nspin == 1 else 1.0
        natoms = len(self.wl.atoms)
        D_in = np.asarray(D0, dtype=np.complex128).copy()
        bounds = [[None] * nk for _ in range(nspin)]
        xs, rs = [], []
        E_prev, small, res = None, 0, None
        for it in range(1, max_iter + 1):
            self._set_D(D_in)
            lams = [[None] * nk for _ in range(nspin)]
            for s in range(nspin):
                for k, hb in enumerate(self.hubs):
                    for _ in range(first_passes if it == 1 else 1):
                        if bounds[s][k] is None:
                            lo, up = hb.lanczos_bound(s, lanczos_steps, v0s[s][k])
                            bounds[s][k] = [lo, lo + 0.1 * (up - lo), up]
                        a_low, a, b = bounds[s][k]
                        hb.chefsi_filter(s, X0s[s][k], degree, a, b, a_low)
                        lam = hb.rayleigh_ritz(s, X0s[s][k])
                        bounds[s][k] = [lam[0], lam[-1], b]
                    lams[s][k] = lam
            ncol = len(lams[0][0])
            eig = np.concatenate([lams[s][k] for s in range(nspin) for k in range(nk)])
            wts = np.concatenate([np.full(ncol, self.kw[k]) for s in range(nspin) for k in range(nk)])
            f_all, mu = fermi_dirac(eig, wts, kT, n_elec, deg)
            f = [[f_all[(s * nk + k) * ncol:(s * nk + k + 1) * ncol] for k in range(nk)] for s in range(nspin)]
            D_out = np.zeros_like(D_in)
            for s in range(nspin):
                for k, hb in enumerate(self.hubs):
                    Dr, Di, _ = hb.occupation(s, X0s[s][k], f[s][k], self.kw[k])
                    D_out[s] += Dr + 1j * Di
            e_band = deg * float(np.sum(wts * f_all * eig))
            e_dc = deg * sum(float(np.real(np.sum(0.5 * self.U[I] * (np.eye(5) - 2.0 * D_in[s, I]) * D_out[s, I].T)))
                             for s in range(nspin) for I in range(len(self.U)))
            e_u = deg * sum(0.5 * self.U[I] * float(np.real(np.trace(D_out[s, I]) - np.trace(D_out[s, I] @ D_out[s, I])))
                            for s in range(nspin) for I in range(len(self.U)))
            ent = deg * sum(self.kw[k] * _entropy(f[s][k]) for s in range(nspin) for k in range(nk)) if kT > 0 else 0.0
            E = e_band - e_dc + e_u - kT * ent
            dD = float(np.max(np.abs(D_out - D_in))) if D_in.size else 0.0
            small = small + 1 if (E_prev is not None and abs(E - E_prev) / natoms < tol_e_atom) else 0
            E_prev = E
            res = {"E": E, "E_U": e_u, "D": D_out, "eig": lams, "f": f, "mu": mu, "iterations": it,
                   "converged": bool(small >= 2 and dD < tol_D)}
            if res["converged"]:
                return res
            x_in = np.concatenate([D_in.real.ravel(), D_in.imag.ravel()])
            x_out = np.concatenate([D_out.real.ravel(), D_out.imag.ravel()])
            xs.append(x_in)
            rs.append(x_out - x_in)
            xs, rs = xs[-hist:], rs[-hist:]
            x = _pulay(xs, rs, beta)
            half = x.size // 2
            D_in = (x[:half] + 1j * x[half:]).reshape(D_in.shape)
        return res
