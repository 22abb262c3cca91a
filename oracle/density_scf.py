"""Plain FP64 CPU oracle for the self-consistent density SCF ("model B"): the fixed-V_eff
SCF of `hubbard.scf_model_a` with the local potential made self-consistent too.

TEST INFRASTRUCTURE ONLY, under the same rules as `oracle.hubbard`: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import it; it shares nothing
with the CUDA path.

Paper: Sec. II.B, last paragraph: the ground state by CheFSI accelerated by real-space
preconditioned Pulay mixing, with the density's mixing coefficients applied to the
occupation matrices as well.  The paper's E_DFT (Eq. E_full_1) is a full semilocal
functional with pseudopotentials; its parts are not printed.  Readings (model B):
  * V_eff^s = V_loc + V_H[rho] + V_x^s[rho], V_loc the workload's fixed local potential;
  * rho(x) = g sum_k w_k sum_n f_n |psi_n(x)|^2 per spin channel (g = 2 when one channel
    stands for both spins), orbitals normalised as dV sum |psi|^2 = 1;
  * V_H: the periodic FD Poisson problem Lap_h V_H = -4 pi (rho - mean rho), mean V_H = 0
    (uniform neutralising background), with the same FD Laplacian as the kinetic term;
  * V_x: local-density (Dirac-Slater, alpha = 2/3) exchange;
  * preconditioner: the Kerker form P = (-Lap_h) (-Lap_h + kappa^2)^-1 on the density part
    of the residual, identity on the D part (the real-space preconditioner of the paper's
    reference applies this operator by a linear solve; here it is evaluated exactly);
  * Pulay on the joint vector [rho, D] with one set of coefficients (Sec. II.B);
  * initial density uniform, N_e / Omega (V_H = 0), initial D as in model A.
Each function states the definition it evaluates.
"""
from __future__ import annotations

from math import pi
import numpy as np

from . import hubbard as hb


# ----------------------------------------------------------------------------------------
# density, Hartree, exchange
# ----------------------------------------------------------------------------------------


def electron_density(X, f, grid: hb.Grid, degeneracy: float = 1.0, kweight: float = 1.0):
    """rho(x_g) = degeneracy * kweight * sum_n f_n |x_n(g)|^2 for X (Nd, ncol), f (ncol,)."""
    return degeneracy * kweight * np.sum(np.asarray(f)[None, :] * np.abs(X) ** 2, axis=1)


def laplacian_symbol(grid: hb.Grid):
    """Eigenvalue of the periodic FD Laplacian on each discrete Fourier mode of the grid,
    as an (n3, n2, n1) array in numpy's FFT order:
        sigma(q) = sum_a h_a^-2 [c0 + 2 sum_p c_p cos(p q_a h_a)],  q_a h_a = 2 pi j / n_a.
    (A real periodic grid function has no Bloch factor: the density and potentials are
    cell-periodic.)"""
    c0, c = hb.fd_laplacian_weights(grid.n0)
    parts = []
    for a in range(3):
        th = 2.0 * pi * np.fft.fftfreq(grid.n[a])          # q_a h_a
        s = c0 + 2.0 * sum(c[p - 1] * np.cos(p * th) for p in range(1, grid.n0 + 1))
        parts.append(s / grid.h[a] ** 2)
    sig = parts[2][:, None, None] + parts[1][None, :, None] + parts[0][None, None, :]
    sig[0, 0, 0] = 0.0       # c0 + 2 sum_p c_p = 0 exactly: the constant mode, not rounding
    return sig


def _to_cube(v, grid):
    return np.asarray(v).reshape(grid.n[2], grid.n[1], grid.n[0])


def hartree_potential(rho, grid: hb.Grid):
    """V_H with Lap_h V_H = -4 pi (rho - mean rho) and mean V_H = 0, solved exactly in the
    discrete Fourier basis (the FD Laplacian is diagonal there; its only zero mode is the
    constant, which the neutralising background removes)."""
    r = np.fft.fftn(_to_cube(rho, grid))
    sig = laplacian_symbol(grid)
    out = np.zeros_like(r)
    nz = np.abs(sig) > 0.0
    out[nz] = -4.0 * pi * r[nz] / sig[nz]
    return np.real(np.fft.ifftn(out)).reshape(-1)


def hartree_energy(rho, grid: hb.Grid):
    """E_H = 1/2 int rho V_H dx (the background's share makes it the energy of rho - mean)."""
    return 0.5 * grid.dV * float(np.dot(rho, hartree_potential(rho, grid)))


C_X = 0.75 * (3.0 / pi) ** (1.0 / 3.0)     # Dirac exchange constant, e_x = -C_X rho^(1/3)


def lda_exchange(rhos, grid: hb.Grid):
    """Local-density exchange of one or two spin densities.
    One channel (total density rho): E_x = -C_X int rho^(4/3), v_x = -(4/3) C_X rho^(1/3).
    Two channels: E_x = -2^(1/3) C_X sum_s int rho_s^(4/3), v_x^s = -(4/3) 2^(1/3) C_X rho_s^(1/3)
    (the spin-scaling relation E_x[a, b] = (E_x[2a] + E_x[2b]) / 2).
    Returns (list of v_x per channel, E_x)."""
    rhos = [np.clip(np.asarray(r, dtype=np.float64), 0.0, None) for r in rhos]
    k = C_X * (2.0 ** (1.0 / 3.0) if len(rhos) == 2 else 1.0)
    v = [-(4.0 / 3.0) * k * np.cbrt(r) for r in rhos]
    E = -k * grid.dV * sum(float(np.sum(r ** (4.0 / 3.0))) for r in rhos)
    return v, E


# ----------------------------------------------------------------------------------------
# preconditioned Pulay on [rho, D]
# ----------------------------------------------------------------------------------------


def kerker(r, grid: hb.Grid, kappa: float):
    """P r with P = (-Lap_h) (-Lap_h + kappa^2)^-1, exact in the discrete Fourier basis:
    long-wavelength density residuals are damped (P -> 0 as q -> 0, P -> 1 at large q); the
    constant mode (the total charge) is removed for every kappa, including kappa = 0."""
    rr = np.fft.fftn(_to_cube(r, grid))
    sig = -laplacian_symbol(grid)                       # >= 0, 0 only for the constant
    ratio = np.zeros_like(sig)
    nz = sig > 0.0
    ratio[nz] = sig[nz] / (sig[nz] + kappa * kappa)
    return np.real(np.fft.ifftn(rr * ratio)).reshape(-1)


class PreconditionedPulay:
    """Pulay (DIIS) mixing of x = [rho (nrho values), D (rest)] with history `hist`:
    coefficients c minimise |sum c_i r_i| subject to sum c_i = 1 over the stored
    (input, residual) pairs, then x_new = sum c_i x_i + beta * P(sum c_i r_i) with P the
    Kerker operator on the density block and the identity on the D block."""

    def __init__(self, grid: hb.Grid, nrho: int, hist: int = 7, beta: float = 0.3,
                 kappa: float = 0.5):
        self.grid, self.nrho, self.hist, self.beta, self.kappa = grid, nrho, hist, beta, kappa
        self.xs, self.rs = [], []

    def precondition(self, r):
        out = np.array(r, dtype=np.float64)
        nd = self.grid.Nd
        for s in range(self.nrho // nd):
            out[s * nd:(s + 1) * nd] = kerker(r[s * nd:(s + 1) * nd], self.grid, self.kappa)
        return out

    def mix(self, x_in, x_out):
        x_in = np.asarray(x_in, dtype=np.float64).ravel()
        r = np.asarray(x_out, dtype=np.float64).ravel() - x_in
        self.xs.append(x_in)
        self.rs.append(r)
        self.xs, self.rs = self.xs[-self.hist:], self.rs[-self.hist:]
        k = len(self.rs)
        A = np.zeros((k + 1, k + 1))
        for i in range(k):
            for j in range(k):
                A[i, j] = np.dot(self.rs[i], self.rs[j])
        A[k, :k] = A[:k, k] = 1.0
        rhs = np.zeros(k + 1)
        rhs[k] = 1.0
        coef = np.linalg.lstsq(A, rhs, rcond=None)[0][:k]
        xbar = sum(c * x for c, x in zip(coef, self.xs))
        rbar = sum(c * rr for c, rr in zip(coef, self.rs))
        return xbar + self.beta * self.precondition(rbar)


# ----------------------------------------------------------------------------------------
# energies and the SCF
# ----------------------------------------------------------------------------------------


def hubbard_double_counting(ham: hb.Hamiltonian, D_out):
    """sum_n f_n <psi_n|V_U|psi_n> of the channel = sum_I sum_{m'm} M_m'm D_out[m, m'] with
    M = (U/2)(I - 2 D_in) the coefficients the Hamiltonian carries (Eq. DerED)."""
    return float(np.real(sum(np.sum(ham.hubbard_coefficients(I) * D_out[I].T)
                             for I in range(len(ham.hub)))))


def direct_energy(grid: hb.Grid, hams, v_loc, Xs, fs, rhos, D_out, U, kT, degeneracy):
    """The model-B energy evaluated directly from the orbitals and their density:
        E = g sum_s sum_n f_n <psi_n| -1/2 Lap_h + V_loc + V_KB |psi_n>
            + E_H[rho] + E_x[rho] + g E_U(D_out) - kT S."""
    e_kin_loc_nl = 0.0
    for s, (ham, X, f) in enumerate(zip(hams, Xs, fs)):
        TX = ham.kinetic(X) + np.asarray(v_loc)[:, None] * X + ham.nonlocal_kb(X)
        e_kin_loc_nl += degeneracy * float(np.real(np.sum(np.asarray(f) * np.einsum(
            "gn,gn->n", X.conj(), TX)))) * grid.dV
    rho_tot = sum(rhos)
    e_h = hartree_energy(rho_tot, grid)
    _, e_x = lda_exchange(rhos, grid)
    e_u = degeneracy * hb.hubbard_energy(D_out, U)
    ent = sum(degeneracy * hb.fermi_entropy(f) for f in fs) if kT > 0 else 0.0
    return e_kin_loc_nl + e_h + e_x + e_u - kT * ent


def scf_model_b(grid_args, v_loc, atoms, D0, X0s, n_elec: float, kT: float, degree: int,
                lanczos_v0s, lanczos_steps: int = 10, max_iter: int = 80, first_passes: int = 3,
                tol_e_atom: float = 1e-5, tol_D: float = 1e-4, tol_rho: float = 1e-4,
                hist: int = 7, beta: float = 0.3, kappa: float = 0.5, eig_solver: str = "chefsi"):
    """Self-consistent density and occupation matrices (model B; readings in the module
    header).  One k-point (Gamma or a Bloch vector with weight 1).

    Per iteration: V_eff^s = V_loc + V_H[rho_in] + V_x^s[rho_in]; per spin channel a
    Chebyshev filter (lower bounds from the previous Rayleigh-Ritz, the upper bound from a
    fresh Lanczos run since V_eff moves) and Rayleigh-Ritz (or a dense eigensolve with
    eig_solver = "dense"); Fermi-Dirac occupations with one mu; D_out and rho_out; the
    Kohn-Sham energy in band-structure form
        E = E_band - sum_s int rho_out^s V_Hx^s[rho_in] + E_H[rho_out] + E_x[rho_out]
            - g sum_s sum_n f_n <V_U[D_in]> + g E_U(D_out) - kT S,
    which equals `direct_energy` at (rho_out, D_out) at every iteration; then Pulay on
    [rho, D] with the Kerker preconditioner.  Converged when |dE|/N_atom < tol_e_atom twice
    in a row, max|D_out - D_in| < tol_D and int|rho_out - rho_in| / N_e < tol_rho."""
    nspin = len(X0s)
    grid = hb.Grid(*grid_args)
    v_loc = np.asarray(v_loc, dtype=np.float64)
    hams = [hb.Hamiltonian(grid, v_loc, atoms) for _ in range(nspin)]
    U = np.array([h[2] for h in hams[0].hub])
    g_deg = 2.0 if nspin == 1 else 1.0
    natoms = len(atoms)
    omega = grid.Nd * grid.dV
    rho_in = [np.full(grid.Nd, n_elec / nspin / omega) for _ in range(nspin)]
    D_in = np.asarray(D0, dtype=np.float64).copy()
    Xs = [np.asarray(X).copy() for X in X0s]
    ncol = Xs[0].shape[1]
    lower = [None] * nspin
    mixer = PreconditionedPulay(grid, nspin * grid.Nd, hist, beta, kappa)
    hist_E, hist_direct, hist_drho = [], [], []
    E_prev, small = None, 0
    result = None
    for it in range(1, max_iter + 1):
        v_h = hartree_potential(sum(rho_in), grid)
        v_x, _ = lda_exchange(rho_in, grid)
        lams = []
        for s in range(nspin):
            hams[s].veff = v_loc + v_h + v_x[s]
            hams[s].set_occupation(D_in[s])
            if eig_solver == "dense":
                w, V = np.linalg.eigh(hams[s].dense())
                lams.append(w[:ncol])
                Xs[s] = V[:, :ncol] / np.sqrt(grid.dV)
                continue
            _, b = hb.lanczos_bounds(hams[s], lanczos_v0s[s], lanczos_steps)
            passes = first_passes if it == 1 else 1
            for _ in range(passes):
                if lower[s] is None:
                    lo, _ = hb.lanczos_bounds(hams[s], lanczos_v0s[s], lanczos_steps)
                    lower[s] = (lo, lo + 0.1 * (b - lo))
                a_low, a = lower[s]
                Y = hb.chebyshev_filter(hams[s], Xs[s], degree, a, b, a_low)
                lam, Xs[s] = hb.rayleigh_ritz(hams[s], Y)
                lower[s] = (lam[0], lam[-1])
            lams.append(lam)
        fs, mu = hb.fermi_dirac(lams, [1.0] * nspin, kT, n_elec, g_deg)
        D_out = np.real(np.array([hb.occupation_matrices(hams[s], Xs[s], fs[s]) for s in range(nspin)]))
        rho_out = [electron_density(Xs[s], fs[s], grid, g_deg) for s in range(nspin)]
        e_band = sum(g_deg * float(np.dot(fs[s], lams[s])) for s in range(nspin))
        e_dc_hx = sum(grid.dV * float(np.dot(rho_out[s], v_h + v_x[s])) for s in range(nspin))
        e_h = hartree_energy(sum(rho_out), grid)
        _, e_x = lda_exchange(rho_out, grid)
        e_dc_u = sum(g_deg * hubbard_double_counting(hams[s], D_out[s]) for s in range(nspin))
        e_u = g_deg * hb.hubbard_energy(D_out, U)
        ent = sum(g_deg * hb.fermi_entropy(fs[s]) for s in range(nspin)) if kT > 0 else 0.0
        E = e_band - e_dc_hx + e_h + e_x - e_dc_u + e_u - kT * ent
        E_dir = direct_energy(grid, hams, v_loc, Xs, fs, rho_out, D_out, U, kT, g_deg)
        dD = float(np.max(np.abs(D_out - D_in)))
        drho = grid.dV * float(sum(np.sum(np.abs(ro - ri)) for ro, ri in zip(rho_out, rho_in))) / n_elec
        hist_E.append(E)
        hist_direct.append(E_dir)
        hist_drho.append(drho)
        small = small + 1 if (E_prev is not None and abs(E - E_prev) / natoms < tol_e_atom) else 0
        E_prev = E
        result = dict(E=E, E_direct=E_dir, E_U=e_u, E_H=e_h, E_x=e_x, E_band=e_band,
                      D=D_out, D_in=D_in, rho=rho_out, rho_in=rho_in, eig=lams, f=fs, mu=mu,
                      iterations=it, converged=False, hist_E=hist_E, hist_direct=hist_direct,
                      hist_drho=hist_drho, X=Xs)
        if small >= 2 and dD < tol_D and drho < tol_rho:
            result["converged"] = True
            return result
        x_in = np.concatenate([np.concatenate(rho_in), D_in.ravel()])
        x_out = np.concatenate([np.concatenate(rho_out), D_out.ravel()])
        x_new = mixer.mix(x_in, x_out)
        nr = nspin * grid.Nd
        rho_in = [x_new[s * grid.Nd:(s + 1) * grid.Nd] for s in range(nspin)]
        D_in = x_new[nr:].reshape(D_in.shape)
    return result


# ----------------------------------------------------------------------------------------
# atom-centred density coefficients (the warm start's density targets)
# ----------------------------------------------------------------------------------------

DENSITY_WIDTHS = (0.5, 1.0, 2.0)     # bohr: s-type Gaussians per atom


def density_basis_atoms(atoms, widths=DENSITY_WIDTHS, rc_factor: float = 3.0):
    """The density basis as atoms whose only functions are s-type Gaussians
    N exp(-r^2 / (2 rs^2)) with the given widths, cut off at rc_factor * max(widths), summed
    over periodic images like every atom-centred function.  Reading: the paper has no learned
    component, so nothing fixes this basis of the warm start's density targets; three widths
    resolve the core, the bond and the tail of a TiO2 atom's density."""
    from workloads import Atom
    rc = rc_factor * max(widths)
    return [Atom(a.species, np.asarray(a.pos, dtype=np.float64), kb_l=(0,) * len(widths),
                 kb_rs=tuple(widths), kb_gamma=(0.0,) * len(widths), kb_rc=rc) for a in atoms]


def density_basis_matrix(grid: hb.Grid, basis_atoms):
    """Dense (Nd, natoms * K) matrix of the basis functions on the grid, atom by atom."""
    cols = []
    for a in basis_atoms:
        idx, vals = hb.atom_function_table(grid, a.pos, list(zip(a.kb_l, a.kb_rs)), a.kb_rc)
        B = np.zeros((grid.Nd, vals.shape[1]))
        B[idx] = np.real(vals)
        cols.append(B)
    return np.concatenate(cols, axis=1)


def fit_density_coefficients(grid: hb.Grid, basis_atoms, rho):
    """Least-squares coefficients c minimising int |rho - sum_i c_i g_i|^2 on the grid:
    the normal equations G c = b with G_ij = <g_i|g_j> and b_i = <g_i|rho> (trapezoidal
    inner products).  Returns (natoms, K)."""
    B = density_basis_matrix(grid, basis_atoms)
    G = grid.dV * (B.T @ B)
    b = grid.dV * (B.T @ np.asarray(rho, dtype=np.float64))
    return np.linalg.solve(G, b).reshape(len(basis_atoms), -1)


def expand_density(grid: hb.Grid, basis_atoms, coef, n_elec=None):
    """rho0 = sum_i c_i g_i on the grid; with n_elec, scaled so that int rho0 = n_elec
    (reading: the starting density of the SCF must carry the electron count)."""
    rho = density_basis_matrix(grid, basis_atoms) @ np.asarray(coef, dtype=np.float64).ravel()
    if n_elec is not None:
        rho = rho * (n_elec / (grid.dV * np.sum(rho)))
    return rho
