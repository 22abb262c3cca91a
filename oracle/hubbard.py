"""Plain FP64 CPU oracle for real-space DFT+U Chebyshev-filtered subspace iteration.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA library against the
paper's definitions.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference leg may import it; the product path never does.  It shares no code
with the CUDA path (no kernels, headers, tables or constants); the two only consume the
same seeded inputs from the ``workloads`` package.

Everything is written as the plain definition, in float64 (complex128 at k != 0), with
numpy as the only helper: a library matmul / Cholesky / symmetric eigensolver may serve as
one step, nothing is blocked or fused.

Paper: "Real-space Hubbard-corrected density functional theory" (arXiv 2507.23612).
  * Sec. II.A.1, Eq. (E_U) .................... Dudarev Hubbard energy
  * Sec. II.A.1, Eq. (orbital_occup_ext) ...... occupation matrix D
  * Sec. II.A.1, Bloch-mapped atomic orbitals . image sum with Bloch phase
  * Sec. II.A.2, Eqs. (DerED) and V_U ......... Hubbard potential applied to orbitals
  * Sec. II.A.3, final force equation ......... Hubbard atomic forces (FD gradient form)
  * Sec. II.A.4, stress definition and result . Hubbard stress tensor (FD gradient form)
  * Sec. II.B, gradient weights equation ...... FD weights family, index wrap, quadrature
  * Sec. II.B, last paragraph ................. CheFSI + Pulay mixing, diagonal initial D
Readings where the paper is silent (Laplacian weights, filter recurrence, Rayleigh-Ritz
variant, smearing, mixing) are stated at each function.

Array conventions: grid functions are 1-D arrays of length Nd = n1*n2*n3, x-fastest
(index i1 + n1*(i2 + n2*i3)); blocks of orbitals are (Nd, ncol) arrays.
"""
from __future__ import annotations

from math import factorial, gamma as _gamma_fn, pi, sqrt
import numpy as np

# ----------------------------------------------------------------------------------------
# Sec. II.B: finite-difference weights
# ----------------------------------------------------------------------------------------


def fd_gradient_weights(n0: int, h: float = 1.0) -> np.ndarray:
    """First-derivative weights w~_p, p = 1..n0 (Sec. II.B, the gradient-weight equation):
    w~_p = (-1)^{p+1} (n0!)^2 / (h p (n0-p)! (n0+p)!).  The derivative is
    sum_p w~_p (f_{i+p} - f_{i-p})."""
    return np.array([(-1.0) ** (p + 1) * factorial(n0) ** 2 /
                     (h * p * factorial(n0 - p) * factorial(n0 + p)) for p in range(1, n0 + 1)])


def fd_laplacian_weights(n0: int):
    """Second-derivative weights for the 2*n0-th order centred stencil.

    The paper uses "high-order centered finite-differences" (Sec. II.B) and prints only the
    gradient weights.  Reading: the standard centred second-derivative weights of the same
    order, from the same closed-form family,
        c_p = 2 (-1)^{p+1} (n0!)^2 / (p^2 (n0-p)! (n0+p)!),   p = 1..n0,
        c_0 = -2 sum_{p=1}^{n0} 1/p^2,
    so that f'' ~ h^-2 [c_0 f_i + sum_p c_p (f_{i+p} + f_{i-p})].
    Returns (c0, array of c_1..c_n0)."""
    c = np.array([2.0 * (-1.0) ** (p + 1) * factorial(n0) ** 2 /
                  (p * p * factorial(n0 - p) * factorial(n0 + p)) for p in range(1, n0 + 1)])
    c0 = -2.0 * sum(1.0 / (p * p) for p in range(1, n0 + 1))
    return c0, c


# ----------------------------------------------------------------------------------------
# Sec. II.B: uniform grid, Bloch-periodic index wrap, trapezoidal quadrature
# ----------------------------------------------------------------------------------------


class Grid:
    """Orthogonal cell with side lengths L_a = n_a h_a (Sec. II.B); det(S) = 1."""

    def __init__(self, n, L, kpt=(0.0, 0.0, 0.0), n0: int = 6):
        self.n = tuple(int(v) for v in n)
        self.L = np.asarray(L, dtype=np.float64)
        self.h = self.L / np.asarray(self.n, dtype=np.float64)
        self.dV = float(np.prod(self.h))          # h1 h2 h3 det(S) with S = I
        self.kpt = np.asarray(kpt, dtype=np.float64)
        self.n0 = int(n0)
        self.Nd = int(np.prod(self.n))
        self.is_complex = bool(np.any(self.kpt != 0.0))

    def coords(self):
        """Cartesian coordinates (Nd, 3) of the nodes x = (i1 h1, i2 h2, i3 h3), 0-based."""
        i1, i2, i3 = np.meshgrid(np.arange(self.n[0]), np.arange(self.n[1]),
                                 np.arange(self.n[2]), indexing="ij")
        x = np.stack([i1 * self.h[0], i2 * self.h[1], i3 * self.h[2]], axis=-1)
        return x.transpose(2, 1, 0, 3).reshape(-1, 3)    # x-fastest flattening

    def integrate(self, f):
        """Trapezoidal rule on the periodic grid (Sec. II.B): h1 h2 h3 det(S) sum f.
        (The printed lower limit j = 2 of the middle sum is read as j = 1.)"""
        return self.dV * np.sum(f, axis=0)

    def inner(self, u, v):
        """<u|v> = int u^* v dx on the grid, for (Nd, p) and (Nd, q) blocks -> (p, q)."""
        return self.dV * (u.conj().T @ v)


def bloch_shift(F, grid: Grid, axis: int, p: int):
    """G(i) = F(i + p) along `axis` (0 = x, 1 = y, 2 = z), with the Bloch-periodic wrap of
    Sec. II.B: a node index outside the grid maps back with the Bloch factor, under the
    convention psi(x + L_a e_a) = exp(i k_a L_a) psi(x).  F is (Nd, ncol)."""
    n1, n2, n3 = grid.n
    ncol = F.shape[1]
    F4 = F.reshape(n3, n2, n1, ncol)          # [z, y, x, col]
    ax = 2 - axis
    n = grid.n[axis]
    j = np.arange(n) + p
    src = np.mod(j, n)
    wraps = (j - src) // n                    # how many cell lengths the index crossed
    G = np.take(F4, src, axis=ax)
    if grid.is_complex:
        phase = np.exp(1j * grid.kpt[axis] * grid.L[axis] * wraps)
        shape = [1, 1, 1, 1]
        shape[ax] = n
        G = G * phase.reshape(shape)
    return G.reshape(F.shape)


def laplacian(F, grid: Grid):
    """FD Laplacian of a block (Nd, ncol): sum_a h_a^-2 [c0 F + sum_p c_p (F_{+p} + F_{-p})]."""
    c0, c = fd_laplacian_weights(grid.n0)
    out = np.zeros_like(F)
    for axis in range(3):
        acc = c0 * F
        for p in range(1, grid.n0 + 1):
            acc = acc + c[p - 1] * (bloch_shift(F, grid, axis, p) + bloch_shift(F, grid, axis, -p))
        out = out + acc / grid.h[axis] ** 2
    return out


def gradient(F, grid: Grid, axis: int):
    """FD gradient component (Sec. II.B): sum_p w~_p (F_{+p} - F_{-p}) along `axis`."""
    w = fd_gradient_weights(grid.n0, grid.h[axis])
    out = np.zeros_like(F)
    for p in range(1, grid.n0 + 1):
        out = out + w[p - 1] * (bloch_shift(F, grid, axis, p) - bloch_shift(F, grid, axis, -p))
    return out


# ----------------------------------------------------------------------------------------
# Sec. II.A.1 and Sec. II.B: atom-centred localized functions
# ----------------------------------------------------------------------------------------


def real_solid_harmonics(l: int, d):
    """r^l Y_lm(d/|d|) for the real, orthonormal spherical harmonics, m = -l..l, without
    the Condon-Shortley sign (reading: the paper does not fix the convention; E_U and the
    spectrum are invariant under an orthogonal change of basis within a shell).
    d: (..., 3) displacement.  Returns (2l+1, ...)."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    if l == 0:
        return np.stack([np.full_like(x, 0.5 / sqrt(pi))])
    if l == 1:
        k = sqrt(3.0 / (4.0 * pi))
        return np.stack([k * y, k * z, k * x])
    if l == 2:
        k1 = 0.5 * sqrt(15.0 / pi)
        k0 = 0.25 * sqrt(5.0 / pi)
        k2 = 0.25 * sqrt(15.0 / pi)
        return np.stack([k1 * x * y, k1 * y * z, k0 * (2 * z * z - x * x - y * y),
                         k1 * x * z, k2 * (x * x - y * y)])
    raise ValueError("l > 2 not used")


def radial_norm(l: int, rs: float) -> float:
    """N such that int_0^inf (N r^l exp(-r^2/(2 rs^2)))^2 r^2 dr = 1."""
    return sqrt(2.0 / (_gamma_fn(l + 1.5) * rs ** (2 * l + 3)))


def atom_function_table(grid: Grid, R, channels, rc: float, moments: bool = False):
    """Grid table of one atom's localized functions, Bloch-periodically mapped.

    Sec. II.A.1: phi_{Ilm}(x, k) = sum_{images I~} phi^(|x - R_I~|) exp(-i k.(R_I - R_I~)).
    Reading: the radial argument is the distance to the image R_I~ = R_I + T and the phase
    is exp(i k.T); each image contributes only within the cutoff rc (the paper truncates
    by a value threshold, Sec. II.B; the workloads fix rc).
    channels: list of (l, rs).  Returns (idx, vals): idx = sorted grid indices touched by
    any image, vals = (len(idx), nproj) with projector order channel by channel, m = -l..l.
    With moments=True also mom (3, len(idx), nproj): the same image sum with each image's
    term multiplied by (x - R_I~)_b, the displacement from that image's centre (the moment
    integrals of the stress, Sec. II.A.4).
    """
    R = np.asarray(R, dtype=np.float64)
    nproj = sum(2 * l + 1 for l, _ in channels)
    dtype = np.complex128 if grid.is_complex else np.float64
    acc = np.zeros((grid.Nd, nproj), dtype=dtype)
    mom = np.zeros((3, grid.Nd, nproj), dtype=dtype) if moments else None
    touched = np.zeros(grid.Nd, dtype=bool)
    n = np.asarray(grid.n)
    # lattice translations whose sphere can meet the cell [0, L)
    tr = [np.arange(int(np.floor((-R[a] - rc) / grid.L[a])) - 1,
                    int(np.ceil((grid.L[a] - R[a] + rc) / grid.L[a])) + 2) for a in range(3)]
    for t1 in tr[0]:
        for t2 in tr[1]:
            for t3 in tr[2]:
                T = np.array([t1, t2, t3]) * grid.L
                c = R + T
                lo = np.maximum(np.ceil((c - rc) / grid.h).astype(int), 0)
                hi = np.minimum(np.floor((c + rc) / grid.h).astype(int), n - 1)
                if np.any(hi < lo):
                    continue
                i1, i2, i3 = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                                         np.arange(lo[2], hi[2] + 1), indexing="ij")
                i1, i2, i3 = i1.ravel(), i2.ravel(), i3.ravel()
                d = np.stack([i1 * grid.h[0], i2 * grid.h[1], i3 * grid.h[2]], axis=-1) - c
                r2 = np.sum(d * d, axis=-1)
                inside = r2 < rc * rc
                if not np.any(inside):
                    continue
                d, r2 = d[inside], r2[inside]
                g = i1[inside] + grid.n[0] * (i2[inside] + grid.n[1] * i3[inside])
                phase = np.exp(1j * np.dot(grid.kpt, T)) if grid.is_complex else 1.0
                col = 0
                for l, rs in channels:
                    vals = radial_norm(l, rs) * np.exp(-r2 / (2.0 * rs * rs)) * \
                        real_solid_harmonics(l, d)
                    acc[g, col:col + 2 * l + 1] += (phase * vals).T
                    if moments:
                        for b_ in range(3):
                            mom[b_, g, col:col + 2 * l + 1] += (phase * vals * d[:, b_]).T
                    col += 2 * l + 1
                touched[g] = True
    idx = np.nonzero(touched)[0]
    if moments:
        return idx, acc[idx], mom[:, idx]
    return idx, acc[idx]


class Hamiltonian:
    """Discretised DFT+U Kohn-Sham Hamiltonian of one spin channel at one k-point.

    H = -1/2 Lap_h + V_eff + sum_I sum_p gamma_Ip |chi_Ip><chi_Ip|
        + sum_I sum_{mm'} (U_I/2)(delta_mm' - 2 D^I_m'm) |phi_Im'><phi_Im|
    The last term is the Hubbard potential of Sec. II.A.2 (see `hubbard` for the index
    order); the KB-type nonlocal term has the same form (Sec. II.B: the DFT+U
    implementation mirrors the nonlocal pseudopotential)."""

    def __init__(self, grid: Grid, veff, atoms, D=None):
        self.grid = grid
        self.veff = np.asarray(veff, dtype=np.float64)
        self.kb = []       # (idx, vals, gamma per projector)
        self.hub = []      # (idx, vals, U)
        for a in atoms:
            if len(a.kb_l):
                idx, vals = atom_function_table(grid, a.pos, list(zip(a.kb_l, a.kb_rs)), a.kb_rc)
                gam = np.concatenate([[g] * (2 * l + 1) for l, g in zip(a.kb_l, a.kb_gamma)])
                self.kb.append((idx, vals, gam))
            if a.hub_l >= 0:
                idx, vals = atom_function_table(grid, a.pos, [(a.hub_l, a.hub_rs)], a.hub_rc)
                self.hub.append((idx, vals, a.hub_U))
        self.set_occupation(D)

    def set_occupation(self, D):
        nh = len(self.hub)
        self.D = np.zeros((nh, 5, 5)) if D is None else np.asarray(D).copy()

    def hubbard_coefficients(self, I: int):
        """M = (U/2)(delta - 2 D) for Hubbard atom I (Eq. DerED)."""
        U = self.hub[I][2]
        return 0.5 * U * (np.eye(self.D.shape[-1]) - 2.0 * self.D[I])

    # --- pieces of H -----------------------------------------------------------------
    def kinetic(self, X):
        return -0.5 * laplacian(X, self.grid)

    def local(self, X):
        return self.veff[:, None] * X

    def nonlocal_kb(self, X):
        Y = np.zeros(X.shape, dtype=np.result_type(X, self.kb[0][1] if self.kb else X))
        for idx, vals, gam in self.kb:
            C = self.grid.dV * (vals.conj().T @ X[idx])        # <chi_p|x>
            Y[idx] += vals @ (gam[:, None] * C)
        return Y

    def hubbard(self, X):
        """V_U X, the functional derivative of E_U (Sec. II.A.2: dE_U/dpsi_n^* = f_n V_U psi_n).

        Since d Tr(D^2) / dD_mm' = 2 D_m'm, the chain rule gives
            V_U x = sum_I sum_{mm'} (U_I/2)(delta_mm' - 2 D_m'm) phi_m' <phi_m|x>,
        i.e. the coefficient of phi_m' is [(U/2)(I - 2D) C]_m' with C_m = <phi_m|x>.
        Reading: the printed final equation carries D_mm' in that slot; the two agree for the
        real symmetric D of the Gamma point, and only the derivative form is consistent with
        E_U for the complex Hermitian D of a general k-point."""
        Y = np.zeros(X.shape, dtype=np.result_type(X, self.hub[0][1] if self.hub else X))
        for I, (idx, vals, U) in enumerate(self.hub):
            M = self.hubbard_coefficients(I)
            C = self.grid.dV * (vals.conj().T @ X[idx])        # C[m, n] = <phi_m|x_n>
            W = M @ C                                           # W[m', n] = sum_m M_m'm C_mn
            Y[idx] += vals @ W
        return Y

    def apply(self, X):
        X = np.asarray(X)
        squeeze = X.ndim == 1
        if squeeze:
            X = X[:, None]
        Y = self.kinetic(X) + self.local(X) + self.nonlocal_kb(X) + self.hubbard(X)
        return Y[:, 0] if squeeze else Y

    def dense(self):
        """The full Nd x Nd matrix, by applying H to the unit vectors (tiny grids only)."""
        dt = np.complex128 if self.grid.is_complex else np.float64
        return self.apply(np.eye(self.grid.Nd, dtype=dt))


# ----------------------------------------------------------------------------------------
# Sec. II.B, last paragraph: Chebyshev-filtered subspace iteration
# ----------------------------------------------------------------------------------------


def chebyshev_filter(ham: Hamiltonian, X, m: int, a: float, b: float, a_low: float):
    """Degree-m Chebyshev filter, scaled three-term recurrence.

    The paper cites CheFSI without printing the filter; reading: the scaled recurrence of
    Zhou, Saad, Tiago and Chelikowsky (2006), which returns p_m(H) X with
    p_m(t) = T_m((t - c)/e) / T_m((a_low - c)/e),  e = (b - a)/2,  c = (b + a)/2."""
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    sigma = e / (a_low - c)
    tau = 2.0 / sigma
    Y = (sigma / e) * (ham.apply(X) - c * X)
    for _ in range(2, m + 1):
        sigma_new = 1.0 / (tau - sigma)
        Ynew = (2.0 * sigma_new / e) * (ham.apply(Y) - c * Y) - (sigma * sigma_new) * X
        X, Y, sigma = Y, Ynew, sigma_new
    return Y


def chebyshev_T(m: int, t):
    """T_m(t): cos(m arccos t) on [-1, 1], (+-1)^m cosh(m arccosh |t|) outside."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1.0
    out[inside] = np.cos(m * np.arccos(t[inside]))
    ta = np.abs(t[~inside])
    out[~inside] = np.sign(t[~inside]) ** m * np.cosh(m * np.arccosh(ta))
    return out


def lanczos_bounds(ham: Hamiltonian, v0, steps: int):
    """k-step Lanczos from v0 (no reorthogonalisation).  Returns (smallest Ritz value,
    largest Ritz value + |beta_k|): the usual CheFSI bound estimate (reading: the paper does
    not print a bound rule)."""
    v = np.asarray(v0) / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    beta_prev = 0.0
    alphas, betas = [], []
    for _ in range(steps):
        w = ham.apply(v) - beta_prev * v_prev
        alpha = float(np.real(np.vdot(v, w)))
        w = w - alpha * v
        beta = float(np.linalg.norm(w))
        alphas.append(alpha)
        betas.append(beta)
        v_prev, v, beta_prev = v, w / beta, beta
    T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    ritz = np.linalg.eigvalsh(T)
    return float(ritz[0]), float(ritz[-1] + abs(betas[-1]))


def rayleigh_ritz(ham: Hamiltonian, X):
    """Cholesky-based Rayleigh-Ritz on span(X) (reading: the paper does not state the variant).
        S = <X|X> = L L^H,   H^ = L^-1 <X|H|X> L^-H  (symmetrised),   H^ = V diag(lam) V^H,
        X <- X L^-H V.
    Returns (ascending eigenvalues, rotated block).  Raises LinAlgError if S is not SPD."""
    g = ham.grid
    HX = ham.apply(X)
    S = g.inner(X, X)
    Hs = g.inner(X, HX)
    L = np.linalg.cholesky(S)
    Linv = np.linalg.inv(L)
    Hh = Linv @ Hs @ Linv.conj().T
    Hh = 0.5 * (Hh + Hh.conj().T)
    lam, V = np.linalg.eigh(Hh)
    Q = Linv.conj().T @ V
    return lam, X @ Q


# ----------------------------------------------------------------------------------------
# Sec. II.A.1: occupations, occupation matrices, Hubbard energy
# ----------------------------------------------------------------------------------------


def fermi_dirac(eigs, weights, kT: float, n_elec: float, degeneracy: float):
    """Occupations f in [0, 1] of every (channel, state): Fermi-Dirac with one chemical
    potential mu, found by bisection so that sum_channels w * degeneracy * sum_n f = n_elec.
    (Reading: the paper does not state its smearing.)  kT = 0 gives the step function: the
    lowest states, each holding w * degeneracy electrons of its channel, are filled until
    n_elec is reached (ties not split).
    eigs: list of 1-D arrays (one per channel), weights: list of channel weights."""
    if kT <= 0.0:
        allv = np.concatenate([np.asarray(e) for e in eigs])
        allw = np.concatenate([np.full(len(e), w) for e, w in zip(eigs, weights)])
        order = np.argsort(allv, kind="stable")
        f_all = np.zeros_like(allv)
        left, mu = n_elec, float(allv[order[0]])
        for i in order:
            if left <= 1e-12:
                break
            f_all[i] = 1.0
            left -= allw[i] * degeneracy
            mu = float(allv[i])
        out, o = [], 0
        for e in eigs:
            out.append(f_all[o:o + len(e)])
            o += len(e)
        return out, mu

    def count(mu):
        return sum(w * degeneracy * np.sum(0.5 * (1.0 - np.tanh((np.asarray(e) - mu) / (2 * kT))))
                   for e, w in zip(eigs, weights))
    lo = min(np.min(e) for e in eigs) - 50 * kT
    hi = max(np.max(e) for e in eigs) + 50 * kT
    for _ in range(200):
        mu = 0.5 * (lo + hi)
        if count(mu) < n_elec:
            lo = mu
        else:
            hi = mu
        if hi - lo < 1e-15:
            break
    mu = 0.5 * (lo + hi)
    return [0.5 * (1.0 - np.tanh((np.asarray(e) - mu) / (2 * kT))) for e in eigs], mu


def occupation_matrices(ham: Hamiltonian, X, f, kweight: float = 1.0):
    """D^I_mm' = sum_n w_k f_n <psi_n|phi_m'> <phi_m|psi_n>   (Eq. orbital_occup_ext).
    X: (Nd, ncol), f: (ncol,).  Returns (nhub, 2l+1, 2l+1)."""
    out = []
    for idx, vals, _ in ham.hub:
        C = ham.grid.dV * (vals.conj().T @ X[idx])            # C[m, n] = <phi_m|psi_n>
        D = np.zeros((C.shape[0], C.shape[0]), dtype=C.dtype)
        for m in range(C.shape[0]):
            for mp in range(C.shape[0]):
                D[m, mp] = kweight * np.sum(np.asarray(f) * np.conj(C[mp]) * C[m])
        out.append(D)
    return np.array(out)


def hubbard_forces(ham: Hamiltonian, X, f, kweight: float = 1.0, D=None):
    """Hubbard atomic forces from one (spin, k-point) set of orbitals (Sec. II.A.3, final
    force equation, with the derivative moved from the atomic orbitals onto the FD
    gradient of the orbitals):

        F_J = Re sum_{mm'} U_J (2 D_J,m'm - delta_mm') sum_n w_k f_n
                 <grad psi_n|phi_Jm'> <phi_Jm|psi_n>

    Reading: the chain rule through dE_U/dD_mm' = (U/2)(delta_mm' - 2 D_m'm) puts D_m'm
    inside the real part; the printed equation carries D_mm' outside it.  The two agree for
    the real symmetric D of the Gamma point; only this form is the derivative of E_U for a
    Hermitian complex D.  D defaults to the occupation matrices the Hamiltonian carries
    (the self-consistent D at convergence).  X: (Nd, ncol), f: (ncol,).
    Returns (nhub, 3) for the Hubbard atoms in order; the force on E_U of this term only
    (the caller sums spins and k-points, and doubles a spin-unpolarized channel)."""
    D = ham.D if D is None else np.asarray(D)
    f = np.asarray(f, dtype=np.float64)
    grads = [gradient(X, ham.grid, a) for a in range(3)]
    out = np.zeros((len(ham.hub), 3))
    for I, (idx, vals, U) in enumerate(ham.hub):
        C = ham.grid.dV * (vals.conj().T @ X[idx])               # <phi_m|psi_n>
        nm = C.shape[0]
        for a in range(3):
            G = ham.grid.dV * (vals.conj().T @ grads[a][idx])     # <phi_m|d_a psi_n>
            acc = 0.0
            for m in range(nm):
                for mp in range(nm):
                    coef = U * (2.0 * D[I][mp, m] - (1.0 if m == mp else 0.0))
                    # <grad psi_n|phi_m'> = conj(<phi_m'|grad psi_n>)
                    s = np.sum(f * np.conj(G[mp]) * C[m])
                    acc += np.real(coef * kweight * s)
            out[I, a] = acc
    return out


def hubbard_stress(ham: Hamiltonian, atoms, X, f, kweight: float = 1.0, D=None):
    """Hubbard stress tensor of one (spin, k-point) set of orbitals (Sec. II.A.4), in
    Ha/bohr^3, from the definition sigma_ab = (1/|Omega|) dE_U/dF_ab at fixed orbitals
    (carried along by the deformation) and the chain rule through D:
      sigma_ab = (1/|Omega|) sum_J (U_J/2) [ -delta_ab sum_mm' (delta_mm' - 2 D_m'm) D_mm'
                  - 2 Re sum_mm' (delta_mm' - 2 D_m'm) kweight sum_n f_n
                        conj(<phi_m'|psi_n>) <(x - R)_b phi_m|d_a psi_n> ]
    with the moment (x - R_I~)_b taken from each periodic image's own centre; in the
    delta_ab term (the volume change of the orbitals' normalisation) D_mm' is this block's
    own contribution kweight sum_n f_n <psi_n|phi_m'><phi_m|psi_n>, so that summing the
    blocks of all spins and k-points gives the stress of the full D (for one k-point with
    its weight it is the full D).
    Readings: the index order of D as for the force; the moment about the image centre
    (the printed (S^T x - S^T R_I') with a sum over images and Bloch phases; only the image
    centre makes the result independent of which image is called the atom); the 1/|Omega|
    of the definition (the printed final expression is dE_U/dF).  Orthogonal cell (S = I).
    atoms: the Hamiltonian's atoms (positions and Hubbard shells).  Returns (3, 3)."""
    D = ham.D if D is None else np.asarray(D)
    f = np.asarray(f, dtype=np.float64)
    g = ham.grid
    grads = [gradient(X, g, a) for a in range(3)]
    omega = g.Nd * g.dV
    sig = np.zeros((3, 3))
    J = 0
    for at in atoms:
        if at.hub_l < 0:
            continue
        idx, vals, mom = atom_function_table(g, at.pos, [(at.hub_l, at.hub_rs)], at.hub_rc, moments=True)
        U = at.hub_U
        C = g.dV * (vals.conj().T @ X[idx])                      # <phi_m|psi_n>
        nm = C.shape[0]
        A = np.array([[(1.0 if m == mp else 0.0) - 2.0 * D[J][mp, m] for mp in range(nm)]
                      for m in range(nm)])                      # A[m, m'] = delta - 2 D_m'm
        D_blk = kweight * np.einsum("n,mn,pn->mp", f, C, np.conj(C))   # this block's D_mm'
        trace_term = float(np.real(np.sum(A * D_blk)))            # sum_mm' A_mm' D_mm'
        for a in range(3):
            for b_ in range(3):
                Gm = g.dV * (mom[b_].conj().T @ grads[a][idx])   # <(x-R)_b phi_m|d_a psi_n>
                s = 0.0
                for m in range(nm):
                    for mp in range(nm):
                        s += np.real(A[m, mp] * kweight * np.sum(f * np.conj(C[mp]) * Gm[m]))
                sig[a, b_] += 0.5 * U * (-(1.0 if a == b_ else 0.0) * trace_term - 2.0 * s) / omega
        J += 1
    return sig


def hubbard_energy(D, U):
    """E_U = sum_I (U_I/2) Tr(D_I - D_I^2)   (Eq. E_U); D: (nspin, nhub, 5, 5) or (nhub, 5, 5)."""
    D = np.asarray(D)
    if D.ndim == 3:
        D = D[None]
    E = 0.0
    for s in range(D.shape[0]):
        for I in range(D.shape[1]):
            E += 0.5 * U[I] * float(np.real(np.trace(D[s, I]) - np.trace(D[s, I] @ D[s, I])))
    return E


def fermi_entropy(f):
    f = np.clip(np.asarray(f, dtype=np.float64), 1e-300, 1.0 - 1e-16)
    g = np.clip(1.0 - f, 1e-300, None)
    return -float(np.sum(f * np.log(f) + g * np.log(g)))


# ----------------------------------------------------------------------------------------
# Sec. II.B, last paragraph: SCF with Pulay mixing of D (model with fixed V_eff)
# ----------------------------------------------------------------------------------------


class Pulay:
    """Pulay (DIIS) mixing of a flat vector x with history `hist` and mixing parameter
    `beta` (Sec. II.B names Pulay mixing; the parameters are a reading)."""

    def __init__(self, hist: int = 7, beta: float = 0.3):
        self.hist, self.beta = hist, beta
        self.xs, self.rs = [], []

    def mix(self, x_in, x_out):
        x_in = np.asarray(x_in, dtype=np.float64).ravel()
        r = np.asarray(x_out, dtype=np.float64).ravel() - x_in
        self.xs.append(x_in)
        self.rs.append(r)
        self.xs, self.rs = self.xs[-self.hist:], self.rs[-self.hist:]
        k = len(self.rs)
        if k == 1:
            return x_in + self.beta * r
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
        return xbar + self.beta * rbar


def scf_model_a(grid_args, veff, atoms, D0, X0s, n_elec: float, kT: float, degree: int,
                lanczos_v0s, lanczos_steps: int = 10, max_iter: int = 60,
                first_passes: int = 3, tol_e_atom: float = 1e-5, tol_D: float = 1e-4,
                hist: int = 7, beta: float = 0.3, eig_solver: str = "chefsi"):
    """Self-consistent DFT+U with a fixed local potential ("model A"): the Hamiltonian depends
    on the orbitals only through D (Sec. II.A.2), D is updated every SCF iteration and
    mixed with Pulay (Sec. II.B, last paragraph).

    Per iteration and spin channel: Chebyshev filter of degree m with bounds from the
    previous Rayleigh-Ritz (first iteration: Lanczos, `first_passes` filter+RR passes), then
    Rayleigh-Ritz; then Fermi-Dirac occupations with one mu; then D_out; then Pulay.
    Energy (reading, fixed V_eff): E = sum f lam - sum_I Tr(M_in D_out) + E_U(D_out) - kT S.
    Converged when |dE|/N_atom < tol_e_atom twice in a row and max|D_out - D_in| < tol_D.
    eig_solver = "dense" replaces CheFSI by a full dense eigensolve (brute force check).
    Returns a dict with E, D, eigenvalues, f, mu, iterations and history."""
    nspin = len(X0s)
    grid = Grid(*grid_args)
    hams = [Hamiltonian(grid, veff, atoms) for _ in range(nspin)]
    U = np.array([h[2] for h in hams[0].hub])
    degeneracy = 2.0 if nspin == 1 else 1.0
    natoms = len(atoms)
    D_in = np.asarray(D0, dtype=np.float64).copy()
    Xs = [np.asarray(X, dtype=np.float64).copy() for X in X0s]
    ncol = Xs[0].shape[1]
    bounds = [None] * nspin
    mixer = Pulay(hist, beta)
    hist_E, hist_dD = [], []
    E_prev, small = None, 0
    for it in range(1, max_iter + 1):
        lams = []
        for s in range(nspin):
            hams[s].set_occupation(D_in[s])
            if eig_solver == "dense":
                w, V = np.linalg.eigh(hams[s].dense())
                lams.append(w[:ncol])
                Xs[s] = V[:, :ncol] / np.sqrt(grid.dV)
                continue
            passes = first_passes if it == 1 else 1
            for _ in range(passes):
                if bounds[s] is None:
                    lo, up = lanczos_bounds(hams[s], lanczos_v0s[s], lanczos_steps)
                    a_low, a, b = lo, lo + 0.1 * (up - lo), up
                    bounds[s] = [a_low, a, b]
                a_low, a, b = bounds[s]
                Y = chebyshev_filter(hams[s], Xs[s], degree, a, b, a_low)
                lam, Xs[s] = rayleigh_ritz(hams[s], Y)
                bounds[s] = [lam[0], lam[-1], b]
            lams.append(lam)
        f, mu = fermi_dirac(lams, [1.0] * nspin, kT, n_elec, degeneracy)
        D_out = np.array([occupation_matrices(hams[s], Xs[s], f[s]) for s in range(nspin)])
        D_out = np.real(D_out)
        e_band = sum(degeneracy * float(np.dot(f[s], lams[s])) for s in range(nspin))
        e_dc = sum(degeneracy * float(np.sum(hams[s].hubbard_coefficients(I) * D_out[s, I]))
                   for s in range(nspin) for I in range(len(U)))
        e_u = degeneracy * hubbard_energy(D_out, U)
        ent = sum(degeneracy * fermi_entropy(f[s]) for s in range(nspin)) if kT > 0 else 0.0
        E = e_band - e_dc + e_u - kT * ent
        dD = float(np.max(np.abs(D_out - D_in)))
        hist_E.append(E)
        hist_dD.append(dD)
        if E_prev is not None and abs(E - E_prev) / natoms < tol_e_atom:
            small += 1
        else:
            small = 0
        E_prev = E
        if small >= 2 and dD < tol_D:
            return dict(E=E, E_U=e_u, E_band=e_band, D=D_out, D_in=D_in, eig=lams, f=f, mu=mu,
                        iterations=it, converged=True, hist_E=hist_E, hist_dD=hist_dD, X=Xs)
        D_in = mixer.mix(D_in, D_out).reshape(D_in.shape)
    return dict(E=E, E_U=e_u, E_band=e_band, D=D_out, D_in=D_in, eig=lams, f=f, mu=mu,
                iterations=max_iter, converged=False, hist_E=hist_E, hist_dD=hist_dD, X=Xs)


def build_hamiltonian(workload, spin: int = 0, kidx: int = 0):
    """Convenience: the oracle Hamiltonian of a `workloads.Workload` (spin, k-point)."""
    grid = Grid(workload.n, workload.L, workload.kpts[kidx], workload.fd_half_order)
    D = None if workload.D0 is None else workload.D0[spin]
    return Hamiltonian(grid, workload.veff, workload.atoms, D)


# ----------------------------------------------------------------------------------------
# Sec. II.B, last paragraph: occupation matrices across MD steps
# ----------------------------------------------------------------------------------------


def alfe_coefficients(R_hist):
    """(alpha, beta) of the second-order extrapolation, fitted to the atomic positions.
    R_hist: positions (natoms, 3) at t - 2dt, t - dt, t and t + dt (oldest first; the last
    are the positions of the step about to be solved).  Least squares over all coordinates:
        R(t+dt) - R(t) ~ alpha (R(t) - R(t-dt)) + beta (R(t-dt) - R(t-2dt)).
    Reading: the paper extrapolates the residual of D "to second order" as it does the
    density, citing Alfe's scheme; this is that scheme's fit.  With three position sets
    beta = 0 and alpha is fitted alone; with fewer, alpha = beta = 0."""
    R = [np.asarray(r, dtype=np.float64).ravel() for r in R_hist]
    if len(R) < 3:
        return 0.0, 0.0
    target = R[-1] - R[-2]
    d1 = R[-2] - R[-3]
    if len(R) == 3:
        den = float(np.dot(d1, d1))
        return (float(np.dot(d1, target)) / den if den > 0 else 0.0), 0.0
    d2 = R[-3] - R[-4]
    g11, g12, g22 = float(np.dot(d1, d1)), float(np.dot(d1, d2)), float(np.dot(d2, d2))
    det = g11 * g22 - g12 * g12
    if det <= 1e-12 * g11 * g22:       # parallel steps: the one-coefficient fit
        return (float(np.dot(d1, target)) / g11 if g11 > 0 else 0.0), 0.0
    b1, b2 = float(np.dot(d1, target)), float(np.dot(d2, target))
    return (g22 * b1 - g12 * b2) / det, (g11 * b2 - g12 * b1) / det


def extrapolate_occupations(D_hist, D_atomic, alpha: float, beta: float):
    """Starting D of the next MD step (Sec. II.B): the atomic guess plus the extrapolated
    residual Delta = D - D_atomic of the converged D of the previous steps (oldest first):
        Delta(t+dt) = Delta(t) + alpha (Delta(t) - Delta(t-dt)) + beta (Delta(t-dt) - Delta(t-2dt)).
    Terms whose history is missing are dropped (no history: the atomic guess)."""
    Da = np.asarray(D_atomic, dtype=np.float64)
    d = [np.asarray(D, dtype=np.float64) - Da for D in D_hist]
    if not d:
        return Da.copy()
    out = d[-1].copy()
    if len(d) >= 2:
        out += alpha * (d[-1] - d[-2])
    if len(d) >= 3:
        out += beta * (d[-2] - d[-3])
    return Da + out


def cutoff_for_threshold(l: int, rs: float, tau: float) -> float:
    """The radius beyond which the radial function N r^l exp(-r^2 / (2 rs^2)) stays below the
    value threshold tau (Sec. II.B: the radial orbitals are truncated where their value falls
    below a threshold).  The function rises to its maximum at r = rs sqrt(l) and decreases
    after it, so the answer is the root of N r^l exp(-r^2/(2 rs^2)) = tau beyond the
    maximum, found by bisection; 0 when tau exceeds the maximum."""
    N = radial_norm(l, rs)
    f = lambda r: N * r ** l * np.exp(-r * r / (2.0 * rs * rs))      # noqa: E731
    r_max = rs * sqrt(l)
    if f(r_max) <= tau:
        return 0.0
    lo, hi = r_max, r_max + rs
    while f(hi) > tau:
        hi += rs
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > tau:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def scf_model_a_kpoints(n, L, kpts, kweights, veff, atoms, D0, X0s, n_elec: float, kT: float,
                        degree: int, lanczos_v0s, n0: int = 6, lanczos_steps: int = 10,
                        max_iter: int = 60, first_passes: int = 3, tol_e_atom: float = 1e-5,
                        tol_D: float = 1e-4, hist: int = 7, beta: float = 0.3,
                        eig_solver: str = "chefsi"):
    """The fixed-V_eff SCF of scf_model_a with Brillouin-zone sampling: the occupation
    matrices are the weighted average over the k-points of Eq. (orbital_occup_ext),
    D = sum_k w_k D_k (sum w_k = 1), one Fermi level for all (spin, k) channels, and the
    Hamiltonian of every k-point carries the same D (complex Hermitian in general; its real
    and imaginary parts are mixed as one real vector).  A k-set with the Gamma point (real
    orbitals there) must be closed under k -> -k, which makes D real (D_-k = conj(D_k)).
    X0s[s][k], lanczos_v0s[s][k]: starting blocks (Nd, ncol) and Lanczos vectors per channel.
    Energy: E = sum w f lam - sum_I Re sum M_in o D_out^T + E_U(D_out) - kT S, with the spin
    degeneracy of one channel for both spins when nspin = 1."""
    nspin, nk = len(X0s), len(kpts)
    grids = [Grid(n, L, k, n0) for k in kpts]
    hams = [[Hamiltonian(grids[k], veff, atoms) for k in range(nk)] for _ in range(nspin)]
    U = np.array([h[2] for h in hams[0][0].hub])
    deg = 2.0 if nspin == 1 else 1.0
    D_in = np.asarray(D0, dtype=np.complex128).copy()
    Xs = [[np.asarray(X0s[s][k]).astype(np.complex128 if grids[k].is_complex else np.float64)
           for k in range(nk)] for s in range(nspin)]
    ncol = Xs[0][0].shape[1]
    bounds = [[None] * nk for _ in range(nspin)]
    mixer = Pulay(hist, beta)
    E_prev, small = None, 0
    for it in range(1, max_iter + 1):
        lams = [[None] * nk for _ in range(nspin)]
        if not all(g.is_complex for g in grids) and np.max(np.abs(D_in.imag)) > 1e-10:
            raise ValueError("a real (Gamma) k-point needs a real D: use a k-set closed under k -> -k")
        for s in range(nspin):
            for k in range(nk):
                ham = hams[s][k]
                ham.set_occupation(D_in[s] if ham.grid.is_complex else np.real(D_in[s]))
                if eig_solver == "dense":
                    w, V = np.linalg.eigh(ham.dense())
                    lams[s][k] = w[:ncol]
                    Xs[s][k] = V[:, :ncol] / np.sqrt(ham.grid.dV)
                    continue
                for _ in range(first_passes if it == 1 else 1):
                    if bounds[s][k] is None:
                        lo, up = lanczos_bounds(ham, lanczos_v0s[s][k], lanczos_steps)
                        bounds[s][k] = [lo, lo + 0.1 * (up - lo), up]
                    a_low, a, b = bounds[s][k]
                    Y = chebyshev_filter(ham, Xs[s][k], degree, a, b, a_low)
                    lam, Xs[s][k] = rayleigh_ritz(ham, Y)
                    bounds[s][k] = [lam[0], lam[-1], b]
                lams[s][k] = lam
        flat = [lams[s][k] for s in range(nspin) for k in range(nk)]
        wts = [kweights[k] for s in range(nspin) for k in range(nk)]
        fl, mu = fermi_dirac(flat, wts, kT, n_elec, deg)
        f = [[fl[s * nk + k] for k in range(nk)] for s in range(nspin)]
        D_out = np.zeros_like(D_in)
        for s in range(nspin):
            for k in range(nk):
                D_out[s] += occupation_matrices(hams[s][k], Xs[s][k], f[s][k], kweights[k])
        e_band = sum(deg * kweights[k] * float(np.dot(f[s][k], lams[s][k]))
                     for s in range(nspin) for k in range(nk))
        e_dc = sum(deg * float(np.real(np.sum(0.5 * U[I] * (np.eye(5) - 2.0 * D_in[s, I]) * D_out[s, I].T)))
                   for s in range(nspin) for I in range(len(U)))
        e_u = deg * hubbard_energy(D_out, U)
        ent = sum(deg * kweights[k] * fermi_entropy(f[s][k]) for s in range(nspin) for k in range(nk)) if kT > 0 else 0.0
        E = e_band - e_dc + e_u - kT * ent
        dD = float(np.max(np.abs(D_out - D_in)))
        small = small + 1 if (E_prev is not None and abs(E - E_prev) / len(atoms) < tol_e_atom) else 0
        E_prev = E
        res = dict(E=E, E_U=e_u, D=D_out, eig=lams, f=f, mu=mu, iterations=it, converged=False)
        if small >= 2 and dD < tol_D:
            res["converged"] = True
            return res
        x_in = np.concatenate([D_in.real.ravel(), D_in.imag.ravel()])
        x_out = np.concatenate([D_out.real.ravel(), D_out.imag.ravel()])
        x = mixer.mix(x_in, x_out)
        half = x.size // 2
        D_in = (x[:half] + 1j * x[half:]).reshape(D_in.shape)
    return res
