/*
 * hub.h -- C ABI of the GB300 (sm_103a) library for real-space DFT+U
 * Chebyshev-filtered subspace iteration (CheFSI).
 *
 * Paper: "Real-space Hubbard-corrected density functional theory" (arXiv 2507.23612).
 *   Sec. II.A.1  Dudarev energy E_U (Eq. E_U), occupation matrix D (Eq. orbital_occup_ext),
 *                Bloch-periodically mapped atomic orbitals.
 *   Sec. II.A.2  Hubbard potential V_U (Eq. DerED and the V_U equation).
 *   Sec. II.A.3  Hubbard atomic forces (final force equation, FD gradient form).
 *   Sec. II.B    uniform grid, 2*n0-th order centred finite differences, Bloch-periodic
 *                index wrap, trapezoidal quadrature, atom-by-atom projector integrals
 *                "computed simultaneously", CheFSI with Pulay mixing of D.
 *
 * Conventions shared by every call
 *   - Grid: orthogonal cell L_a = n_a h_a; node (i1,i2,i3) at (i1 h1, i2 h2, i3 h3);
 *     grid functions are flattened x-fastest: g = i1 + n1*(i2 + n2*i3); Nd = n1 n2 n3.
 *   - A block of ncol orbitals is column-major: element (g, j) at X[g + j*ld], ld >= Nd.
 *   - Element type of X/Y/work is fixed by the handle: HUB_F64 -> double, HUB_F32,
 *     HUB_MIXED_BF16 and HUB_MIXED_F16 -> float; with ncomplex = 1 it is the interleaved
 *     complex of that type (re, im).  Occupation matrices, eigenvalues and energies are
 *     always double.
 *   - Inner products carry the quadrature weight dV = h1 h2 h3: <u|v> = dV sum_g u_g^* v_g,
 *     so Rayleigh-Ritz returns orbitals with dV X^H X = I.
 *   - Ownership: array arguments marked "device" are caller-owned device memory (e.g.
 *     torch tensors); "host" arrays are caller-owned host memory.  The handle owns only its
 *     grid metadata, projector tables, occupation matrices and internal workspaces, all
 *     released by hub_destroy.
 *   - Streams: every call is ordered on the CUDA stream given at creation.  Calls that
 *     return host values (eigenvalues, D, bounds, SCF results) synchronise that stream;
 *     the others are asynchronous.
 *   - Errors: every function returns 0 (HUB_OK) or a negative hub_status; hub_last_error
 *     returns a message for the last failure on that handle.  Device-side checks (a
 *     non-SPD Gram matrix, a non-finite value, a bounded wait that ran out) surface at the
 *     next call that synchronises.
 */
#ifndef HUB_H
#define HUB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hub_ctx* hub_t;

typedef enum {
    HUB_OK = 0,
    HUB_EINVAL = -1,      /* bad argument: size, pointer, alignment, state order */
    HUB_ENOMEM = -2,      /* device or host allocation failed */
    HUB_ECUDA = -3,       /* a CUDA runtime call failed */
    HUB_ENOTSPD = -4,     /* Cholesky of the Gram matrix broke down */
    HUB_ENONFINITE = -5,  /* a NaN or Inf appeared in a result */
    HUB_ENOCONV = -6,     /* SCF or eigensolver did not converge within its limit */
    HUB_ETIMEOUT = -7     /* a bounded device wait ran out (the kernel returned early) */
} hub_status;

typedef enum {
    HUB_F64 = 0,          /* every step in double */
    HUB_F32 = 1,          /* filter and Rayleigh-Ritz products in float; dense steps double */
    HUB_MIXED_BF16 = 2,   /* float filter; X^T X (always the hi/lo BF16 split), X^T H X and
                             X Q as BF16 tensor-core products with float accumulation;
                             Cholesky, eigensolve, D and E_U double */
    HUB_MIXED_F16 = 3     /* as HUB_MIXED_BF16 with FP16 operands (11 significand bits, 22
                             with the hi/lo split): each operand block is scaled by a power
                             of two so that its largest magnitude lies in [2^14, 2^15) (FP16
                             overflows at 65504), the scale is removed from the FP32 result */
} hub_prec;

/* Create a handle for one grid, one Bloch wavevector and one precision.
 *   n1,n2,n3      grid points per axis (each >= 1)
 *   L1,L2,L3      cell side lengths in bohr (h_a = L_a / n_a)
 *   fd_half_order n0 of the 2*n0-th order centred Laplacian (Sec. II.B); 1 <= n0 <= 6
 *   ncomplex      0: real orbitals (Gamma point, kpt ignored); 1: complex Bloch orbitals
 *   kpt           Bloch wavevector (bohr^-1, Cartesian), host [3]; NULL means Gamma.
 *                 Wrap convention: psi(x + L_a e_a) = exp(i k_a L_a) psi(x).
 *   prec          hub_prec
 *   cuda_stream   cudaStream_t to order all work on (NULL = legacy default stream)
 * Errors: HUB_EINVAL (sizes), HUB_ENOMEM, HUB_ECUDA. */
int hub_create_grid(hub_t* out, int n1, int n2, int n3, double L1, double L2, double L3,
                    int fd_half_order, int ncomplex, const double* kpt, int prec,
                    void* cuda_stream);

/* Release every resource of the handle (synchronises its stream).  NULL is accepted. */
int hub_destroy(hub_t h);

/* Message of the last error on this handle (static string owned by the handle). */
const char* hub_last_error(hub_t h);

/* Local effective potential V_eff (Ha) on the grid, device double [Nd]; copied into the
 * handle (and rounded to float for HUB_F32 and the mixed handles). */
int hub_set_veff(hub_t h, const double* veff_dev);

/* Atoms and their localized functions (Sec. II.A.1 Bloch-mapped orbitals; Sec. II.B: the
 * Hubbard orbitals are handled like nonlocal pseudopotential projectors).  All host arrays.
 *   natoms           number of atoms
 *   pos              [natoms*3] Cartesian positions (bohr); any value, images are summed
 *   kb_nchan         [natoms] KB channels per atom (0 allowed)
 *   kb_l, kb_rs, kb_gamma   [sum kb_nchan] per channel: angular momentum l (0..2), Gaussian
 *                    width rs (bohr) of R(r) = N r^l exp(-r^2/(2 rs^2)), energy gamma (Ha)
 *   kb_rc            [natoms] KB cutoff radius (bohr)
 *   hub_l            [natoms] -1 = no Hubbard shell, else l (only 2 is supported)
 *   hub_rs, hub_rc, hub_U  [natoms] Hubbard radial width (bohr), cutoff (bohr), U (Ha)
 * Every localized function is radial(|x - R - T|) * real Y_lm (orthonormal, m = -l..l, no
 * Condon-Shortley sign) summed over lattice images T within the cutoff, with Bloch phase
 * exp(i k.T).  The tables are built on the device.  Resets the occupation matrices to 0.
 * Errors: HUB_EINVAL (l out of range, rc <= 0, NULL pointers with nonzero counts). */
int hub_set_atoms_projectors(hub_t h, int natoms, const double* pos,
                             const int* kb_nchan, const int* kb_l, const double* kb_rs,
                             const double* kb_gamma, const double* kb_rc,
                             const int* hub_l, const double* hub_rs, const double* hub_rc,
                             const double* hub_U);

/* Number of atoms that carry a Hubbard shell (the leading dimension of D arrays). */
int hub_num_hubbard_atoms(hub_t h, int* nhub);

/* Occupation matrices D^I of one spin channel (spin 0 or 1), host double
 * [nhub*5*5] row-major per atom (D_re; D_im is NULL at Gamma or a host array of the same
 * shape).  Sets the Hubbard coefficients M_I = (U_I/2)(I - 2 D_I) used by hub_apply_H for
 * that spin (Eq. DerED; coefficient of phi_m' is sum_m M_m'm <phi_m|psi>). */
int hub_set_occupation_matrix(hub_t h, int spin, const double* D_re, const double* D_im);

/* Mixed handles (HUB_MIXED_BF16, HUB_MIXED_F16): how the Rayleigh-Ritz block products
 * are taken.  t16 is the handle's 16-bit type (BF16: 8 significand bits; FP16: 11, after
 * the power-of-two scaling of each operand block described at HUB_MIXED_F16).
 * terms = 1: operands rounded to t16, one tensor-core product;
 * terms = 3: every float operand split as hi + lo (hi = t16(x), lo = t16(x - hi)) and
 *            the product taken as hi*hi + hi*lo + lo*hi (about 16 significand bits with
 *            BF16, 22 with FP16);
 * terms = 0: float products on CUDA cores (24 significand bits).
 * Tensor-core products accumulate in FP32.  Default 3.  Errors: HUB_EINVAL. */
int hub_set_bf16_terms(hub_t h, int terms);

/* Y = H X for ncol columns (device, column-major, leading dimension ld):
 *   H = -1/2 Lap_h + V_eff + sum_I sum_p gamma_Ip |chi_Ip><chi_Ip|
 *       + sum_I sum_mm' (U_I/2)(delta_mm' - 2 D_m'm) |phi_Im'><phi_Im|
 * X and Y must not overlap.  Errors: HUB_EINVAL (ncol < 0, ld < Nd, state not set). */
int hub_apply_H(hub_t h, int spin, const void* X, void* Y, int ncol, int ld);

/* Chebyshev filter in place: X <- p_m(H) X with
 *   p_m(t) = T_m((t - c)/e) / T_m((a_low - c)/e),  e = (b - a)/2,  c = (b + a)/2,
 * evaluated by the scaled three-term recurrence (CheFSI, Sec. II.B).  Requires
 * a_low < a < b.  work: device scratch of >= ld*ncol elements, or NULL to use a buffer
 * owned by the handle (allocated on first use).  Errors: HUB_EINVAL. */
int hub_chefsi_filter(hub_t h, int spin, void* X, int ncol, int ld, int degree,
                      double a, double b, double a_low, void* work);

/* Cholesky Rayleigh-Ritz in place (CheFSI, Sec. II.B):
 *   S = <X|X> = L L^H;  H^ = L^-1 <X|H|X> L^-H;  H^ = V diag(eig) V^H;  X <- X L^-H V.
 * eig_host: host double [ncol], ascending.  work: device scratch >= ld*ncol elements or
 * NULL (handle-owned).  Real orbitals (Gamma point) and complex Bloch orbitals (ncomplex =
 * 1: S and H^ are Hermitian, L is complex lower triangular with a real diagonal and the
 * eigensolver is a complex Jacobi).  Mixed handles take the block products of a complex
 * block in float on CUDA cores (the 16-bit tensor-core products are real only).
 * Errors: HUB_ENOTSPD (X rank-deficient), HUB_ENOCONV (Jacobi sweep limit),
 * HUB_ETIMEOUT, HUB_EINVAL. */
int hub_rayleigh_ritz(hub_t h, int spin, void* X, int ncol, int ld, double* eig_host,
                      void* work);

/* Block product of Rayleigh-Ritz (CheFSI, Sec. II.B): G = alpha * A^H B for two column
 * blocks A [ld x ncol_a] and B [ld x ncol_b] (device, handle element type), summed over the
 * Nd grid rows; with alpha = dV this is the overlap <A|B> (the Gram matrix S = <X|X>, or
 * <X|HX> with B = H X).  G_dev: device, row-major [ncol_a x ncol_b], overwritten: double
 * on a real handle, complex double (interleaved re/im, 2 * ncol_a * ncol_b doubles) on a
 * complex one.  When A == B and ncol_a == ncol_b only the upper tiles are computed and
 * mirrored (conjugated).  On real mixed handles the product runs on the BF16 or FP16
 * tensor cores (see hub_set_bf16_terms) with float accumulation.  Uses handle-owned
 * split-K scratch (allocated on first use).  Errors: HUB_EINVAL. */
int hub_gram(hub_t h, const void* A, int ncol_a, const void* B, int ncol_b, int ld,
             double alpha, double* G_dev);

/* hub_gram_noalloc: the hub_gram product for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a service entry point of the library.
 * Callers that cannot allocate: code running while a CUDA graph is being captured (a
 * cudaMalloc there is not allowed and would invalidate the capture), services that give
 * all device memory to a pooling allocator at start-up and forbid later cudaMalloc /
 * cudaFree (both synchronise the whole device and can fail once the pool holds the
 * memory), and callers that cannot create or keep a hub handle.  This call allocates
 * nothing: its split-K partial sums live in one static device array of 32 MiB
 * (4 Mi doubles) that every GPU which loads this library keeps until the process exits.
 *   G_dev[i*ncol_b + j] = alpha * sum_{g < nrows} A[g + i*ld] * B[g + j*ld]
 * A, B: device, real, double (prec = HUB_F64) or float (prec = HUB_F32), column-major
 * with leading dimension ld >= nrows; G_dev: device double, row-major
 * [ncol_a x ncol_b], overwritten; cuda_stream: the stream to run on (NULL = default).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current: make that first call before any stream capture.  The address
 * is kept for the life of the process and belongs to the device's primary context as it
 * was then: after cudaDeviceReset (or anything else that tears that context down) this
 * entry point must not be called again in the same process.  All calls on
 * a device share the one array and it keeps the last call's contents; every call writes
 * each partial sum it reads, so nothing needs clearing, but calls that overlap on the GPU
 * (two streams, or two host threads) race on the array and must be serialised.
 * Errors: HUB_EINVAL for bad arguments or when ncol_a * ncol_b exceeds 4 Mi (one split's
 * partial tile would not fit); HUB_ECUDA when a CUDA call fails. */
int hub_gram_noalloc(const void* A, int ncol_a, const void* B, int ncol_b, long long nrows,
                     int ld, int prec, double alpha, double* G_dev, void* cuda_stream);

/* Occupation matrices and Hubbard energy of one (spin, k) block (Eq. orbital_occup_ext,
 * Eq. E_U):  D^I_mm' = kweight sum_n f_n <psi_n|phi_m'><phi_m|psi_n>,
 *            EU = sum_I (U_I/2) Tr(D^I - D^I D^I)   (of this D alone).
 * f_host: host double [ncol].  D_re_out: host double [nhub*25] (overwritten); D_im_out:
 * NULL or host [nhub*25] (zeros at Gamma); EU_out: NULL or host double.  Synchronises. */
int hub_occupation(hub_t h, int spin, const void* X, int ncol, int ld, const double* f_host,
                   double kweight, double* D_re_out, double* D_im_out, double* EU_out);

/* Fermi-Dirac occupations with one chemical potential over weighted states: f_i in [0, 1]
 * with sum_i w_i * degeneracy * f_i = n_elec, f_i = 1 / (1 + exp((eig_i - mu) / kT)), mu by
 * bisection; kT = 0 fills the lowest states (by weight) with f = 1 (ties not split).  w_i is
 * the k-point weight of state i (1 for one k-point).  Host arithmetic, no handle.
 * Errors: HUB_EINVAL (n < 1, NULL arrays, kT < 0, n_elec outside the states' capacity). */
int hub_fermi_dirac(int n, const double* eig, const double* w, double kT, double n_elec,
                    double degeneracy, double* f_out, double* mu_out);

/* Cutoff radius of the value-threshold truncation (Sec. II.B: a radial orbital is cut where
 * its value falls below a threshold): for R(r) = N r^l exp(-r^2 / (2 rs^2)) (N normalising
 * int R^2 r^2 dr to 1) the radius beyond which R < tau, i.e. the root beyond the maximum at
 * r = rs sqrt(l); 0 when tau exceeds the maximum.  Host arithmetic, no handle.
 * Errors: HUB_EINVAL (l outside 0..2, rs <= 0, tau <= 0, NULL output). */
int hub_cutoff_radius(int l, double rs, double tau, double* rc_out);

/* Number of projector rows of the handle's tables (KB-type rows and Hubbard rows, atom by
 * atom in the order of hub_set_atoms_projectors; per atom its KB channels, then its Hubbard
 * shell; m = -l..l within a channel). */
int hub_num_projectors(hub_t h, int* nproj);

/* Projector inner products of a block (Sec. II.B: all integrals of an atom computed
 * together): C_host[p * ncol + n] = dV <proj_p|x_n> for every row p of the tables
 * (complex handles: (re, im) pairs).  X device [ld x ncol], handle element type; C_host host
 * double [nproj * ncol] (x2 complex).  Needs hub_set_atoms_projectors only.  Synchronises. */
int hub_project(hub_t h, const void* X, int ncol, int ld, double* C_host);

/* The adjoint: Y[g, n] += alpha * sum_p proj_p(g) W[p, n] for a host coefficient matrix
 * W_host double [nproj * ncol] (x2 complex), rounded to the handle's working type.
 * Y device [ld x ncol].  Asynchronous (the coefficients are copied before return). */
int hub_expand(hub_t h, const double* W_host, int ncol, void* Y, int ld, double alpha);

/* Hubbard atomic forces of one (spin, k) block (Sec. II.A.3, final force equation, with
 * the derivative carried by the FD gradient of the orbitals of Sec. II.B):
 *   F_J,a = Re sum_mm' U_J (2 D_J,m'm - delta_mm') kweight sum_n f_n
 *             conj(<phi_Jm'|d_a x_n>) <phi_Jm|x_n>
 * with D the occupation matrices last set for `spin` (hub_set_occupation_matrix; the
 * self-consistent D).  This is -dE_U/dR_J of this block alone: the caller sums spins and
 * k-points and folds a spin degeneracy into kweight.
 * X: device block [ld x ncol] (handle element type).  f_host: host double [ncol].
 * F_host: host double [natoms * 3] (the atoms of hub_set_atoms_projectors, x, y, z),
 * overwritten; atoms without a Hubbard shell get 0.  work: NULL (internal workspace) or a
 * device buffer of at least ld * ncol elements of the handle type, which receives the
 * gradient blocks.  Synchronises.  Errors: HUB_EINVAL (bad arguments, NULL pointers),
 * HUB_ECUDA. */
int hub_hubbard_forces(hub_t h, int spin, const void* X, int ncol, int ld, const double* f_host,
                       double kweight, double* F_host, void* work);

/* Hubbard stress tensor of one (spin, k) block (Sec. II.A.4: sigma = (1/|Omega|) dE_U/dF,
 * the derivative carried by the FD gradient of the orbitals), Ha/bohr^3:
 *   sigma_ab = (1/|Omega|) sum_J [ -delta_ab sum_mm' M_m'm Dblk_mm'
 *              - 2 Re sum_mm' M_m'm kweight sum_n f_n conj(<phi_m'|x_n>) <(x - R_T)_b phi_m|d_a x_n> ]
 * with M = (U/2)(I - 2D) from the D last set for `spin`, Dblk = kweight sum_n f_n <x_n|phi_m'>
 * <phi_m|x_n> this block's own occupation, and the moment (x - R_T)_b about each periodic
 * image's centre.  Blocks of all spins and k-points add up to the stress of E_U.
 * sigma_host: host double [9], row-major (a, b), overwritten.  work: as for
 * hub_hubbard_forces.  Synchronises.  Errors: HUB_EINVAL, HUB_ECUDA. */
int hub_hubbard_stress(hub_t h, int spin, const void* X, int ncol, int ld, const double* f_host,
                       double kweight, double* sigma_host, void* work);

/* k-step Lanczos from the device vector v0 [Nd] (handle element type): returns the
 * smallest Ritz value and the largest Ritz value plus |beta_k| (the CheFSI bound
 * estimate).  1 <= steps <= 64.  Synchronises. */
int hub_lanczos_bound(hub_t h, int spin, int steps, const void* v0, double* lo_out,
                      double* up_out);

/* ---------------------------------------------------------------------------------
 * SCF driver with a fixed local potential (the Hamiltonian depends on the orbitals only
 * through D; D is updated every iteration and Pulay-mixed, Sec. II.B last paragraph).
 * Per iteration and spin: filter (bounds from the previous Rayleigh-Ritz; Lanczos and
 * first_passes filter+RR passes in the first iteration), Rayleigh-Ritz; then Fermi-Dirac
 * occupations with one chemical potential; D_out; energy
 *   E = sum f eig - sum_I Tr(M_in D_out) + E_U(D_out) - kT S;
 * then Pulay mixing of D.  Converged when |dE|/natoms < tol_e_atom in two consecutive
 * iterations and max|D_out - D_in| < tol_D.
 * --------------------------------------------------------------------------------- */
typedef struct {
    int nspin;            /* 1 (every state holds 2 electrons) or 2 (one each) */
    int ncol;             /* orbitals per spin */
    int ld;               /* leading dimension of the X blocks */
    int degree;           /* Chebyshev degree */
    int max_iter;
    int first_passes;     /* filter+RR passes in the first iteration */
    int lanczos_steps;
    int pulay_history;
    int natoms;           /* for the per-atom energy tolerance */
    double pulay_beta;
    double kT;            /* Ha; 0 = step occupations */
    double n_elec;
    double tol_e_atom;    /* Ha/atom */
    double tol_D;
    int ladder;           /* mixed handles only: 1 = one 16-bit tensor-core product per
                             Rayleigh-Ritz product until |dE|/natoms < ladder_tol, then float
                             products (hub_set_bf16_terms 0) for the remaining iterations;
                             0 = keep the handle's setting */
    double ladder_tol;    /* Ha/atom */
    /* self-consistent density (appended; zero-initialised parameters keep the fixed-V_eff
     * SCF).  density = 1: V_eff^s = V_loc + V_H[rho_in] + v_x^s[rho_in], V_loc the potential
     * last set by hub_set_veff; V_H from -Lap_h V_H = 4 pi (rho - mean rho) (mean zero, the
     * kinetic term's FD Laplacian); v_x local-density (Dirac-Slater) exchange, spin-scaled
     * for two channels; rho_in starts uniform (n_elec / volume); the upper filter bound is
     * re-estimated by Lanczos every iteration; Pulay (pulay_history, pulay_beta) on the
     * joint vector [rho, D] with the Kerker preconditioner (-Lap)(-Lap + kappa^2)^-1 on the
     * density block (Sec. II.B: preconditioned Pulay whose coefficients also mix D); energy
     *   E = sum f eig - sum_s int rho_out^s (V_H + v_x^s)[rho_in] + E_H[rho_out] + E_x[rho_out]
     *       - sum_I Tr(M_in D_out) + E_U(D_out) - kT S;
     * converged when, in addition, int |rho_out - rho_in| / n_elec < tol_rho.  From the first
     * density-mode iteration on, the handle's H uses the SCF's V_eff^s of each spin (also in
     * hub_apply_H and the filter) until hub_set_veff is called again. */
    int density;
    double kerker_kappa;  /* bohr^-1 (0.5 when 0) */
    double tol_rho;       /* (1e-4 when 0) */
    double cg_tol;        /* relative residual of the Poisson and Kerker CG solves (1e-10 when 0) */
} hub_scf_params;

typedef struct {
    int iter;             /* iterations done */
    int converged;        /* 1 once the criterion above holds */
    double E, E_band, E_U, dE, dD, mu;
    int bf16_terms;       /* products used in this iteration on mixed handles (1, 3, 0) */
    int jacobi_sweeps;    /* sweeps of the last subspace eigensolve */
    /* self-consistent density only (appended): Hartree and exchange energies of rho_out,
     * int |rho_out - rho_in| / n_elec, and the CG iterations of this iteration's solves */
    double E_H, E_x, drho;
    int cg_iters;
} hub_scf_result;

/* Start an SCF: X[nspin] device blocks (ld*ncol each; updated in place every iteration),
 * v0[nspin] device Lanczos start vectors [Nd], D0 host [nspin*nhub*25] starting D. */
int hub_scf_begin(hub_t h, const hub_scf_params* p, void* const* X, const void* const* v0,
                  const double* D0);
/* One SCF iteration; fills *res.  Synchronises.  Returns HUB_OK also when not converged. */
int hub_scf_iterate(hub_t h, hub_scf_result* res);
/* Run iterations until converged or max_iter; HUB_ENOCONV if max_iter was reached. */
int hub_scf_run(hub_t h, hub_scf_result* res);
/* Results of the last iteration: eig/occ host [nspin*ncol] (may be NULL),
 * D_out host [nspin*nhub*25] (may be NULL). */
int hub_scf_get(hub_t h, double* eig, double* occ, double* D_out);
/* Hubbard forces (and optionally the Hubbard stress) of the SCF's last iteration: the sum
 * over spin channels of hub_hubbard_forces / hub_hubbard_stress of the SCF's orbitals and
 * occupations (times 2 for one spin-unpolarized channel), with D = the last iteration's
 * D_out (the occupation of those orbitals), which becomes the handle's occupation matrix.
 * F_host host [natoms * 3]; sigma_host NULL or host [9].  Synchronises. */
int hub_scf_forces(hub_t h, double* F_host, double* sigma_host);

/* SCF with Brillouin-zone sampling over one handle per k-point (Eq. orbital_occup_ext:
 * D = sum_k w_k D_k; Sec. II.B: D updated and Pulay-mixed every iteration).  The handles
 * share the grid, the atoms, V_eff and the precision; each carries its own Bloch vector
 * (real handles for Gamma).  One Fermi level spans every (spin, k) state, each weighted
 * by w_k; every k-point's Hamiltonian carries the same D, complex Hermitian in general
 * (its real and imaginary parts are Pulay-mixed as one real vector); a real handle needs
 * a real D, so a k-set holding Gamma must be closed under k -> -k.  Per iteration and
 * channel: filter + Rayleigh-Ritz (first_passes in the first iteration; bounds as for
 * hub_scf_iterate), then D_out, the energy
 *   E = sum_{s,k,n} deg w_k f eig - sum Re Tr(M_in D_out) + E_U(D_out) - kT S,
 *   M_in = (U/2)(I - 2 D_in), deg = 2 for one spin channel, else 1,
 * and the convergence test of hub_scf_iterate (natoms, tol_e_atom, tol_D).
 * hubs[nk]: the handles (not owned; they must outlive the object); kweights[nk] >= 0,
 * summing to 1 (within 1e-12); p: as for hub_scf_begin (density must be 0; ladder
 * unused); X[nspin*nk] and v0[nspin*nk] device blocks / Lanczos vectors of each channel,
 * index s*nk + k, in the element type of handle k (updated in place); D0_re host
 * [nspin*nhub*25], D0_im NULL (zero) or host of the same shape.
 * Errors: HUB_EINVAL (bad arguments, handles that disagree). */
typedef struct hub_kscf* hub_kscf_t;
int hub_kscf_create(hub_kscf_t* out, int nk, hub_t const* hubs, const double* kweights,
                    const hub_scf_params* p, void* const* X, const void* const* v0,
                    const double* D0_re, const double* D0_im);
/* One iteration; fills *res (E, E_band, E_U, dE, dD, mu, iter, converged).  Synchronises.
 * Errors: a handle's status (its message in hub_kscf_last_error); HUB_EINVAL when a real
 * handle would get a D with an imaginary part above 1e-10. */
int hub_kscf_iterate(hub_kscf_t s, hub_scf_result* res);
/* Iterations until converged or max_iter (then HUB_ENOCONV). */
int hub_kscf_run(hub_kscf_t s, hub_scf_result* res);
/* Last iteration: eig, occ host [nspin*nk*ncol] (channel s*nk + k), D_re, D_im host
 * [nspin*nhub*25] (D_out); any may be NULL. */
int hub_kscf_get(hub_kscf_t s, double* eig, double* occ, double* D_re, double* D_im);
const char* hub_kscf_last_error(hub_kscf_t s);
int hub_kscf_destroy(hub_kscf_t s);
/* Batched form (many snapshots or cells at once): one iteration of each of nobj k-point
 * SCFs (distinct objects over distinct handles; one Chebyshev degree) whose Chebyshev
 * filters run together: per filter pass and spin, every (object, k) channel still due that
 * pass goes through one hub_batch_filter call (one CUDA graph), then each channel's
 * Rayleigh-Ritz, then each object's Fermi level, D, energy and mixing as in
 * hub_kscf_iterate.  Objects that have converged are left as they are.  res: host
 * [nobj].  cuda_stream: the stream of the batched filters.  Errors: as hub_kscf_iterate
 * and hub_batch_filter. */
int hub_kscf_iterate_batch(int nobj, hub_kscf_t* objs, hub_scf_result* res, void* cuda_stream);
/* Batched iterations until every object has converged (HUB_OK) or reached its max_iter
 * (HUB_ENOCONV; the message is on that object). */
int hub_kscf_run_batch(int nobj, hub_kscf_t* objs, hub_scf_result* res, void* cuda_stream);

/* Self-consistent density SCF: replace the starting density (uniform by default) before the
 * first iteration; rho_dev device double [Nd], the total density (split evenly between two
 * spin channels).  HUB_EINVAL outside density mode or after the first iteration. */
int hub_scf_set_density(hub_t h, const double* rho_dev);

/* Self-consistent density SCF: the output density of the last iteration, summed over the
 * spin channels, into rho_dev (device double [Nd]).  HUB_EINVAL when the SCF is not in
 * density mode.  Synchronises. */
int hub_scf_density(hub_t h, double* rho_dev);

/* Starting occupation matrices of the next MD step (Sec. II.B, last paragraph: D split into
 * the atomic guess and a residual extrapolated to second order, as for the density):
 *   Delta = D - D_atomic,
 *   Delta(t+dt) = Delta(t) + alpha (Delta(t) - Delta(t-dt)) + beta (Delta(t-dt) - Delta(t-2dt)),
 * (alpha, beta) the least-squares fit R(t+dt) - R(t) ~ alpha (R(t) - R(t-dt))
 * + beta (R(t-dt) - R(t-2dt)) over all coordinates (beta = 0 with alpha fitted alone when
 * the two steps are parallel or only three position sets are given; terms without history
 * are dropped; no history gives D_atomic).  Host arithmetic only, no handle, no GPU.
 *   n         numbers per D set (e.g. nspin * nhub * 25)
 *   nhist     converged D sets given, 0..3, oldest first: D_hist host [nhist * n]
 *   D_atomic  host [n]
 *   natoms, R_hist  host [(nhist + 1) * natoms * 3]: the positions of those steps and, last,
 *             of the step to be solved
 *   coef_out  NULL or host [2]: alpha, beta.   D_out host [n].
 * Errors: HUB_EINVAL (nhist outside 0..3, NULL arrays with nonzero sizes). */
int hub_extrapolate_occupations(int n, int nhist, const double* D_hist, const double* D_atomic,
                                int natoms, const double* R_hist, double* coef_out, double* D_out);

/* ---------------------------------------------------------------------------------
 * Grid-sized steps of the self-consistent density SCF (Sec. II.B, last paragraph: CheFSI
 * with preconditioned Pulay mixing; the functional pieces are readings, the paper does not
 * print E_DFT).  All vectors are device double [Nd], cell-periodic; the FD Laplacian is the
 * kinetic term's (order 2 n0, periodic).
 * --------------------------------------------------------------------------------- */
/* rho[g] += scale * sum_n f_n |x_n(g)|^2 for one (spin, k) block X (handle element type,
 * [ld x ncol]); scale = spin degeneracy * k weight.  f_host host [ncol].  Accumulates:
 * the caller zeroes rho.  Asynchronous. */
int hub_density(hub_t h, const void* X, int ncol, int ld, const double* f_host, double scale,
                double* rho_dev);
/* Hartree potential: -Lap_h V = 4 pi (rho - mean rho), mean V = 0, by conjugate gradients
 * (FP64) from the V given (warm start) to |r| <= tol |b|.  iters_out, EH_out (= 1/2 dV sum
 * rho V) may be NULL.  Synchronises.  HUB_ENOCONV when max_iter is reached. */
int hub_hartree(hub_t h, const double* rho_dev, double* V_dev, double tol, int max_iter,
                int* iters_out, double* EH_out);
/* Local-density exchange of one channel (rho1, vx1 NULL: the total density) or two spin
 * channels: v_x = -(4/3) k rho^(1/3), E_x = -k dV sum rho^(4/3), k = (3/4)(3/pi)^(1/3),
 * times 2^(1/3) for each channel of a spin-polarized pair.  Negative densities count as 0.
 * Ex_out (host) may be NULL.  Synchronises. */
int hub_lda_exchange(hub_t h, int nchan, const double* rho0, const double* rho1, double* vx0,
                     double* vx1, double* Ex_out);
/* Kerker preconditioner z = (-Lap_h)(-Lap_h + kappa^2)^-1 r by conjugate gradients on
 * (-Lap_h + kappa^2) z = -Lap_h r from z = 0 (the constant part of r is removed).
 * Synchronises.  HUB_ENOCONV when max_iter is reached. */
int hub_kerker(hub_t h, const double* r_dev, double* z_dev, double kappa, double tol, int max_iter,
               int* iters_out);

/* ---------------------------------------------------------------------------------
 * Batched filtering and tuning.
 * --------------------------------------------------------------------------------- */

/* Autotuner: times the candidate stencil tile shapes of this handle's kernel family on the
 * block X (device, ncol columns, leading dimension ld; X is only read), for
 * mixed handles the split-K factor of the tensor-core Gram product, and for real
 * float handles the projector form (point-major, 8x8x4 bricks on CUDA cores, or 8x8x4
 * bricks as TF32 tensor-core products for the gather or for gather and scatter; gather and
 * scatter timed together); keeps the fastest
 * for the handle and for every later handle of the same grid shape, precision and ncol
 * (process-wide cache).  variant_out: NULL or the chosen stencil variant.
 * Synchronises.  Errors: HUB_EINVAL. */
int hub_autotune(hub_t h, int spin, const void* X, int ncol, int ld, int* variant_out);
/* Tuning of this handle without timing: stencil_variant in 0 .. n_variants-1 (the tile
 * shapes the autotuner chooses from; 0 is the default), gemm_split >= 1 (split-K factor of
 * the tensor-core Gram product, in units of one wave of tiles), gather_form 0 (point-major
 * projector gather and scatter), 1 (8x8x4 brick form on CUDA cores; real float handles
 * only), 2 (the brick gather as tcgen05 products, D[128 orbitals x functions] = X_b^T Phi_b
 * in TF32 with both operands split hi + lo and FP32 accumulation, the brick scatter on CUDA
 * cores) or 3 (gather and scatter both as tcgen05 products; the scatter per brick and 128
 * orbitals, D[128 points x 128 orbitals] = Phi_b W_b^T, added to Y by TMA reduce-add).
 * Forms 2 and 3 need real float handles whose n1 is a multiple of 4 and blocks that start
 * on 16-byte boundaries with ld a multiple of 4.  hub_set_atoms_projectors sets form 3
 * where its tables exist, else 0.
 * Pass -1 to keep any of them.  Errors: HUB_EINVAL. */
int hub_set_tuning(hub_t h, int stencil_variant, int gemm_split, int gather_form);
/* Current tuning of the handle and the number of stencil variants of its kernel family
 * (any pointer may be NULL). */
int hub_get_tuning(hub_t h, int* stencil_variant, int* n_variants, int* gemm_split, int* gather_form);

/* Chebyshev filter of nsys independent systems (snapshots, Bloch wavevectors, spins) in
 * one CUDA graph (CheFSI, Sec. II.B): X_i <- p_m^(i)(H_i) X_i with the bounds
 * (a[i], b[i], a_low[i]) of system i, each a_low < a < b, on handles sys[i] (distinct,
 * same device, any grid, precision or k), spin[i], blocks X[i] (device, ncol[i] columns,
 * leading dimension ld[i]).  The first call for a set of (handle, block) pairs autotunes
 * every handle (hub_autotune), captures one chain of kernels per system on forked streams
 * into a graph (the chains run concurrently) and instantiates it; later calls with the same
 * handles, blocks and degree only copy the new filter coefficients to the device and
 * replay the graph.  Every kernel reads its recurrence coefficients from a device table, so
 * new bounds need no new capture.  A graph is rebuilt after a handle reallocates a
 * workspace or its projector tables.  Work runs on cuda_stream; the call synchronises it.
 * Errors: HUB_EINVAL, HUB_ENOMEM, HUB_ECUDA. */
int hub_batch_filter(int nsys, const hub_t* sys, const int* spin, void* const* X,
                     const int* ncol, const int* ld, int degree, const double* a,
                     const double* b, const double* a_low, void* cuda_stream);

/* ---------------------------------------------------------------------------------
 * Warm start.  The paper has no learned component; this model only proposes the starting
 * occupation matrices D of an SCF (Sec. II.B starts from a diagonal D), and the SCF still
 * converges to its own fixed point.  Descriptors of a Hubbard atom (per neighbour species,
 * over periodic images within rc, cosine cutoff fc(r) = (cos(pi r/rc) + 1)/2):
 *   nrad radial Gaussians exp(-(r - mu_k)^2/(2 eta^2)) fc(r), mu_k = linspace(0.5, rc-0.5),
 *   then the sums of Y_1m(r/|r|) fc(r) (m = -1..1) and Y_2m(r/|r|) fc(r) (m = -2..2).
 * Model: n_in -> n_layers hidden layers of n_hidden (SiLU) -> n_out, with input and output
 * standardisation; FP32 master weights, an FP16 weight copy for the products when
 * weight_fp16, FP32 accumulation; loss = mean of ((y - t)/sd_out)^2; Adam (0.9, 0.999,
 * 1e-8).  Parameters are flat: for every layer W (out x in, row-major) then b (out).
 * All X / T / Y arrays are device float, row-major [batch x features].
 * --------------------------------------------------------------------------------- */
typedef struct hub_mlp_ctx* hub_mlp_t;

/* Descriptors of the centre atoms (host pos [natoms*3] bohr, species [natoms] in
 * 0..nspecies-1 (nspecies <= 2), L [3] orthogonal cell, centers [ncenter]) into out_dev
 * [ncenter x nspecies*(nrad+8)] float.  nrad <= 32.  Synchronises cuda_stream. */
int hub_descriptors(int natoms, const double* pos, const int* species, const double* L, int ncenter,
                    const int* centers, int nspecies, double rc, int nrad, double eta, float* out_dev,
                    void* cuda_stream);
/* Model with seeded initialisation U(-1/sqrt(in), 1/sqrt(in)) (SplitMix64 of seed + index). */
int hub_mlp_create(hub_mlp_t* out, int n_in, int n_hidden, int n_layers, int n_out, int weight_fp16,
                   unsigned long long seed, void* cuda_stream);
int hub_mlp_destroy(hub_mlp_t m);
const char* hub_mlp_last_error(hub_mlp_t m);
int hub_mlp_num_params(hub_mlp_t m, long long* n);
/* Host float [n_params] in / out; set also resets the Adam state. */
int hub_mlp_set_params(hub_mlp_t m, const float* host);
int hub_mlp_get_params(hub_mlp_t m, float* host);
/* Standardisation from host arrays, or fitted on the device to the columns of X and T. */
int hub_mlp_set_normalization(hub_mlp_t m, const float* mu_in, const float* sd_in,
                              const float* mu_out, const float* sd_out);
int hub_mlp_fit_normalization(hub_mlp_t m, const float* X_dev, const float* T_dev, int batch);
/* Y = model(X). */
int hub_mlp_forward(hub_mlp_t m, const float* X_dev, int batch, float* Y_dev);
/* Loss and gradient (host float [n_params], NULL to skip) of the batch.  Synchronises. */
int hub_mlp_loss_grad(hub_mlp_t m, const float* X_dev, const float* T_dev, int batch, float* loss_host,
                      float* grad_host);
/* One Adam step on the batch; loss_host NULL or the loss before the step (synchronises). */
int hub_mlp_train_step(hub_mlp_t m, const float* X_dev, const float* T_dev, int batch, float lr,
                       float* loss_host);

/* ---------------------------------------------------------------------------------
 * Measurement.  Every kernel launch of a handle is counted; with profiling on, each launch
 * is also bracketed by a pair of CUDA events recorded on the handle's stream (the stream
 * the kernel runs on), so per-kernel device time can be read back without a profiler.
 * --------------------------------------------------------------------------------- */
typedef enum {
    HUB_K_STENCIL = 0,    /* fused FD Laplacian + V_eff + recurrence axpby */
    HUB_K_GATHER,         /* projector / orbital inner products */
    HUB_K_TRANSFORM,      /* reduction of gather partials + gamma / M coefficients */
    HUB_K_SCATTER,        /* projector scatter into H X */
    HUB_K_GRAM,           /* X^T Y split-K partial products */
    HUB_K_GRAM_REDUCE,    /* reduction of the split-K partials */
    HUB_K_ROTATE,         /* X Q */
    HUB_K_CHOLESKY,
    HUB_K_TRI_INVERSE,
    HUB_K_DGEMM,          /* small n x n products */
    HUB_K_JACOBI,         /* subspace eigensolver */
    HUB_K_EIG_MISC,       /* symmetrise, identity, sort */
    HUB_K_OCCUPATION,     /* D and E_U reduction; per-atom Hubbard force reduction */
    HUB_K_LANCZOS,        /* Lanczos vector updates and dot products */
    HUB_K_COPY,           /* block copies and conversions */
    HUB_K_TABLE,          /* projector table values */
    HUB_K_FORCE,          /* FD gradient of the orbitals (Hubbard forces) */
    HUB_K_DENSITY,        /* density SCF: density, Poisson / Kerker CG, exchange */
    HUB_K_COUNT
} hub_kernel_kind;

/* enable = 1: start recording events; 0: stop (records kept); -1: drop all records. */
int hub_profile(hub_t h, int enable);
/* Sum of recorded device time (ms) and number of recorded launches of one kernel kind.
 * Synchronises the handle's stream. */
int hub_profile_read(hub_t h, int kind, double* total_ms, long long* launches);
/* Kernels launched by this handle since it was created. */
int hub_launch_count(hub_t h, long long* launches);

/* Size of the projector tables of the handle (after hub_set_atoms_projectors):
 * function_points = sum over sites of (grid points in the site's support) x (functions),
 * the number of multiply-adds per column of one gather or scatter; site_points = sum of the
 * supports.  Either pointer may be NULL. */
int hub_projector_stats(hub_t h, long long* function_points, long long* site_points);

/* Measured FMA throughput of the device (GFLOP/s, multiply-add = 2 flop) in FP64 and FP32:
 * eight independent FMA chains per thread over a full grid, best of five timed launches on
 * cuda_stream.  The denominators of ALU-bound rooflines; the paper has no counterpart.
 * Synchronises.  Errors: HUB_ECUDA, HUB_ENOMEM. */
int hub_alu_peaks(double* fp64_gflops, double* fp32_gflops, void* cuda_stream);

/* Library build information: writes a short string (arch, version) into buf. */
int hub_version(char* buf, int len);

#ifdef __cplusplus
}
#endif

#endif /* HUB_H */
