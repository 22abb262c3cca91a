// Internal declarations of the hub library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define HUB_HAVE_NVTX 1
#endif
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/hub.h"

namespace hub {

constexpr int kMaxHalf = 8;      // largest supported n0
constexpr int kMaxProj = 9;      // most projectors one atom carries in one table (s+p+d)

// ---------------------------------------------------------------------------- errors
struct Error {
    int code;
    std::string msg;
};

#define HUB_CUDA_TRY(h, expr)                                                         \
    do {                                                                              \
        cudaError_t _e = (expr);                                                      \
        if (_e != cudaSuccess) {                                                      \
            return hub::fail((h), HUB_ECUDA, std::string(#expr) + ": " +              \
                                                  cudaGetErrorString(_e));            \
        }                                                                             \
    } while (0)

// ---------------------------------------------------------------------------- tables
// A "site" is one (atom, kind) pair: kind 0 = KB-type nonlocal projectors, kind 1 = a
// Hubbard shell.  Its points are table rows [pt_off, pt_off + npts) (grid index in idx);
// its values are point-major at vals[val_off + (row - pt_off) * nproj + p] (complex: pairs);
// its projector rows in C / W are [proj_off, proj_off + nproj).
struct SiteDev {
    double R[3];
    double rc;
    int tlo[3], thi[3];   // lattice translations whose sphere meets the cell
    int nch;
    int l[3];
    double rs[3];
    double N[3];
    int pt_off, npts, nproj, val_off, proj_off;
    int kind;
    int hub_index;        // Hubbard sites: index among Hubbard atoms, else -1
};

// Brick form of the projector tables (real float): the grid in bricks of 8 x 8 x 4 points
// (point p = x + 8 row of a brick, row = y + 8 z), at most BRF functions per entry.
constexpr int BRX = 8, BRY = 8, BRZ = 4, BRP = BRX * BRY * BRZ, BRF = 64;
// position of point p of a brick inside a function's 256 values: the two 4-point halves of
// the 32 rows are stored as two planes, [half][row][4], so that a warp reading one half of
// 32 consecutive rows touches 512 contiguous bytes
__host__ __device__ __forceinline__ int brick_slot(int p) {
    return ((p >> 2) & 1) * 128 + (p >> 3) * 4 + (p & 3);
}

struct Table {
    int nsites = 0, nproj = 0, npts = 0, nvals = 0, nhub = 0, nitems = 0;
    std::vector<SiteDev> h_sites;
    std::vector<int> h_hub_sites;     // site index of each Hubbard atom
    std::vector<int> h_hub_atom;      // atom index of each Hubbard atom
    int natoms = 0;
    std::vector<double> h_U;          // U per Hubbard atom (Ha)
    std::vector<int> h_item_first;    // first gather item of each site, size nsites + 1
    SiteDev* d_sites = nullptr;
    int* d_items = nullptr;           // [nitems*3]: site, first absolute row, count
    int* d_item_first = nullptr;
    int* d_idx = nullptr;             // [npts] grid index of each row
    void* d_vals = nullptr;           // working type, [nvals] (x2 complex)
    int* d_csr_off = nullptr;         // [Nd+1] entries per grid point
    int2* d_csr_ent = nullptr;        // per entry: x = value index of its first projector,
                                      // y = (projector row of its site << 4) | nproj
    int* d_order = nullptr;           // [norder] grid points with entries, grouped by the
    int norder = 0;                   // list of sites that touch them (scatter order)
    double* d_gamma = nullptr;        // [nproj] KB energy per projector row (0 for Hubbard)
    int* d_hub_sites = nullptr;
    double* d_U = nullptr;
    double* d_M[2] = {nullptr, nullptr};  // per spin [nhub*25] (x2 complex), row p, col m
    std::vector<double> h_M[2];
    // dense brick form (real float only): the grid in 8x8x4 bricks; per brick, entries of at
    // most 64 functions with their values as a dense [256 points][fp] block
    int dense = 0;                    // 1 when the brick tables below are built
    int nbx = 0, nby = 0, nbz = 0;
    int nbent = 0, nbused = 0;        // entries, bricks with at least one entry
    long npart_rows = 0;              // sum of fp over entries (gather partial rows)
    int4* d_bent = nullptr;           // per entry: brick, fp, value offset, partial row base
    int* d_bfirst = nullptr;          // [nbused + 1] first entry of each used brick
    float* d_phi = nullptr;           // dense values
    int* d_frow = nullptr;            // [npart_rows] global projector row (-1: padding)
    int* d_roff = nullptr;            // [nproj + 1] partial rows of each projector row (CSR)
    int* d_rent = nullptr;
    // tensor-core form of the brick gather (built with the bricks when n1 % 4 == 0): the
    // entries of each brick packed into groups of at most 64 functions, per group its values
    // in the 128-byte-swizzled K-major layout of tcgen05 operands, split as TF32 hi + lo,
    // function slots padded to a multiple of 16
    int tc = 0;                       // 1 when the arrays below are built
    int ntcg = 0;                     // groups
    int4* d_tcg = nullptr;            // per group: brick, float offset into d_tchi / d_tclo,
                                      // slots NP, first slot
    int* d_tcg_row = nullptr;         // per slot: partial row of its function (-1: padding)
    float* d_tchi = nullptr;
    float* d_tclo = nullptr;
    // tensor-core form of the brick scatter: per used brick (brick, float offset, function
    // slots), the W row of each slot (-1: padding), values point-major per 32-slot chunk
    int4* d_tcs_brick = nullptr;
    int* d_tcs_frow = nullptr;
    float* d_tcs_hi = nullptr;
    float* d_tcs_lo = nullptr;
};

// ---------------------------------------------------------------------------- profiling
struct ProfEvt {
    int kind;
    cudaEvent_t a, b;
};

// ---------------------------------------------------------------------------- handle
struct ScfState;
void free_table(Table& t);

}  // namespace hub

struct hub_ctx {
    int n1 = 0, n2 = 0, n3 = 0;
    int64_t Nd = 0;
    double L[3] = {0, 0, 0};
    double h[3] = {0, 0, 0};
    double dV = 0;
    int n0 = 6;
    int cplx = 0;
    double kpt[3] = {0, 0, 0};
    int prec = HUB_F64;
    int esize = 8;                // bytes per real component of the working type
    int bf16_terms = 3;           // mixed handles: 1 = one 16-bit product, 3 = hi/lo split products
    int stencil_variant = 0;      // tile shape chosen by the autotuner (stencil_variants)
    int gather_dense = 0;         // real float: gather in the brick form (else point-major)
    int gemm_split = 2;           // tensor-core split-K: CTAs per SM of the Gram products
    int capturing = 0;            // work is being captured into a CUDA graph
    long long mem_gen = 0;        // bumped whenever a workspace or table is reallocated
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;

    void* d_veff = nullptr;       // working type [Nd]
    bool veff_set = false;

    hub::Table proj;
    bool atoms_set = false;
    bool D_set[2] = {false, false};

    // workspaces (grown on demand)
    void* d_work = nullptr;       size_t work_bytes = 0;    // one X-sized block
    void* d_work2 = nullptr;      size_t work2_bytes = 0;   // second X-sized block
    void* d_part = nullptr;       size_t part_bytes = 0;    // gather partial sums
    void* d_C = nullptr;          size_t C_bytes = 0;       // projector coefficients
    void* d_W = nullptr;          size_t W_bytes = 0;
    void* d_small = nullptr;      size_t small_bytes = 0;   // n x n matrices (double)
    void* d_gpart = nullptr;      size_t gpart_bytes = 0;   // split-K GEMM partials
    void* d_bf16 = nullptr;       size_t bf16_bytes = 0;    // bf16 operand copies
    void* d_aux = nullptr;        size_t aux_bytes = 0;     // occupations and D output
    void* d_dens = nullptr;       size_t dens_bytes = 0;    // density SCF: CG vectors, partials
    // density SCF: per-spin V_eff in the working type (used by apply_H when veff_per_spin),
    // and the double buffers of the density model (V_loc, rho, V_H, v_x, Pulay history)
    void* d_veff_spin[2] = {nullptr, nullptr};
    int veff_per_spin = 0;
    double* d_rho_ws = nullptr;   size_t rho_ws_bytes = 0;
    double* d_vloc = nullptr;     size_t vloc_bytes = 0;    // double copy of the set V_eff
    int* d_flags = nullptr;       // [8] device error flags (0..5), Jacobi sweep count (6)
    unsigned int* d_bar = nullptr;  // [4] grid-barrier state
    double* d_scal = nullptr;     // [256] device scalars (Lanczos, reductions)
    unsigned* d_tcmax = nullptr;  // [4] max |x| bit patterns of the FP16 operands (scales)

    hub::ScfState* scf = nullptr;

    long long launches = 0;       // kernels launched by this handle
    int last_sweeps = 0;          // Jacobi sweeps of the last Rayleigh-Ritz (device slot 6)
    int prof_on = 0;              // record a CUDA event pair around every launch
    std::vector<hub::ProfEvt> prof;

    std::string last_error;
};

namespace hub {

int fail(hub_t h, int code, const std::string& msg);

// Counts one kernel launch; with profiling on, brackets it with CUDA events on the handle's
// stream (the stream the kernel runs on), so durations are measured where the work runs.
struct ProfScope {
    hub_t h;
    int kind;
    cudaEvent_t a = nullptr;
    ProfScope(hub_t h_, int k) : h(h_), kind(k) {
        h->launches++;
        if (h->prof_on && !h->capturing && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, h->stream);
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b;
        if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
        cudaEventRecord(b, h->stream);
        h->prof.push_back(ProfEvt{kind, a, b});
    }
};
int ensure(hub_t h, void** p, size_t* have, size_t need);

// An NVTX range around one ABI call (visible to Nsight tools; without a tool attached the
// calls return at once; compiled out where the toolkit has no NVTX headers)
struct NvtxRange {
#ifdef HUB_HAVE_NVTX
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
#else
    explicit NvtxRange(const char*) {}   // toolkits without the NVTX headers: no ranges
#endif
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// flags
enum { FLAG_NOTSPD = 0, FLAG_NONFINITE = 1, FLAG_TIMEOUT = 2, FLAG_NOCONV = 3 };
int check_flags(hub_t h);   // syncs stream, reads and clears flags, maps to a status

// ---------------------------------------------------------------------------- launchers
// stencil.cu
struct StencilArgs {
    const void* Y;       // current block
    const void* Yprev;   // previous block or nullptr (beta ignored)
    void* Yout;
    const void* V;       // working type [Nd]
    int n1, n2, n3, ld, ncol;
    double w[3][kMaxHalf];  // alpha * (-1/2) c_p / h_a^2
    double center;          // alpha * ((-1/2) c0 sum_a h_a^-2 - shift)
    double alpha;           // multiplies V
    double beta;
    int n0;
    double phase[3][2];     // exp(i k_a L_a) (re, im), complex only
    const double* coef;     // device {alpha, beta, shift} or nullptr (then w/center/alpha/beta)
    double wbase[3][kMaxHalf];  // (-1/2) c_p / h_a^2 (alpha = 1)
};
int launch_stencil(hub_t h, const StencilArgs& a);
int stencil_variants(hub_t h);

// projectors.cu
int build_tables(hub_t h, int natoms, const double* pos, const int* kb_nchan, const int* kb_l,
                 const double* kb_rs, const double* kb_gamma, const double* kb_rc,
                 const int* hub_l, const double* hub_rs, const double* hub_rc,
                 const double* hub_U);
void free_table(Table& t);
// C[P x ncol] (double, x2 complex) = dV * <proj_p|x_n>; with want_W also W = transform(C)
// in the working type (gamma .* C for KB rows, M_spin C for Hubbard rows).
int launch_gather(hub_t h, const void* X, int ncol, int ld, int spin, bool want_W);
// Y[g, n] += alpha * sum_e vals_e . W[rows_e, n]   (W from the last launch_gather); with
// alpha_dev != nullptr alpha is read on the device
int launch_scatter(hub_t h, void* Y, int ncol, int ld, double alpha, const double* alpha_dev = nullptr);
// D per Hubbard atom (double, [nhub*50] re/im pairs) and E_U into d_scal[0] from the C of
// the last launch_gather; f_dev [ncol] double.
int launch_occupation(hub_t h, int ncol, const double* f_dev, double kweight, double* D_dev);
// F_dev[hsite*3 + axis] = -2 kweight Re sum_n f_n sum_m' conj(G_m'n) (M_spin C)_m'n per
// Hubbard atom, from C0 (the C of a gather of X, copied aside) and the C of the last
// launch_gather (a gather of d_axis X)
int launch_hub_force(hub_t h, int spin, int ncol, const double* f_dev, double kweight,
                     const void* C0, int axis, double* F_dev);

// projectors_tc.cu: tensor-core tables of the brick gather, and the gather itself (the
// partial rows of d_part, as the SIMT brick gather writes them)
int build_tc_tables(hub_t h, Table& t);
int launch_gather_tc(hub_t h, const void* X, int ncol, int ld);
// Y += alpha Phi W (W of the last launch_gather) in the tensor-core brick form
int launch_scatter_tc(hub_t h, void* Y, int ncol, int ld, double alpha, const double* alpha_dev);

// Moment integrals of the stress: Gm_b = dV <(x - R_image)_b phi_m | G> for the Hubbard rows
// (layout of d_C: [nproj x ncol] doubles, x2 complex; other rows untouched), b = x, y, z
int launch_moment_gather(hub_t h, const void* G, int ld, int ncol, double* Gm0, double* Gm1, double* Gm2);

// stencil.cu: G = d_axis X by the FD gradient of Sec. II.B (weights w[p-1] include 1/h),
// Bloch factor exp(i k_a L_a) per wrap (complex only); X, G share ld
int launch_fd_gradient(hub_t h, const void* X, int ld, int ncol, int axis, const double* w,
                       void* G);

// gemm.cu
// G[m x n] = alpha * A^H B, A: [K x m] (lda), B: [K x n] (ldb); K = Nd. Out double, row-major
// G[i*n + j].  sym: only blocks i <= j are computed and mirrored.
int launch_gram(hub_t h, const void* A, int lda, const void* B, int ldb, int m, int n,
                double alpha, bool sym, double* G);
// Y[K x n] = X[K x k] Q[k x n]; Q double column-major [k x n] (ldq = k)
int launch_rotate(hub_t h, const void* X, int ldx, const double* Q, int k, int n, void* Y,
                  int ldy);
// mixed-precision variants (tcgen05 path; 16-bit operand type from h->prec)
// true when the Rayleigh-Ritz block products of this handle run on the tensor cores: a mixed
// handle (BF16 or FP16 operands), real blocks, and a product form with 1 or 3 terms
inline bool tensor_mixed(const hub_ctx* h) {
    return (h->prec == HUB_MIXED_BF16 || h->prec == HUB_MIXED_F16) && h->bf16_terms > 0 && !h->cplx;
}
int launch_gram_bf16(hub_t h, const void* A, int lda, const void* B, int ldb, int m, int n,
                     double alpha, bool sym, double* G);
int launch_rotate_bf16(hub_t h, const void* X, int ldx, const double* Q, int k, int n,
                       void* Y, int ldy);

// dense.cu (double, n x n, row-major)
int dense_cholesky(hub_t h, double* A, int n);                 // lower L in place
int dense_tri_inverse(hub_t h, const double* L, double* Linv, int n);
// C = alpha op(A) op(B) + beta C ; row-major n x n style small matrices
int dense_gemm(hub_t h, bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
               int lda, const double* B, int ldb, double beta, double* C, int ldc);
int dense_jacobi_eigh(hub_t h, double* A, double* V, double* eig, int n);  // ascending
// one or two independent n x n problems in one cooperative launch (half the SMs each)
int dense_jacobi_eigh_multi(hub_t h, int nmat, double* const* A, double* const* V, double* const* eig, int n);
int dense_symmetrize(hub_t h, double* A, int n);

// api.cu: centred second-derivative weights of order 2 n0 (c0 and c_1..c_n0)
void fd_laplacian_weights(int n0, double* c0, double* c);
// api.cu: Fermi-Dirac entropy -sum f ln f + (1 - f) ln(1 - f) of occupations f; Pulay / DIIS
// coefficients from the k x k Gram matrix of the residuals (false: bordered system singular)
double fd_entropy(const std::vector<double>& f);
bool pulay_solve(const std::vector<double>& G, int k, std::vector<double>& coef);

// density.cu: reductions and vector algebra of the density SCF on [Nd] double vectors
int density_sum(hub_t h, const double* x, double* out_host);
int density_dot(hub_t h, const double* x, const double* y, int absdiff, double* out_host);
// y = sum_i c_i v_i + beta z (z may be nullptr); k <= 8; y may alias a v_i
int density_lincomb(hub_t h, double* y, int k, const double* const* v, const double* c,
                    const double* z, double beta);
int density_add3(hub_t h, double* y, const double* a, const double* b, const double* c);
int density_fill(hub_t h, double* y, double value);

// misc.cu
int launch_copy_convert_veff(hub_t h, const double* src, void* dst);
int launch_axpby_vec(hub_t h, int op, void* w, const void* v, const void* vprev, int step);
int launch_lanczos(hub_t h, int spin, int steps, const void* v0, double* lo, double* up);
int launch_copy_block(hub_t h, const void* src, int lds, void* dst, int ldd, int ncol);

// api: Rayleigh-Ritz of both spin channels of one handle (blocks X[0], X[1] of the same
// shape), the two subspace eigenproblems in one cooperative launch, half the SMs each
int rr_two_spins(hub_t h, void* const* X, int n, int ld, double* const* eig_host);

// api: apply_H with explicit buffers (used by filter / RR / Lanczos)
// Y = alpha (H X - shift X) + beta Yprev  (Yprev may alias Y; X, Y, Yprev share ld)
int apply_H_internal(hub_t h, int spin, const void* X, int ld, void* Y, int ncol, double alpha,
                     double shift, const void* Yprev, double beta, const double* coef_dev = nullptr);

}  // namespace hub
