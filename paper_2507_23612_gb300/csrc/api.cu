// C ABI of the hub library (declared in include/hub.h): handle lifecycle, H application,
// Chebyshev filter, Rayleigh-Ritz, occupation matrices, Lanczos bounds and the SCF driver.
// Host code here only orchestrates: every step on grid-sized data runs in this library's
// kernels.  The SCF driver's scalar work (Fermi level bisection over the eigenvalues, Pulay
// mixing of the 25-entry D matrices) runs on the host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "hub_internal.cuh"

namespace hub {

int fail(hub_t h, int code, const std::string& msg) {
    if (h) h->last_error = msg;
    return code;
}

int ensure(hub_t h, void** p, size_t* have, size_t need) {
    if (*have >= need && *p) return HUB_OK;
    h->mem_gen++;
    if (*p) {
        cudaStreamSynchronize(h->stream);
        cudaFree(*p);
        *p = nullptr;
        *have = 0;
    }
    if (need == 0) return HUB_OK;
    cudaError_t e = cudaMalloc(p, need);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(h, HUB_ENOMEM, std::string("cudaMalloc of workspace failed: ") + cudaGetErrorString(e));
    }
    *have = need;
    return HUB_OK;
}

int check_flags(hub_t h) {
    int f[8];
    HUB_CUDA_TRY(h, cudaMemcpyAsync(f, h->d_flags, sizeof(f), cudaMemcpyDeviceToHost, h->stream));
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->last_sweeps = std::max(f[6], f[7]);
    bool any = false;
    for (int i = 0; i < 6; ++i) any |= f[i] != 0;
    if (!any) return HUB_OK;
    HUB_CUDA_TRY(h, cudaMemsetAsync(h->d_flags, 0, 6 * sizeof(int), h->stream));
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (f[FLAG_TIMEOUT]) return fail(h, HUB_ETIMEOUT, "a bounded device wait ran out");
    if (f[FLAG_NOTSPD]) return fail(h, HUB_ENOTSPD, "Gram matrix is not positive definite");
    if (f[FLAG_NONFINITE]) return fail(h, HUB_ENONFINITE, "non-finite value");
    if (f[FLAG_NOCONV]) return fail(h, HUB_ENOCONV, "Jacobi eigensolver hit its sweep limit");
    return HUB_OK;
}

void fd_laplacian_weights(int n0, double* c0, double* c) {
    // centred second-derivative weights of order 2 n0:
    // c_p = 2 (-1)^{p+1} (n0!)^2 / (p^2 (n0-p)! (n0+p)!),  c_0 = -2 sum 1/p^2
    auto fact = [](int k) { double r = 1.0; for (int i = 2; i <= k; ++i) r *= i; return r; };
    double s = 0.0;
    for (int p = 1; p <= n0; ++p) {
        c[p - 1] = 2.0 * ((p % 2) ? 1.0 : -1.0) * fact(n0) * fact(n0) / ((double)p * p * fact(n0 - p) * fact(n0 + p));
        s += 1.0 / ((double)p * p);
    }
    *c0 = -2.0 * s;
}

// first-derivative weights of Sec. II.B per axis, 1/h_a included:
// w_p = (-1)^{p+1} (n0!)^2 / (h_a p (n0-p)! (n0+p)!)
static void fd_gradient_weights(hub_t h, double w[3][kMaxHalf]) {
    auto fact = [](int k) { double r = 1.0; for (int i = 2; i <= k; ++i) r *= i; return r; };
    for (int ax = 0; ax < 3; ++ax)
        for (int p = 1; p <= h->n0; ++p)
            w[ax][p - 1] = ((p % 2) ? 1.0 : -1.0) * fact(h->n0) * fact(h->n0) /
                           (h->h[ax] * p * fact(h->n0 - p) * fact(h->n0 + p));
}

int apply_H_internal(hub_t h, int spin, const void* X, int ld, void* Y, int ncol, double alpha,
                     double shift, const void* Yprev, double beta, const double* coef_dev) {
    int rc;
    if (h->proj.nsites > 0)
        if ((rc = launch_gather(h, X, ncol, ld, spin, true))) return rc;
    StencilArgs a{};
    a.Y = X;
    a.Yprev = Yprev;
    a.Yout = Y;
    a.V = (h->veff_per_spin && h->d_veff_spin[spin]) ? h->d_veff_spin[spin] : h->d_veff;
    a.n1 = h->n1; a.n2 = h->n2; a.n3 = h->n3; a.ld = ld; a.ncol = ncol;
    a.n0 = h->n0;
    double c0, c[kMaxHalf];
    fd_laplacian_weights(h->n0, &c0, c);
    double inv2 = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        const double ih2 = 1.0 / (h->h[ax] * h->h[ax]);
        inv2 += ih2;
        for (int p = 0; p < h->n0; ++p) {
            a.w[ax][p] = alpha * (-0.5) * c[p] * ih2;
            a.wbase[ax][p] = (-0.5) * c[p] * ih2;
        }
        a.phase[ax][0] = std::cos(h->kpt[ax] * h->L[ax]);
        a.phase[ax][1] = std::sin(h->kpt[ax] * h->L[ax]);
    }
    a.center = alpha * (-0.5 * c0 * inv2 - shift);
    a.alpha = alpha;
    a.beta = beta;
    a.coef = coef_dev;
    if ((rc = launch_stencil(h, a))) return rc;
    if (h->proj.nsites > 0)
        if ((rc = launch_scatter(h, Y, ncol, ld, alpha, coef_dev))) return rc;
    return HUB_OK;
}

static size_t elem_bytes(hub_t h) { return (size_t)h->esize * (h->cplx ? 2 : 1); }

static int check_block(hub_t h, int spin, const void* X, int ncol, int ld) {
    if (!h) return HUB_EINVAL;
    if (spin < 0 || spin > 1) return fail(h, HUB_EINVAL, "spin must be 0 or 1");
    if (ncol < 0) return fail(h, HUB_EINVAL, "ncol must be >= 0");
    if (ncol > 0 && !X) return fail(h, HUB_EINVAL, "NULL block");
    if ((long)ld < h->Nd) return fail(h, HUB_EINVAL, "ld must be >= n1*n2*n3");
    if (!h->veff_set) return fail(h, HUB_EINVAL, "hub_set_veff has not been called");
    if (!h->atoms_set) return fail(h, HUB_EINVAL, "hub_set_atoms_projectors has not been called");
    return HUB_OK;
}

// ---------------------------------------------------------------------------- SCF state
struct ScfState {
    hub_scf_params p{};
    std::vector<void*> X;
    std::vector<const void*> v0;
    std::vector<double> D_in, D_out, eig, occ;
    std::vector<std::vector<double>> hx, hr;   // Pulay history of inputs and residuals
    double bounds[2][3] = {{0, 0, 0}, {0, 0, 0}};
    bool have_bounds[2] = {false, false};
    int iter = 0;
    int small = 0;
    bool laddered = false;            // switched to the hi/lo split
    bool have_prev = false;
    double E_prev = 0.0;
    hub_scf_result last{};
    // self-consistent density: device vectors [Nd] inside hub_ctx::d_rho_ws
    bool density = false;
    double *vh = nullptr, *vh_out = nullptr, *tmp = nullptr, *rbar = nullptr, *z = nullptr;
    double *vx[2] = {nullptr, nullptr}, *vx_out[2] = {nullptr, nullptr};
    double *rho_in[2] = {nullptr, nullptr}, *rho_out[2] = {nullptr, nullptr};
    std::vector<double*> hist_x, hist_r;   // per history slot: nspin vectors each
    std::vector<int> slots;               // history slot of each entry of hx / hr
};

}  // namespace hub

using namespace hub;

extern "C" {

int hub_version(char* buf, int len) {
    const char* s = "hub 0.2 (sm_103a; real-space DFT+U CheFSI, forces, stress, density SCF)";
    if (!buf || len <= 0) return HUB_EINVAL;
    std::strncpy(buf, s, (size_t)len - 1);
    buf[len - 1] = 0;
    return HUB_OK;
}

int hub_create_grid(hub_t* out, int n1, int n2, int n3, double L1, double L2, double L3,
                    int fd_half_order, int ncomplex, const double* kpt, int prec, void* cuda_stream) {
    if (!out) return HUB_EINVAL;
    *out = nullptr;
    if (n1 < 1 || n2 < 1 || n3 < 1 || !(L1 > 0) || !(L2 > 0) || !(L3 > 0)) return HUB_EINVAL;
    if (fd_half_order < 1 || fd_half_order > 6) return HUB_EINVAL;
    if (prec < HUB_F64 || prec > HUB_MIXED_F16) return HUB_EINVAL;
    if ((long)n1 * n2 * n3 > 2000000000L) return HUB_EINVAL;
    hub_t h = new (std::nothrow) hub_ctx();
    if (!h) return HUB_ENOMEM;
    h->n1 = n1; h->n2 = n2; h->n3 = n3;
    h->Nd = (int64_t)n1 * n2 * n3;
    h->L[0] = L1; h->L[1] = L2; h->L[2] = L3;
    h->h[0] = L1 / n1; h->h[1] = L2 / n2; h->h[2] = L3 / n3;
    h->dV = h->h[0] * h->h[1] * h->h[2];
    h->n0 = fd_half_order;
    h->cplx = ncomplex ? 1 : 0;
    if (kpt && h->cplx) { h->kpt[0] = kpt[0]; h->kpt[1] = kpt[1]; h->kpt[2] = kpt[2]; }
    h->prec = prec;
    h->esize = prec == HUB_F64 ? 8 : 4;
    h->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_flags, 8 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_bar, 4 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_scal, 4096 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_tcmax, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_veff, (size_t)h->Nd * h->esize);
    if (e == cudaSuccess) e = cudaMemset(h->d_flags, 0, 8 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_scal, 0, 4096 * sizeof(double));
    if (e != cudaSuccess) {
        hub_destroy(h);
        return e == cudaErrorMemoryAllocation ? HUB_ENOMEM : HUB_ECUDA;
    }
    *out = h;
    return HUB_OK;
}

int hub_destroy(hub_t h) {
    if (!h) return HUB_OK;
    cudaStreamSynchronize(h->stream);
    for (auto& e : h->prof) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    free_table(h->proj);
    void* ptrs[] = {h->d_veff, h->d_work, h->d_work2, h->d_part, h->d_C, h->d_W, h->d_small,
                    h->d_gpart, h->d_bf16, h->d_aux, h->d_flags, h->d_bar, h->d_scal, h->d_tcmax, h->d_dens,
                    h->d_veff_spin[0], h->d_veff_spin[1], h->d_rho_ws, h->d_vloc};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete h->scf;
    delete h;
    return HUB_OK;
}

const char* hub_last_error(hub_t h) {
    if (!h) return "NULL handle";
    return h->last_error.c_str();
}

int hub_set_veff(hub_t h, const double* veff_dev) {
    if (!h) return HUB_EINVAL;
    if (!veff_dev) return fail(h, HUB_EINVAL, "NULL potential");
    int rc = launch_copy_convert_veff(h, veff_dev, h->d_veff);
    if (rc) return rc;
    // the double copy is the local potential of a self-consistent density SCF
    if ((rc = ensure(h, (void**)&h->d_vloc, &h->vloc_bytes, (size_t)h->Nd * sizeof(double)))) return rc;
    HUB_CUDA_TRY(h, cudaMemcpyAsync(h->d_vloc, veff_dev, (size_t)h->Nd * sizeof(double),
                                    cudaMemcpyDeviceToDevice, h->stream));
    h->veff_per_spin = 0;
    h->veff_set = true;
    return HUB_OK;
}

int hub_set_atoms_projectors(hub_t h, int natoms, const double* pos, const int* kb_nchan,
                             const int* kb_l, const double* kb_rs, const double* kb_gamma,
                             const double* kb_rc, const int* hub_l, const double* hub_rs,
                             const double* hub_rc, const double* hub_U) {
    if (!h) return HUB_EINVAL;
    if (natoms < 0) return fail(h, HUB_EINVAL, "natoms < 0");
    if (natoms > 0 && (!pos || !kb_nchan || !kb_rc || !hub_l || !hub_rs || !hub_rc || !hub_U))
        return fail(h, HUB_EINVAL, "NULL per-atom array");
    int nch = 0;
    for (int a = 0; a < natoms; ++a) nch += kb_nchan[a];
    if (nch > 0 && (!kb_l || !kb_rs || !kb_gamma)) return fail(h, HUB_EINVAL, "NULL KB channel array");
    int rc = build_tables(h, natoms, pos, kb_nchan, kb_l, kb_rs, kb_gamma, kb_rc, hub_l, hub_rs,
                          hub_rc, hub_U);
    if (rc) return rc;
    h->atoms_set = true;
    h->D_set[0] = h->D_set[1] = false;
    // real float blocks: the tensor-core brick gather and scatter when their tables exist (the
    // fastest form measured on the rutile workload; hub_autotune and hub_set_tuning can
    // change it)
    h->gather_dense = h->proj.tc ? 3 : 0;
    return HUB_OK;
}

int hub_num_hubbard_atoms(hub_t h, int* nhub) {
    if (!h || !nhub) return HUB_EINVAL;
    *nhub = h->proj.nhub;
    return HUB_OK;
}

int hub_set_occupation_matrix(hub_t h, int spin, const double* D_re, const double* D_im) {
    if (!h) return HUB_EINVAL;
    if (spin < 0 || spin > 1) return fail(h, HUB_EINVAL, "spin must be 0 or 1");
    if (!h->atoms_set) return fail(h, HUB_EINVAL, "hub_set_atoms_projectors has not been called");
    const int nh = h->proj.nhub;
    if (nh == 0) return HUB_OK;
    if (!D_re) return fail(h, HUB_EINVAL, "NULL D");
    const int cw = h->cplx ? 2 : 1;
    std::vector<double>& M = h->proj.h_M[spin];
    M.assign((size_t)nh * 25 * cw, 0.0);
    for (int i = 0; i < nh; ++i) {
        const double U = h->proj.h_U[i];
        for (int p = 0; p < 5; ++p)
            for (int m = 0; m < 5; ++m) {
                // M_pm = (U/2)(delta_pm - 2 D_pm); the transform applies W_p = sum_m M_pm C_m
                const size_t q = (size_t)i * 25 + p * 5 + m;
                M[q * cw] = 0.5 * U * ((p == m ? 1.0 : 0.0) - 2.0 * D_re[q]);
                if (cw == 2) M[q * cw + 1] = 0.5 * U * (-2.0 * (D_im ? D_im[q] : 0.0));
            }
    }
    HUB_CUDA_TRY(h, cudaMemcpyAsync(h->proj.d_M[spin], M.data(), M.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, h->stream));
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->D_set[spin] = true;
    return HUB_OK;
}

int hub_set_bf16_terms(hub_t h, int terms) {
    if (!h) return HUB_EINVAL;
    if (terms != 0 && terms != 1 && terms != 3) return fail(h, HUB_EINVAL, "terms must be 0, 1 or 3");
    h->bf16_terms = terms;
    return HUB_OK;
}

int hub_apply_H(hub_t h, int spin, const void* X, void* Y, int ncol, int ld) {
    hub::NvtxRange nvtx_("hub_apply_H");
    int rc = check_block(h, spin, X, ncol, ld);
    if (rc) return rc;
    if (ncol > 0 && !Y) return fail(h, HUB_EINVAL, "NULL output");
    if (ncol == 0) return HUB_OK;
    return apply_H_internal(h, spin, X, ld, Y, ncol, 1.0, 0.0, nullptr, 0.0);
}

int hub_chefsi_filter(hub_t h, int spin, void* X, int ncol, int ld, int degree, double a, double b,
                      double a_low, void* work) {
    hub::NvtxRange nvtx_("hub_chefsi_filter");
    int rc = check_block(h, spin, X, ncol, ld);
    if (rc) return rc;
    if (degree < 1) return fail(h, HUB_EINVAL, "degree must be >= 1");
    if (!(a_low < a && a < b)) return fail(h, HUB_EINVAL, "filter bounds need a_low < a < b");
    if (ncol == 0) return HUB_OK;
    void* B1 = work;
    if (!B1) {
        if ((rc = ensure(h, &h->d_work, &h->work_bytes, (size_t)ld * ncol * elem_bytes(h)))) return rc;
        B1 = h->d_work;
    }
    const double e = 0.5 * (b - a), c = 0.5 * (b + a);
    double sigma = e / (a_low - c);
    const double tau = 2.0 / sigma;
    if ((rc = apply_H_internal(h, spin, X, ld, B1, ncol, sigma / e, c, nullptr, 0.0))) return rc;
    void* cur = B1;
    void* prev = X;
    for (int i = 2; i <= degree; ++i) {
        const double sn = 1.0 / (tau - sigma);
        if ((rc = apply_H_internal(h, spin, cur, ld, prev, ncol, 2.0 * sn / e, c, prev, -sigma * sn))) return rc;
        std::swap(cur, prev);
        sigma = sn;
    }
    if (cur != X)
        if ((rc = launch_copy_block(h, cur, ld, X, ld, ncol))) return rc;
    return HUB_OK;
}

namespace hub {
// Rayleigh-Ritz in two halves around the subspace eigensolve, so that the SCF can solve the
// two spin channels' eigenproblems in one launch.  ws: 6 n x n matrices + n doubles (S, Hs,
// Linv, T, Vs, Q, eig; each matrix n^2 doubles, or n^2 double2 on a complex handle); HX: a
// block like X.  Complex (Bloch) blocks: S = dV X^H X = L L^H, Hs = dV X^H HX, H^ = L^-1 Hs
// L^-H (Hermitian), H^ = V diag(eig) V^H, X <- X L^-H V.
static size_t rr_mat(hub_t h, int n) { return (size_t)n * n * (h->cplx ? 2 : 1); }
static size_t rr_ws_doubles(hub_t h, int n) { return 6 * rr_mat(h, n) + n; }

static int rr_prepare(hub_t h, int spin, void* X, int n, int ld, void* HX, double* ws) {
    const size_t nn = rr_mat(h, n);
    double* S = ws;
    double* Hs = S + nn;
    double* Linv = Hs + nn;
    double* T = Linv + nn;
    int rc;
    if ((rc = apply_H_internal(h, spin, X, ld, HX, n, 1.0, 0.0, nullptr, 0.0))) return rc;
    const bool tensor = tensor_mixed(h);
    if (tensor) {
        // the Gram matrix feeds the Cholesky factor: always the hi/lo split (about 16
        // significand bits)
        const int terms = h->bf16_terms;
        h->bf16_terms = 3;
        rc = launch_gram_bf16(h, X, ld, X, ld, n, n, h->dV, true, S);
        h->bf16_terms = terms;
        if (rc) return rc;
        if ((rc = launch_gram_bf16(h, X, ld, HX, ld, n, n, h->dV, true, Hs))) return rc;
    } else {
        if ((rc = launch_gram(h, X, ld, X, ld, n, n, h->dV, true, S))) return rc;
        if ((rc = launch_gram(h, X, ld, HX, ld, n, n, h->dV, true, Hs))) return rc;
    }
    if ((rc = dense_cholesky(h, S, n))) return rc;
    if ((rc = check_flags(h))) return rc;
    if ((rc = dense_tri_inverse(h, S, Linv, n))) return rc;
    if ((rc = dense_gemm(h, false, false, n, n, n, 1.0, Linv, n, Hs, n, 0.0, T, n))) return rc;
    if ((rc = dense_gemm(h, false, true, n, n, n, 1.0, T, n, Linv, n, 0.0, Hs, n))) return rc;
    return dense_symmetrize(h, Hs, n);
}

static int rr_finish(hub_t h, void* X, int n, int ld, void* HX, double* ws, double* eig_host) {
    const size_t nn = rr_mat(h, n);
    double* Linv = ws + 2 * nn;
    double* Vs = ws + 4 * nn;
    double* Q = ws + 5 * nn;
    double* eig = ws + 6 * nn;
    int rc;
    if ((rc = dense_gemm(h, true, false, n, n, n, 1.0, Linv, n, Vs, n, 0.0, Q, n))) return rc;
    if (tensor_mixed(h)) {
        if ((rc = launch_rotate_bf16(h, X, ld, Q, n, n, HX, ld))) return rc;
    } else {
        if ((rc = launch_rotate(h, X, ld, Q, n, n, HX, ld))) return rc;
    }
    if ((rc = launch_copy_block(h, HX, ld, X, ld, n))) return rc;
    HUB_CUDA_TRY(h, cudaMemcpyAsync(eig_host, eig, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if ((rc = check_flags(h))) return rc;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(eig_host[i])) return fail(h, HUB_ENONFINITE, "non-finite Ritz value");
    return HUB_OK;
}

// Rayleigh-Ritz of both spin channels (blocks X[0], X[1] of the same shape): the two
// subspace eigenproblems are solved in one cooperative launch, half the SMs each.
extern "C++" int rr_two_spins(hub_t h, void* const* X, int n, int ld, double* const* eig_host) {
    const size_t nn = rr_mat(h, n), wsz = rr_ws_doubles(h, n);
    const size_t blk = (size_t)ld * n * elem_bytes(h);
    int rc;
    if ((rc = ensure(h, &h->d_work, &h->work_bytes, std::max(2 * blk, h->work_bytes)))) return rc;
    if ((rc = ensure(h, &h->d_small, &h->small_bytes, std::max(2 * wsz * sizeof(double), h->small_bytes))))
        return rc;
    void* HX[2] = {h->d_work, (char*)h->d_work + blk};
    double* ws[2] = {(double*)h->d_small, (double*)h->d_small + wsz};
    for (int s = 0; s < 2; ++s)
        if ((rc = rr_prepare(h, s, X[s], n, ld, HX[s], ws[s]))) return rc;
    double* Hs[2] = {ws[0] + nn, ws[1] + nn};
    double* Vs[2] = {ws[0] + 4 * nn, ws[1] + 4 * nn};
    double* eig[2] = {ws[0] + 6 * nn, ws[1] + 6 * nn};
    if ((rc = dense_jacobi_eigh_multi(h, 2, Hs, Vs, eig, n))) return rc;
    for (int s = 0; s < 2; ++s)
        if ((rc = rr_finish(h, X[s], n, ld, HX[s], ws[s], eig_host[s]))) return rc;
    return HUB_OK;
}
}  // namespace hub

int hub_rayleigh_ritz(hub_t h, int spin, void* X, int ncol, int ld, double* eig_host, void* work) {
    hub::NvtxRange nvtx_("hub_rayleigh_ritz");
    int rc = check_block(h, spin, X, ncol, ld);
    if (rc) return rc;
    if (ncol > 0 && !eig_host) return fail(h, HUB_EINVAL, "NULL eigenvalue output");
    if (ncol == 0) return HUB_OK;
    const int n = ncol;
    void* HX = work;
    if (!HX) {
        if ((rc = ensure(h, &h->d_work, &h->work_bytes, (size_t)ld * ncol * elem_bytes(h)))) return rc;
        HX = h->d_work;
    }
    const size_t nn = rr_mat(h, n);
    if ((rc = ensure(h, &h->d_small, &h->small_bytes, rr_ws_doubles(h, n) * sizeof(double)))) return rc;
    double* ws = (double*)h->d_small;
    if ((rc = rr_prepare(h, spin, X, n, ld, HX, ws))) return rc;
    if ((rc = dense_jacobi_eigh(h, ws + nn, ws + 4 * nn, ws + 6 * nn, n))) return rc;
    return rr_finish(h, X, n, ld, HX, ws, eig_host);
}

int hub_gram(hub_t h, const void* A, int ncol_a, const void* B, int ncol_b, int ld, double alpha,
             double* G_dev) {
    if (!h) return HUB_EINVAL;
    if (ncol_a < 0 || ncol_b < 0) return fail(h, HUB_EINVAL, "negative column count");
    if ((long)ld < h->Nd) return fail(h, HUB_EINVAL, "ld must be >= n1*n2*n3");
    if (ncol_a == 0 || ncol_b == 0) return HUB_OK;
    if (!A || !B || !G_dev) return fail(h, HUB_EINVAL, "NULL pointer");
    const bool sym = (A == B) && (ncol_a == ncol_b);
    if (tensor_mixed(h))
        return launch_gram_bf16(h, A, ld, B, ld, ncol_a, ncol_b, alpha, sym, G_dev);
    return launch_gram(h, A, ld, B, ld, ncol_a, ncol_b, alpha, sym, G_dev);
}

int hub_occupation(hub_t h, int spin, const void* X, int ncol, int ld, const double* f_host,
                   double kweight, double* D_re_out, double* D_im_out, double* EU_out) {
    hub::NvtxRange nvtx_("hub_occupation");
    int rc = check_block(h, spin, X, ncol, ld);
    if (rc) return rc;
    const int nh = h->proj.nhub;
    if (nh > 0 && !D_re_out) return fail(h, HUB_EINVAL, "NULL D output");
    if (ncol > 0 && !f_host) return fail(h, HUB_EINVAL, "NULL occupations");
    if (nh == 0 || ncol == 0) {
        if (D_re_out) std::fill(D_re_out, D_re_out + (size_t)nh * 25, 0.0);
        if (D_im_out) std::fill(D_im_out, D_im_out + (size_t)nh * 25, 0.0);
        if (EU_out) *EU_out = 0.0;
        return HUB_OK;
    }
    if ((rc = launch_gather(h, X, ncol, ld, spin, false))) return rc;
    const size_t need = (size_t)ncol * sizeof(double) + (size_t)nh * 50 * sizeof(double);
    if ((rc = ensure(h, &h->d_aux, &h->aux_bytes, std::max(need, h->aux_bytes)))) return rc;
    double* f_dev = (double*)h->d_aux;
    double* D_dev = f_dev + ncol;
    HUB_CUDA_TRY(h, cudaMemcpyAsync(f_dev, f_host, ncol * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if ((rc = launch_occupation(h, ncol, f_dev, kweight, D_dev))) return rc;
    std::vector<double> D((size_t)nh * 50);
    double eu = 0.0;
    HUB_CUDA_TRY(h, cudaMemcpyAsync(D.data(), D_dev, D.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HUB_CUDA_TRY(h, cudaMemcpyAsync(&eu, h->d_scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if ((rc = check_flags(h))) return rc;
    for (size_t q = 0; q < (size_t)nh * 25; ++q) {
        D_re_out[q] = D[2 * q];
        if (D_im_out) D_im_out[q] = D[2 * q + 1];
    }
    if (EU_out) *EU_out = eu;
    return HUB_OK;
}

int hub_num_projectors(hub_t h, int* nproj) {
    if (!h || !nproj) return HUB_EINVAL;
    *nproj = h->proj.nproj;
    return HUB_OK;
}

static int check_tables(hub_t h, const void* X, int ncol, int ld) {
    if (!h) return HUB_EINVAL;
    if (ncol < 0) return fail(h, HUB_EINVAL, "ncol must be >= 0");
    if (ncol > 0 && !X) return fail(h, HUB_EINVAL, "NULL block");
    if ((long)ld < h->Nd) return fail(h, HUB_EINVAL, "ld must be >= n1*n2*n3");
    if (!h->atoms_set) return fail(h, HUB_EINVAL, "hub_set_atoms_projectors has not been called");
    return HUB_OK;
}

int hub_project(hub_t h, const void* X, int ncol, int ld, double* C_host) {
    int rc = check_tables(h, X, ncol, ld);
    if (rc) return rc;
    const int cw = h->cplx ? 2 : 1;
    const size_t n = (size_t)h->proj.nproj * ncol * cw;
    if (n == 0) return HUB_OK;
    if (!C_host) return fail(h, HUB_EINVAL, "NULL output");
    if ((rc = launch_gather(h, X, ncol, ld, 0, false))) return rc;
    HUB_CUDA_TRY(h, cudaMemcpyAsync(C_host, h->d_C, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return check_flags(h);
}

int hub_expand(hub_t h, const double* W_host, int ncol, void* Y, int ld, double alpha) {
    int rc = check_tables(h, Y, ncol, ld);
    if (rc) return rc;
    const int cw = h->cplx ? 2 : 1;
    const size_t n = (size_t)h->proj.nproj * ncol * cw;
    if (n == 0) return HUB_OK;
    if (!W_host) return fail(h, HUB_EINVAL, "NULL coefficients");
    if ((rc = ensure(h, &h->d_W, &h->W_bytes, std::max(n * h->esize, h->W_bytes)))) return rc;
    if (h->esize == 8) {
        HUB_CUDA_TRY(h, cudaMemcpyAsync(h->d_W, W_host, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    } else {
        std::vector<float> wf(W_host, W_host + n);
        HUB_CUDA_TRY(h, cudaMemcpyAsync(h->d_W, wf.data(), n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));     // wf goes out of scope
    }
    return launch_scatter(h, Y, ncol, ld, alpha);
}

int hub_hubbard_forces(hub_t h, int spin, const void* X, int ncol, int ld, const double* f_host,
                       double kweight, double* F_host, void* work) {
    hub::NvtxRange nvtx_("hub_hubbard_forces");
    int rc = check_block(h, spin, X, ncol, ld);
    if (rc) return rc;
    if (!F_host) return fail(h, HUB_EINVAL, "NULL force output");
    if (ncol > 0 && !f_host) return fail(h, HUB_EINVAL, "NULL occupations");
    const Table& t = h->proj;
    std::fill(F_host, F_host + (size_t)t.natoms * 3, 0.0);
    if (t.nhub == 0 || ncol == 0) return HUB_OK;
    double w[3][kMaxHalf];
    fd_gradient_weights(h, w);
    void* G = work;
    if (!G) {
        if ((rc = ensure(h, &h->d_work, &h->work_bytes, (size_t)ld * ncol * elem_bytes(h)))) return rc;
        G = h->d_work;
    }
    // C of X set aside, then one gather of each gradient component
    if ((rc = launch_gather(h, X, ncol, ld, spin, false))) return rc;
    const int cw = h->cplx ? 2 : 1;
    const size_t nC = (size_t)t.nproj * ncol * cw;
    const size_t need = (nC + ncol + (size_t)t.nhub * 3) * sizeof(double);
    if ((rc = ensure(h, &h->d_aux, &h->aux_bytes, std::max(need, h->aux_bytes)))) return rc;
    double* C0 = (double*)h->d_aux;
    double* f_dev = C0 + nC;
    double* F_dev = f_dev + ncol;
    HUB_CUDA_TRY(h, cudaMemcpyAsync(C0, h->d_C, nC * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    HUB_CUDA_TRY(h, cudaMemcpyAsync(f_dev, f_host, ncol * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    for (int ax = 0; ax < 3; ++ax) {
        if ((rc = launch_fd_gradient(h, X, ld, ncol, ax, w[ax], G))) return rc;
        if ((rc = launch_gather(h, G, ncol, ld, spin, false))) return rc;
        if ((rc = launch_hub_force(h, spin, ncol, f_dev, kweight, C0, ax, F_dev))) return rc;
    }
    std::vector<double> F((size_t)t.nhub * 3);
    HUB_CUDA_TRY(h, cudaMemcpyAsync(F.data(), F_dev, F.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if ((rc = check_flags(h))) return rc;
    for (int i = 0; i < t.nhub; ++i)
        for (int ax = 0; ax < 3; ++ax) F_host[(size_t)t.h_hub_atom[i] * 3 + ax] = F[(size_t)i * 3 + ax];
    return HUB_OK;
}

int hub_hubbard_stress(hub_t h, int spin, const void* X, int ncol, int ld, const double* f_host,
                       double kweight, double* sigma_host, void* work) {
    hub::NvtxRange nvtx_("hub_hubbard_stress");
    int rc = check_block(h, spin, X, ncol, ld);
    if (rc) return rc;
    if (!sigma_host) return fail(h, HUB_EINVAL, "NULL stress output");
    if (ncol > 0 && !f_host) return fail(h, HUB_EINVAL, "NULL occupations");
    std::fill(sigma_host, sigma_host + 9, 0.0);
    const Table& t = h->proj;
    if (t.nhub == 0 || ncol == 0) return HUB_OK;
    double w[3][kMaxHalf];
    fd_gradient_weights(h, w);
    void* G = work;
    if (!G) {
        if ((rc = ensure(h, &h->d_work, &h->work_bytes, (size_t)ld * ncol * elem_bytes(h)))) return rc;
        G = h->d_work;
    }
    // C = <phi|x> stays in d_C for the whole call (the moment gathers write their own rows)
    if ((rc = launch_gather(h, X, ncol, ld, spin, false))) return rc;
    const int cw = h->cplx ? 2 : 1;
    const size_t nC = (size_t)t.nproj * ncol * cw;
    const size_t need = (ncol + (size_t)t.nhub * 50 + 3 * nC + 9 * (size_t)t.nhub) * sizeof(double);
    if ((rc = ensure(h, &h->d_aux, &h->aux_bytes, std::max(need, h->aux_bytes)))) return rc;
    double* f_dev = (double*)h->d_aux;
    double* Dblk = f_dev + ncol;
    double* Gm = Dblk + (size_t)t.nhub * 50;
    double* out = Gm + 3 * nC;                       // [a][hsite * 3 + b]
    HUB_CUDA_TRY(h, cudaMemsetAsync(Gm, 0, 3 * nC * sizeof(double), h->stream));
    HUB_CUDA_TRY(h, cudaMemcpyAsync(f_dev, f_host, ncol * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if ((rc = launch_occupation(h, ncol, f_dev, kweight, Dblk))) return rc;
    for (int a = 0; a < 3; ++a) {
        if ((rc = launch_fd_gradient(h, X, ld, ncol, a, w[a], G))) return rc;
        if ((rc = launch_moment_gather(h, G, ld, ncol, Gm, Gm + nC, Gm + 2 * nC))) return rc;
        for (int b = 0; b < 3; ++b)
            if ((rc = launch_hub_force(h, spin, ncol, f_dev, kweight, Gm + b * nC, b,
                                       out + (size_t)a * t.nhub * 3))) return rc;
    }
    std::vector<double> o((size_t)9 * t.nhub), D((size_t)t.nhub * 50);
    HUB_CUDA_TRY(h, cudaMemcpyAsync(o.data(), out, o.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HUB_CUDA_TRY(h, cudaMemcpyAsync(D.data(), Dblk, D.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if ((rc = check_flags(h))) return rc;
    const std::vector<double>& M = t.h_M[spin];
    const double omega = h->dV * (double)h->Nd;
    for (int J = 0; J < t.nhub; ++J) {
        // sum_mm' M_m'm Dblk_mm' (real part); M row m', column m
        double tr = 0.0;
        if (!M.empty())
            for (int m = 0; m < 5; ++m)
                for (int mp = 0; mp < 5; ++mp) {
                    const size_t qm = (size_t)J * 25 + mp * 5 + m, qd = (size_t)J * 25 + m * 5 + mp;
                    tr += M[qm * cw] * D[2 * qd] - (cw == 2 ? M[qm * cw + 1] * D[2 * qd + 1] : 0.0);
                }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                sigma_host[a * 3 + b] += ((a == b ? -tr : 0.0) + o[(size_t)a * t.nhub * 3 + J * 3 + b]) / omega;
    }
    return HUB_OK;
}

int hub_projector_stats(hub_t h, long long* function_points, long long* site_points) {
    if (!h) return HUB_EINVAL;
    if (function_points) *function_points = h->proj.nvals;
    if (site_points) *site_points = h->proj.npts;
    return HUB_OK;
}

int hub_lanczos_bound(hub_t h, int spin, int steps, const void* v0, double* lo_out, double* up_out) {
    int rc = check_block(h, spin, v0, 1, (int)h->Nd);
    if (rc) return rc;
    if (steps < 1 || steps > 64) return fail(h, HUB_EINVAL, "1 <= steps <= 64");
    if (!lo_out || !up_out) return fail(h, HUB_EINVAL, "NULL output");
    if ((rc = launch_lanczos(h, spin, steps, v0, lo_out, up_out))) return rc;
    return check_flags(h);
}

// ---------------------------------------------------------------------------- SCF driver

static void fermi_dirac(const std::vector<double>& e, double kT, double nel, double deg,
                        std::vector<double>& f, double& mu) {
    const size_t n = e.size();
    f.assign(n, 0.0);
    if (kT <= 0.0) {
        std::vector<size_t> ord(n);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return e[a] < e[b]; });
        const long nfill = std::lround(nel / deg);
        for (long i = 0; i < nfill && i < (long)n; ++i) f[ord[i]] = 1.0;
        mu = nfill > 0 ? e[ord[std::min<long>(nfill, n) - 1]] : e[ord[0]];
        return;
    }
    auto count = [&](double m) {
        double s = 0.0;
        for (size_t i = 0; i < n; ++i) s += deg * 0.5 * (1.0 - std::tanh((e[i] - m) / (2.0 * kT)));
        return s;
    };
    double lo = *std::min_element(e.begin(), e.end()) - 50 * kT;
    double hi = *std::max_element(e.begin(), e.end()) + 50 * kT;
    for (int it = 0; it < 200; ++it) {
        const double m = 0.5 * (lo + hi);
        if (count(m) < nel) lo = m; else hi = m;
        if (hi - lo < 1e-15) break;
    }
    mu = 0.5 * (lo + hi);
    for (size_t i = 0; i < n; ++i) f[i] = 0.5 * (1.0 - std::tanh((e[i] - mu) / (2.0 * kT)));
}

}  // extern "C"

namespace hub {
double fd_entropy(const std::vector<double>& f) {
    double s = 0.0;
    for (double x : f) {
        const double a = std::min(std::max(x, 1e-300), 1.0 - 1e-16);
        const double b = std::max(1.0 - a, 1e-300);
        s -= a * std::log(a) + b * std::log(b);
    }
    return s;
}

// Pulay / DIIS coefficients: minimise |sum c_i r_i| subject to sum c_i = 1, from the k x k
// Gram matrix A (row-major) of the residuals.  false when the bordered system is singular.
bool pulay_solve(const std::vector<double>& G, int k, std::vector<double>& coef) {
    coef.assign(k, 0.0);
    if (k < 2) return false;
    const int m = k + 1;
    std::vector<double> A((size_t)m * m, 0.0), b(m, 0.0);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) A[(size_t)i * m + j] = G[(size_t)i * k + j];
    for (int i = 0; i < k; ++i) { A[(size_t)i * m + k] = 1.0; A[(size_t)k * m + i] = 1.0; }
    b[k] = 1.0;
    // Gaussian elimination with partial pivoting
    double scale = 0.0;
    for (double v : A) scale = std::max(scale, std::fabs(v));
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r2 = c + 1; r2 < m; ++r2)
            if (std::fabs(A[(size_t)r2 * m + c]) > std::fabs(A[(size_t)piv * m + c])) piv = r2;
        if (std::fabs(A[(size_t)piv * m + c]) <= 1e-14 * scale) return false;
        if (piv != c) {
            for (int q = 0; q < m; ++q) std::swap(A[(size_t)c * m + q], A[(size_t)piv * m + q]);
            std::swap(b[c], b[piv]);
        }
        for (int r2 = c + 1; r2 < m; ++r2) {
            const double fct = A[(size_t)r2 * m + c] / A[(size_t)c * m + c];
            for (int q = c; q < m; ++q) A[(size_t)r2 * m + q] -= fct * A[(size_t)c * m + q];
            b[r2] -= fct * b[c];
        }
    }
    std::vector<double> x(m);
    for (int c = m - 1; c >= 0; --c) {
        double sm = b[c];
        for (int q = c + 1; q < m; ++q) sm -= A[(size_t)c * m + q] * x[q];
        x[c] = sm / A[(size_t)c * m + c];
    }
    for (int i = 0; i < k; ++i) coef[i] = x[i];
    return true;
}

}  // namespace hub

extern "C" {

// pushes (xin, xout - xin) into the D history (at most pulay_history entries)
static void pulay_push(ScfState& st, const std::vector<double>& xin, const std::vector<double>& xout) {
    const size_t n = xin.size();
    std::vector<double> r(n);
    for (size_t i = 0; i < n; ++i) r[i] = xout[i] - xin[i];
    st.hx.push_back(xin);
    st.hr.push_back(r);
    const int hist = std::max(1, st.p.pulay_history);
    while ((int)st.hx.size() > hist) { st.hx.erase(st.hx.begin()); st.hr.erase(st.hr.begin()); }
}

// Gram matrix of the stored D residuals
static std::vector<double> pulay_gram_D(const ScfState& st) {
    const int k = (int)st.hr.size();
    std::vector<double> G((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double sm = 0.0;
            for (size_t q = 0; q < st.hr[i].size(); ++q) sm += st.hr[i][q] * st.hr[j][q];
            G[(size_t)i * k + j] = sm;
        }
    return G;
}

// Pulay / DIIS on D alone: x = sum c_i (x_i + beta r_i); linear mixing while the history is
// one entry long or its system is singular
static std::vector<double> pulay_mix(ScfState& st, const std::vector<double>& xin,
                                     const std::vector<double>& xout) {
    pulay_push(st, xin, xout);
    const int k = (int)st.hr.size();
    const double beta = st.p.pulay_beta;
    const size_t n = xin.size();
    std::vector<double> out(n), coef;
    if (!pulay_solve(pulay_gram_D(st), k, coef)) {
        const std::vector<double>& r = st.hr.back();
        for (size_t q = 0; q < n; ++q) out[q] = xin[q] + beta * r[q];
        return out;
    }
    for (size_t q = 0; q < n; ++q) {
        double xs = 0.0, rs = 0.0;
        for (int i = 0; i < k; ++i) { xs += coef[i] * st.hx[i][q]; rs += coef[i] * st.hr[i][q]; }
        out[q] = xs + beta * rs;
    }
    return out;
}

// ---------------------------------------------------------------------------- density SCF
constexpr int kCgMaxIter = 20000;
static double dens_kappa(const hub_scf_params& p) { return p.kerker_kappa > 0 ? p.kerker_kappa : 0.5; }
static double dens_tol_rho(const hub_scf_params& p) { return p.tol_rho > 0 ? p.tol_rho : 1e-4; }
static double dens_cg_tol(const hub_scf_params& p) { return p.cg_tol > 0 ? p.cg_tol : 1e-10; }

// device vectors of the density model: V_H, V_H of rho_out, scratch, Pulay combination,
// preconditioned residual, v_x of rho_in and of rho_out, rho_in, rho_out, and the Pulay
// history of densities and residuals; per-spin V_eff in the working type
static int density_setup(hub_t h, ScfState& st) {
    const int ns = st.p.nspin;
    const int H = std::max(1, st.p.pulay_history);
    const size_t Nd = (size_t)h->Nd;
    const size_t nvec = 5 + 4 * (size_t)ns + 2 * (size_t)H * ns;
    int rc;
    if ((rc = ensure(h, (void**)&h->d_rho_ws, &h->rho_ws_bytes, nvec * Nd * sizeof(double)))) return rc;
    HUB_CUDA_TRY(h, cudaMemsetAsync(h->d_rho_ws, 0, nvec * Nd * sizeof(double), h->stream));
    double* v = h->d_rho_ws;
    auto take = [&]() { double* q = v; v += Nd; return q; };
    st.vh = take(); st.vh_out = take(); st.tmp = take(); st.rbar = take(); st.z = take();
    for (int s = 0; s < ns; ++s) { st.vx[s] = take(); st.vx_out[s] = take(); st.rho_in[s] = take(); st.rho_out[s] = take(); }
    st.hist_x.assign(H, nullptr);
    st.hist_r.assign(H, nullptr);
    for (int i = 0; i < H; ++i) {
        st.hist_x[i] = v; v += ns * Nd;
        st.hist_r[i] = v; v += ns * Nd;
    }
    for (int s = 0; s < ns; ++s)
        if (!h->d_veff_spin[s])
            HUB_CUDA_TRY(h, cudaMalloc(&h->d_veff_spin[s], Nd * h->esize));
    const double vol = h->dV * (double)h->Nd;
    for (int s = 0; s < ns; ++s)
        if ((rc = density_fill(h, st.rho_in[s], st.p.n_elec / ns / vol))) return rc;
    st.density = true;
    return HUB_OK;
}

// total density of the channels into st.tmp (or the one channel itself)
static int density_total(hub_t h, ScfState& st, double* const* rho, const double** out) {
    if (st.p.nspin == 1) { *out = rho[0]; return HUB_OK; }
    const double* v[2] = {rho[0], rho[1]};
    const double c[2] = {1.0, 1.0};
    *out = st.tmp;
    return density_lincomb(h, st.tmp, 2, v, c, nullptr, 0.0);
}

// V_eff^s = V_loc + V_H[rho_in] + v_x^s[rho_in] for every channel; fresh upper bounds
static int density_potentials(hub_t h, ScfState& st, int* cg_iters) {
    const hub_scf_params& p = st.p;
    const int ns = p.nspin;
    int rc, it = 0;
    const double* rho_tot;
    if ((rc = density_total(h, st, st.rho_in, &rho_tot))) return rc;
    if ((rc = hub_hartree(h, rho_tot, st.vh, dens_cg_tol(p), kCgMaxIter, &it, nullptr))) return rc;
    *cg_iters += it;
    if ((rc = hub_lda_exchange(h, ns, st.rho_in[0], ns == 2 ? st.rho_in[1] : nullptr, st.vx[0],
                               ns == 2 ? st.vx[1] : nullptr, nullptr))) return rc;
    for (int s = 0; s < ns; ++s) {
        if ((rc = density_add3(h, st.tmp, h->d_vloc, st.vh, st.vx[s]))) return rc;
        if ((rc = launch_copy_convert_veff(h, st.tmp, h->d_veff_spin[s]))) return rc;
    }
    h->veff_per_spin = 1;
    for (int s = 0; s < ns; ++s) {
        double lo, up;
        if ((rc = hub_lanczos_bound(h, s, p.lanczos_steps, st.v0[s], &lo, &up))) return rc;
        if (!st.have_bounds[s]) {
            st.bounds[s][0] = lo;
            st.bounds[s][1] = lo + 0.1 * (up - lo);
            st.have_bounds[s] = true;
        }
        st.bounds[s][2] = up;
    }
    return HUB_OK;
}

// rho_out of the iteration and the density terms of the energy
static int density_terms(hub_t h, ScfState& st, double deg, double* e_dc_hx, double* e_h, double* e_x,
                         double* drho, int* cg_iters) {
    const hub_scf_params& p = st.p;
    const int ns = p.nspin;
    int rc;
    *e_dc_hx = 0.0;
    *drho = 0.0;
    for (int s = 0; s < ns; ++s) {
        HUB_CUDA_TRY(h, cudaMemsetAsync(st.rho_out[s], 0, (size_t)h->Nd * sizeof(double), h->stream));
        if ((rc = hub_density(h, st.X[s], p.ncol, p.ld, st.occ.data() + (size_t)s * p.ncol, deg,
                              st.rho_out[s]))) return rc;
        double a = 0.0, b = 0.0, d = 0.0;
        if ((rc = density_dot(h, st.rho_out[s], st.vh, 0, &a))) return rc;
        if ((rc = density_dot(h, st.rho_out[s], st.vx[s], 0, &b))) return rc;
        if ((rc = density_dot(h, st.rho_out[s], st.rho_in[s], 1, &d))) return rc;
        *e_dc_hx += h->dV * (a + b);
        *drho += h->dV * d;
    }
    *drho /= std::max(p.n_elec, 1e-300);
    const double* rho_tot;
    if ((rc = density_total(h, st, st.rho_out, &rho_tot))) return rc;
    HUB_CUDA_TRY(h, cudaMemcpyAsync(st.vh_out, st.vh, (size_t)h->Nd * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    int it = 0;
    if ((rc = hub_hartree(h, rho_tot, st.vh_out, dens_cg_tol(p), kCgMaxIter, &it, e_h))) return rc;
    *cg_iters += it;
    return hub_lda_exchange(h, ns, st.rho_out[0], ns == 2 ? st.rho_out[1] : nullptr, st.vx_out[0],
                            ns == 2 ? st.vx_out[1] : nullptr, e_x);
}

// Pulay on [rho, D] with one set of coefficients; the density block of the combined
// residual goes through the Kerker preconditioner
static int density_mix(hub_t h, ScfState& st, int* cg_iters) {
    const hub_scf_params& p = st.p;
    const int ns = p.nspin;
    const int H = std::max(1, p.pulay_history);
    const size_t Nd = (size_t)h->Nd;
    int rc;
    int slot;
    if ((int)st.slots.size() < H) slot = (int)st.slots.size();
    else { slot = st.slots.front(); st.slots.erase(st.slots.begin()); }
    pulay_push(st, st.D_in, st.D_out);
    st.slots.push_back(slot);
    for (int s = 0; s < ns; ++s) {
        HUB_CUDA_TRY(h, cudaMemcpyAsync(st.hist_x[slot] + s * Nd, st.rho_in[s], Nd * sizeof(double),
                                        cudaMemcpyDeviceToDevice, h->stream));
        const double* v[2] = {st.rho_out[s], st.rho_in[s]};
        const double c[2] = {1.0, -1.0};
        if ((rc = density_lincomb(h, st.hist_r[slot] + s * Nd, 2, v, c, nullptr, 0.0))) return rc;
    }
    const int k = (int)st.slots.size();
    std::vector<double> G = pulay_gram_D(st);
    for (int i = 0; i < k; ++i)
        for (int j = i; j < k; ++j) {
            double d = 0.0;
            for (int s = 0; s < ns; ++s) {
                double ds = 0.0;
                if ((rc = density_dot(h, st.hist_r[st.slots[i]] + s * Nd, st.hist_r[st.slots[j]] + s * Nd, 0, &ds))) return rc;
                d += ds;
            }
            G[(size_t)i * k + j] += d;
            if (j != i) G[(size_t)j * k + i] += d;
        }
    std::vector<double> coef;
    if (!pulay_solve(G, k, coef)) { coef.assign(k, 0.0); coef[k - 1] = 1.0; }   // linear mixing
    const double beta = p.pulay_beta;
    for (int s = 0; s < ns; ++s) {
        const double* vr[8];
        const double* vx[8];
        for (int i = 0; i < k; ++i) {
            vr[i] = st.hist_r[st.slots[i]] + s * Nd;
            vx[i] = st.hist_x[st.slots[i]] + s * Nd;
        }
        if ((rc = density_lincomb(h, st.rbar, k, vr, coef.data(), nullptr, 0.0))) return rc;
        int it = 0;
        if ((rc = hub_kerker(h, st.rbar, st.z, dens_kappa(p), dens_cg_tol(p), kCgMaxIter, &it))) return rc;
        *cg_iters += it;
        if ((rc = density_lincomb(h, st.rho_in[s], k, vx, coef.data(), st.z, beta))) return rc;
    }
    const size_t n = st.D_in.size();
    std::vector<double> out(n);
    for (size_t q = 0; q < n; ++q) {
        double xs = 0.0, rs = 0.0;
        for (int i = 0; i < k; ++i) { xs += coef[i] * st.hx[i][q]; rs += coef[i] * st.hr[i][q]; }
        out[q] = xs + beta * rs;
    }
    st.D_in = out;
    return HUB_OK;
}

int hub_scf_begin(hub_t h, const hub_scf_params* p, void* const* X, const void* const* v0,
                  const double* D0) {
    if (!h || !p || !X || !v0) return HUB_EINVAL;
    if (p->nspin < 1 || p->nspin > 2) return fail(h, HUB_EINVAL, "nspin must be 1 or 2");
    if (p->ncol < 1 || p->degree < 1 || p->max_iter < 1 || p->lanczos_steps < 1 || p->lanczos_steps > 64)
        return fail(h, HUB_EINVAL, "bad SCF parameters");
    if (h->cplx) return fail(h, HUB_EINVAL, "the SCF driver runs real (Gamma-point) orbitals");
    for (int s = 0; s < p->nspin; ++s) {
        int rc = check_block(h, s, X[s], p->ncol, p->ld);
        if (rc) return rc;
        if (!v0[s]) return fail(h, HUB_EINVAL, "NULL Lanczos start vector");
    }
    const int nh = h->proj.nhub;
    if (nh > 0 && !D0) return fail(h, HUB_EINVAL, "NULL starting D");
    delete h->scf;
    h->scf = new ScfState();
    ScfState& st = *h->scf;
    st.p = *p;
    st.X.assign(X, X + p->nspin);
    st.v0.assign(v0, v0 + p->nspin);
    st.D_in.assign(D0 ? D0 : nullptr, D0 ? D0 + (size_t)p->nspin * nh * 25 : nullptr);
    st.D_in.resize((size_t)p->nspin * nh * 25, 0.0);
    st.D_out.assign(st.D_in.size(), 0.0);
    st.eig.assign((size_t)p->nspin * p->ncol, 0.0);
    st.occ.assign(st.eig.size(), 0.0);
    h->veff_per_spin = 0;
    if (p->density) {
        if (p->pulay_history > 8) return fail(h, HUB_EINVAL, "density SCF: pulay_history <= 8");
        if (!(p->n_elec > 0)) return fail(h, HUB_EINVAL, "density SCF: n_elec must be > 0");
        if (!h->d_vloc) return fail(h, HUB_EINVAL, "density SCF: no local potential");
        int rc = density_setup(h, st);
        if (rc) return rc;
    }
    return HUB_OK;
}

int hub_scf_forces(hub_t h, double* F_host, double* sigma_host) {
    if (!h || !h->scf) return fail(h, HUB_EINVAL, "hub_scf_begin has not been called");
    if (!F_host) return fail(h, HUB_EINVAL, "NULL force output");
    ScfState& st = *h->scf;
    if (st.iter == 0) return fail(h, HUB_EINVAL, "no SCF iteration has run");
    const hub_scf_params& p = st.p;
    const int nh = h->proj.nhub, na = h->proj.natoms;
    const double deg = p.nspin == 1 ? 2.0 : 1.0;
    std::fill(F_host, F_host + (size_t)na * 3, 0.0);
    if (sigma_host) std::fill(sigma_host, sigma_host + 9, 0.0);
    std::vector<double> F((size_t)std::max(na, 1) * 3), sig(9);
    int rc;
    for (int s = 0; s < p.nspin; ++s) {
        if ((rc = hub_set_occupation_matrix(h, s, st.D_out.data() + (size_t)s * nh * 25, nullptr))) return rc;
        const double* f = st.occ.data() + (size_t)s * p.ncol;
        if ((rc = hub_hubbard_forces(h, s, st.X[s], p.ncol, p.ld, f, deg, F.data(), nullptr))) return rc;
        for (size_t q = 0; q < (size_t)na * 3; ++q) F_host[q] += F[q];
        if (sigma_host) {
            if ((rc = hub_hubbard_stress(h, s, st.X[s], p.ncol, p.ld, f, deg, sig.data(), nullptr))) return rc;
            for (int q = 0; q < 9; ++q) sigma_host[q] += sig[q];
        }
    }
    return HUB_OK;
}

int hub_scf_set_density(hub_t h, const double* rho_dev) {
    if (!h || !h->scf) return fail(h, HUB_EINVAL, "hub_scf_begin has not been called");
    ScfState& st = *h->scf;
    if (!st.density) return fail(h, HUB_EINVAL, "the SCF is not in density mode");
    if (st.iter != 0) return fail(h, HUB_EINVAL, "the starting density is set before the first iteration");
    if (!rho_dev) return fail(h, HUB_EINVAL, "NULL density");
    const double c = 1.0 / st.p.nspin;
    for (int s = 0; s < st.p.nspin; ++s) {
        const double* v[1] = {rho_dev};
        int rc = density_lincomb(h, st.rho_in[s], 1, v, &c, nullptr, 0.0);
        if (rc) return rc;
    }
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return HUB_OK;
}

int hub_scf_density(hub_t h, double* rho_dev) {
    if (!h || !h->scf) return fail(h, HUB_EINVAL, "hub_scf_begin has not been called");
    ScfState& st = *h->scf;
    if (!st.density) return fail(h, HUB_EINVAL, "the SCF is not in density mode");
    if (!rho_dev) return fail(h, HUB_EINVAL, "NULL density");
    const size_t bytes = (size_t)h->Nd * sizeof(double);
    if (st.p.nspin == 1) {
        HUB_CUDA_TRY(h, cudaMemcpyAsync(rho_dev, st.rho_out[0], bytes, cudaMemcpyDeviceToDevice, h->stream));
    } else {
        const double* v[2] = {st.rho_out[0], st.rho_out[1]};
        const double c[2] = {1.0, 1.0};
        int rc = density_lincomb(h, rho_dev, 2, v, c, nullptr, 0.0);
        if (rc) return rc;
    }
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return HUB_OK;
}

int hub_scf_iterate(hub_t h, hub_scf_result* res) {
    hub::NvtxRange nvtx_("hub_scf_iterate");
    if (!h || !h->scf) return fail(h, HUB_EINVAL, "hub_scf_begin has not been called");
    ScfState& st = *h->scf;
    const hub_scf_params& p = st.p;
    const int nh = h->proj.nhub;
    const int ns = p.nspin;
    const double deg = ns == 1 ? 2.0 : 1.0;
    int rc;
    if (p.ladder && (h->prec == HUB_MIXED_BF16 || h->prec == HUB_MIXED_F16)) h->bf16_terms = st.laddered ? 0 : 1;
    // per spin channel: filter + Rayleigh-Ritz passes; with two channels both are filtered
    // first and their Rayleigh-Ritz projections share one eigensolver launch
    const int passes = st.iter == 0 ? std::max(1, p.first_passes) : 1;
    for (int s = 0; s < ns; ++s)
        if ((rc = hub_set_occupation_matrix(h, s, st.D_in.data() + (size_t)s * nh * 25, nullptr))) return rc;
    int cg_iters = 0;
    if (st.density)
        if ((rc = density_potentials(h, st, &cg_iters))) return rc;
    for (int pass = 0; pass < passes; ++pass) {
        for (int s = 0; s < ns; ++s) {
            if (!st.have_bounds[s]) {
                double lo, up;
                if ((rc = hub_lanczos_bound(h, s, p.lanczos_steps, st.v0[s], &lo, &up))) return rc;
                st.bounds[s][0] = lo;
                st.bounds[s][1] = lo + 0.1 * (up - lo);
                st.bounds[s][2] = up;
                st.have_bounds[s] = true;
            }
            if ((rc = hub_chefsi_filter(h, s, st.X[s], p.ncol, p.ld, p.degree, st.bounds[s][1],
                                        st.bounds[s][2], st.bounds[s][0], nullptr))) return rc;
            if (ns == 1) {
                double* eg = st.eig.data();
                if ((rc = hub_rayleigh_ritz(h, s, st.X[s], p.ncol, p.ld, eg, nullptr))) return rc;
            }
        }
        if (ns == 2) {
            double* eg[2] = {st.eig.data(), st.eig.data() + p.ncol};
            if ((rc = rr_two_spins(h, st.X.data(), p.ncol, p.ld, eg))) return rc;
        }
        for (int s = 0; s < ns; ++s) {
            const double* eg = st.eig.data() + (size_t)s * p.ncol;
            st.bounds[s][0] = eg[0];
            st.bounds[s][1] = eg[p.ncol - 1];
        }
    }
    double mu = 0.0;
    fermi_dirac(st.eig, p.kT, p.n_elec, deg, st.occ, mu);
    double e_band = 0.0, e_dc = 0.0, e_u = 0.0, ent = 0.0;
    for (int s = 0; s < ns; ++s) {
        double eu_s = 0.0;
        const double* f = st.occ.data() + (size_t)s * p.ncol;
        if ((rc = hub_occupation(h, s, st.X[s], p.ncol, p.ld, f, 1.0,
                                 st.D_out.data() + (size_t)s * nh * 25, nullptr, &eu_s))) return rc;
        e_u += deg * eu_s;
        for (int n = 0; n < p.ncol; ++n) e_band += deg * f[n] * st.eig[(size_t)s * p.ncol + n];
        for (int i = 0; i < nh; ++i) {
            const double U = h->proj.h_U[i];
            for (int a = 0; a < 5; ++a)
                for (int b = 0; b < 5; ++b) {
                    const size_t q = ((size_t)s * nh + i) * 25 + a * 5 + b;
                    const double M = 0.5 * U * ((a == b ? 1.0 : 0.0) - 2.0 * st.D_in[q]);
                    e_dc += deg * M * st.D_out[q];
                }
        }
    }
    if (p.kT > 0) {
        for (int s = 0; s < ns; ++s) {
            std::vector<double> f(st.occ.begin() + (size_t)s * p.ncol, st.occ.begin() + (size_t)(s + 1) * p.ncol);
            ent += deg * fd_entropy(f);
        }
    }
    double e_dc_hx = 0.0, e_h = 0.0, e_x = 0.0, drho = 0.0;
    if (st.density)
        if ((rc = density_terms(h, st, deg, &e_dc_hx, &e_h, &e_x, &drho, &cg_iters))) return rc;
    const double E = e_band - e_dc + e_u - p.kT * ent - e_dc_hx + e_h + e_x;
    double dD = 0.0;
    for (size_t q = 0; q < st.D_in.size(); ++q) dD = std::max(dD, std::fabs(st.D_out[q] - st.D_in[q]));
    const double dE = st.have_prev ? E - st.E_prev : 0.0;
    if (st.have_prev && std::fabs(dE) / std::max(1, p.natoms) < p.tol_e_atom) st.small++;
    else st.small = 0;
    st.have_prev = true;
    st.E_prev = E;
    st.iter++;
    hub_scf_result r{};
    r.iter = st.iter;
    r.converged = (st.small >= 2 && dD < p.tol_D && (!st.density || drho < dens_tol_rho(p))) ? 1 : 0;
    r.E_H = e_h; r.E_x = e_x; r.drho = drho; r.cg_iters = cg_iters;
    r.E = E; r.E_band = e_band; r.E_U = e_u; r.dE = dE; r.dD = dD; r.mu = mu;
    r.bf16_terms = (h->prec == HUB_MIXED_BF16 || h->prec == HUB_MIXED_F16) ? h->bf16_terms : 0;
    r.jacobi_sweeps = h->last_sweeps;
    if (p.ladder && !st.laddered && st.iter > 1 && std::fabs(dE) / std::max(1, p.natoms) < p.ladder_tol) {
        st.laddered = true;
        st.small = 0;       // the converged-energy count restarts at the finer precision
        r.converged = 0;
    }
    if (!r.converged) {
        if (st.density) {
            if ((rc = density_mix(h, st, &r.cg_iters))) return rc;
        } else {
            st.D_in = pulay_mix(st, st.D_in, st.D_out);
        }
    }
    st.last = r;
    if (res) *res = r;
    return HUB_OK;
}

int hub_scf_run(hub_t h, hub_scf_result* res) {
    if (!h || !h->scf) return fail(h, HUB_EINVAL, "hub_scf_begin has not been called");
    hub_scf_result r{};
    while (h->scf->iter < h->scf->p.max_iter) {
        int rc = hub_scf_iterate(h, &r);
        if (rc) return rc;
        if (r.converged) break;
    }
    if (res) *res = r;
    return r.converged ? HUB_OK : fail(h, HUB_ENOCONV, "SCF reached max_iter");
}

int hub_profile(hub_t h, int enable) {
    if (!h) return HUB_EINVAL;
    if (enable < 0) {
        cudaStreamSynchronize(h->stream);
        for (auto& e : h->prof) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
        h->prof.clear();
        h->prof_on = 0;
        return HUB_OK;
    }
    h->prof_on = enable ? 1 : 0;
    return HUB_OK;
}

int hub_profile_read(hub_t h, int kind, double* total_ms, long long* launches) {
    if (!h || !total_ms || !launches) return HUB_EINVAL;
    if (kind < 0 || kind >= HUB_K_COUNT) return fail(h, HUB_EINVAL, "unknown kernel kind");
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    double t = 0.0;
    long long n = 0;
    for (auto& e : h->prof) {
        if (e.kind != kind) continue;
        float ms = 0.f;
        HUB_CUDA_TRY(h, cudaEventElapsedTime(&ms, e.a, e.b));
        t += ms;
        n++;
    }
    *total_ms = t;
    *launches = n;
    return HUB_OK;
}

int hub_launch_count(hub_t h, long long* launches) {
    if (!h || !launches) return HUB_EINVAL;
    *launches = h->launches;
    return HUB_OK;
}

int hub_scf_get(hub_t h, double* eig, double* occ, double* D_out) {
    if (!h || !h->scf) return fail(h, HUB_EINVAL, "hub_scf_begin has not been called");
    ScfState& st = *h->scf;
    if (eig) std::copy(st.eig.begin(), st.eig.end(), eig);
    if (occ) std::copy(st.occ.begin(), st.occ.end(), occ);
    if (D_out) std::copy(st.D_out.begin(), st.D_out.end(), D_out);
    return HUB_OK;
}

}  // extern "C"
