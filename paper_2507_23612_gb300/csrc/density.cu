// Grid-sized steps of the self-consistent density SCF: the electron density of a block of
// orbitals, the periodic FD Poisson problem of the Hartree potential, local-density
// exchange, the Kerker preconditioner, and the vector algebra of Pulay mixing on the
// density.  Sec. II.B (last paragraph) names CheFSI with real-space preconditioned Pulay
// mixing whose density coefficients also mix the occupation matrices; the functional
// pieces are readings (the paper does not print E_DFT):
//   rho(g)  = scale * sum_n f_n |x_n(g)|^2
//   V_H:    -Lap_h V_H = 4 pi (rho - mean rho), mean V_H = 0 (neutralising background)
//   v_x:    -(4/3) k rho^(1/3), E_x = -k dV sum rho^(4/3), k = (3/4)(3/pi)^(1/3) (x 2^(1/3)
//           per channel of a spin-polarized pair)
//   Kerker: z = (-Lap_h)(-Lap_h + kappa^2)^-1 r
// Both linear problems are solved by conjugate gradients on (-Lap_h + shift), FP64, with the
// same 2*n0-th order FD Laplacian as the kinetic term (periodic: the density and the
// potentials are cell-periodic).  CG scalars stay on the device; the host reads the residual
// every kCgCheck iterations.  Reductions are two-stage with a fixed order (deterministic).
#include <algorithm>
#include <cmath>
#include <vector>

#include "hub_internal.cuh"
#include "cplx.cuh"

namespace hub {

namespace {

constexpr int kThreads = 256;
constexpr int kCgCheck = 16;          // CG iterations between host residual checks
constexpr int kMaxLin = 8;            // vectors of one linear combination

__device__ __forceinline__ double abs2(double v) { return v * v; }
__device__ __forceinline__ double abs2(float v) { return (double)v * v; }
__device__ __forceinline__ double abs2(double2 v) { return v.x * v.x + v.y * v.y; }
__device__ __forceinline__ double abs2(float2 v) { return (double)v.x * v.x + (double)v.y * v.y; }

// block sum of one double per thread into part[blockIdx.x] (blockDim.x == kThreads)
__device__ __forceinline__ void block_partial(double v, double* part) {
    __shared__ double red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// out[slot] = scale * sum(part[0..n)); one CTA, fixed order.  With copy_from >= 0 also
// out[copy_to] = out[copy_from] first (the CG's rr <- rr_new hand-over).
__global__ void k_reduce(const double* __restrict__ part, int n, double scale, double* __restrict__ out,
                         int slot, int copy_from, int copy_to) {
    __shared__ double red[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (copy_from >= 0) out[copy_to] = out[copy_from];
        out[slot] = scale * red[0];
    }
}

// ---------------------------------------------------------------------------- density
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_density(const T* __restrict__ X, int ld, int ncol, long Nd, const double* __restrict__ f, double scale,
          double* __restrict__ rho) {
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    if (g >= Nd) return;
    double acc = 0.0;
    int n = 0;
    for (; n + 4 <= ncol; n += 4) {
        const T a = X[(long)n * ld + g], b = X[(long)(n + 1) * ld + g];
        const T c = X[(long)(n + 2) * ld + g], d = X[(long)(n + 3) * ld + g];
        acc += f[n] * abs2(a) + f[n + 1] * abs2(b) + f[n + 2] * abs2(c) + f[n + 3] * abs2(d);
    }
    for (; n < ncol; ++n) acc += f[n] * abs2(X[(long)n * ld + g]);
    rho[g] += scale * acc;
}

// ---------------------------------------------------------------------------- Laplacian
struct LapArgs {
    double w[3][kMaxHalf];   // c_p / h_a^2
    double center;           // c_0 sum_a h_a^-2
    int n0, n1, n2, n3;
};

// y = shift x - Lap_h x (periodic); with part != nullptr also block partials of x . y
__global__ void __launch_bounds__(kThreads)
k_neg_lap(const double* __restrict__ x, double* __restrict__ y, LapArgs a, double shift, double* __restrict__ part) {
    const long Nd = (long)a.n1 * a.n2 * a.n3;
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    double dot = 0.0;
    if (g < Nd) {
        const int i = (int)(g % a.n1);
        const long t = g / a.n1;
        const int j = (int)(t % a.n2);
        const int k = (int)(t / a.n2);
        const long sy = a.n1, sz = (long)a.n1 * a.n2;
        const double* row = x + (g - i);                      // (0, j, k)
        const double* col = x + (g - (long)j * sy);           // (i, 0, k)
        const double* pil = x + (g - (long)k * sz);           // (i, j, 0)
        const double x0 = x[g];
        double lap = a.center * x0;
        for (int p = 1; p <= a.n0; ++p) {
            int ip = i + p, im = i - p, jp = j + p, jm = j - p, kp = k + p, km = k - p;
            while (ip >= a.n1) ip -= a.n1;
            while (im < 0) im += a.n1;
            while (jp >= a.n2) jp -= a.n2;
            while (jm < 0) jm += a.n2;
            while (kp >= a.n3) kp -= a.n3;
            while (km < 0) km += a.n3;
            lap = fma(a.w[0][p - 1], row[ip] + row[im], lap);
            lap = fma(a.w[1][p - 1], col[(long)jp * sy] + col[(long)jm * sy], lap);
            lap = fma(a.w[2][p - 1], pil[(long)kp * sz] + pil[(long)km * sz], lap);
        }
        const double out = shift * x0 - lap;
        y[g] = out;
        dot = x0 * out;
    }
    if (part) block_partial(dot, part);
}

// ---------------------------------------------------------------------------- CG steps
// scalar slots: 0 rr, 1 pq, 2 rr_new, 3 bb, 4 scratch
enum { S_RR = 0, S_PQ = 1, S_RRN = 2, S_BB = 3, S_TMP = 4 };

// r = b - q, p = r; partials of r . r and of b . b (part, part + nblk)
__global__ void __launch_bounds__(kThreads)
k_cg_start(const double* __restrict__ b, const double* __restrict__ q, double* __restrict__ r, double* __restrict__ p,
           long n, double* __restrict__ part, int nblk) {
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    double rr = 0.0, bb = 0.0;
    if (g < n) {
        const double v = b[g] - q[g];
        r[g] = v;
        p[g] = v;
        rr = v * v;
        bb = b[g] * b[g];
    }
    block_partial(rr, part);
    __syncthreads();
    block_partial(bb, part + nblk);
}

// alpha = rr / pq; x += alpha p; r -= alpha q; partials of r . r
__global__ void __launch_bounds__(kThreads)
k_cg_update(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p, const double* __restrict__ q,
            long n, const double* __restrict__ s, double* __restrict__ part) {
    const double pq = s[S_PQ];
    const double alpha = pq > 0.0 ? s[S_RR] / pq : 0.0;
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    double rr = 0.0;
    if (g < n) {
        x[g] = fma(alpha, p[g], x[g]);
        const double v = fma(-alpha, q[g], r[g]);
        r[g] = v;
        rr = v * v;
    }
    block_partial(rr, part);
}

// beta = rr_new / rr; p = r + beta p
__global__ void __launch_bounds__(kThreads)
k_cg_direction(const double* __restrict__ r, double* __restrict__ p, long n, const double* __restrict__ s) {
    const double rr = s[S_RR];
    const double beta = rr > 0.0 ? s[S_RRN] / rr : 0.0;
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    if (g < n) p[g] = fma(beta, p[g], r[g]);
}

// y = c0 * (x - s[slot] / n) (c0 = 4 pi: the Poisson right-hand side; slot holds sum x)
// (x and y may be the same vector)
__global__ void k_center_scale(const double* x, double* y, long n, double c0, const double* __restrict__ s,
                               int slot) {
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    if (g < n) y[g] = c0 * (x[g] - s[slot] / (double)n);
}

__global__ void __launch_bounds__(kThreads)
k_partial_sum(const double* __restrict__ x, long n, double* __restrict__ part) {
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    block_partial(g < n ? x[g] : 0.0, part);
}

__global__ void __launch_bounds__(kThreads)
k_partial_dot(const double* __restrict__ x, const double* __restrict__ y, long n, double* __restrict__ part) {
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    block_partial(g < n ? x[g] * y[g] : 0.0, part);
}

__global__ void __launch_bounds__(kThreads)
k_partial_absdiff(const double* __restrict__ x, const double* __restrict__ y, long n, double* __restrict__ part) {
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    block_partial(g < n ? fabs(x[g] - y[g]) : 0.0, part);
}

// ---------------------------------------------------------------------------- exchange
__global__ void __launch_bounds__(kThreads)
k_lda_x(const double* __restrict__ rho, double* __restrict__ vx, long n, double k, double* __restrict__ part) {
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    double e = 0.0;
    if (g < n) {
        const double r = fmax(rho[g], 0.0);
        const double c = cbrt(r);
        vx[g] = -(4.0 / 3.0) * k * c;
        e = -k * r * c;                       // -k rho^(4/3)
    }
    block_partial(e, part);
}

// ---------------------------------------------------------------------------- linear algebra
struct LinArgs {
    const double* v[kMaxLin];
    double c[kMaxLin];
    int k;
};

// y = sum_i c_i v_i (+ beta * z when z != nullptr)
// (y may be one of the v_i)
__global__ void k_lincomb(double* y, long n, LinArgs a, const double* z, double beta) {
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    if (g >= n) return;
    double s = 0.0;
    for (int i = 0; i < a.k; ++i) s = fma(a.c[i], a.v[i][g], s);
    if (z) s = fma(beta, z[g], s);
    y[g] = s;
}

__global__ void k_add3(double* __restrict__ y, const double* __restrict__ a, const double* __restrict__ b,
                       const double* __restrict__ c, long n) {
    const long g = (long)blockIdx.x * kThreads + threadIdx.x;
    if (g < n) y[g] = a[g] + b[g] + c[g];
}

unsigned blocks_for(long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

// ---------------------------------------------------------------------------- host side
// workspace: [nblk*2 partials][8 scalars][r][p][q][b] doubles
static int dens_ws(hub_t h, double** part, double** s, double** r, double** p, double** q, double** b) {
    const long n = h->Nd;
    const long nblk = blocks_for(n);
    const size_t need = (size_t)(2 * nblk + 8 + 4 * n) * sizeof(double);
    int rc = ensure(h, &h->d_dens, &h->dens_bytes, need);
    if (rc) return rc;
    double* base = (double*)h->d_dens;
    *part = base;
    *s = base + 2 * nblk;
    *r = *s + 8;
    *p = *r + n;
    *q = *p + n;
    *b = *q + n;
    return HUB_OK;
}

static LapArgs lap_args(hub_t h) {
    LapArgs a{};
    double c0, c[kMaxHalf];
    fd_laplacian_weights(h->n0, &c0, c);
    double inv2 = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        const double ih2 = 1.0 / (h->h[ax] * h->h[ax]);
        inv2 += ih2;
        for (int p = 0; p < h->n0; ++p) a.w[ax][p] = c[p] * ih2;
    }
    a.center = c0 * inv2;
    a.n0 = h->n0;
    a.n1 = h->n1; a.n2 = h->n2; a.n3 = h->n3;
    return a;
}

// s[slot] = scale * sum of the partials of the last partial kernel
static int reduce_to(hub_t h, const double* part, int nblk, double scale, double* s, int slot,
                     int copy_from = -1, int copy_to = -1) {
    k_reduce<<<1, kThreads, 0, h->stream>>>(part, nblk, scale, s, slot, copy_from, copy_to);
    h->launches++;
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

// (-Lap_h + shift) x = b by CG from the x given; |r| <= tol |b| or max_iter iterations.
// b lives in the workspace slot `bw` (untouched).  Returns HUB_ENOCONV past max_iter.
static int cg_solve(hub_t h, double shift, const double* bw, double* x, double tol, int max_iter, int* iters) {
    double *part, *s, *r, *p, *q, *b;
    int rc = dens_ws(h, &part, &s, &r, &p, &q, &b);
    if (rc) return rc;
    const long n = h->Nd;
    const unsigned nb = blocks_for(n);
    const LapArgs la = lap_args(h);
    ProfScope ps(h, HUB_K_DENSITY);                    // counts the first launch
    k_neg_lap<<<nb, kThreads, 0, h->stream>>>(x, q, la, shift, nullptr);
    k_cg_start<<<nb, kThreads, 0, h->stream>>>(bw, q, r, p, n, part, (int)nb);
    h->launches += 1;
    HUB_CUDA_TRY(h, cudaGetLastError());
    if ((rc = reduce_to(h, part, nb, 1.0, s, S_RRN))) return rc;
    if ((rc = reduce_to(h, part + nb, nb, 1.0, s, S_BB))) return rc;
    double chk[4];
    HUB_CUDA_TRY(h, cudaMemcpyAsync(chk, s, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const double bb = chk[S_BB];
    int it = 0;
    if (bb == 0.0) {
        HUB_CUDA_TRY(h, cudaMemsetAsync(x, 0, n * sizeof(double), h->stream));
        if (iters) *iters = 0;
        return HUB_OK;
    }
    double rr = chk[S_RRN];
    while (rr > tol * tol * bb && it < max_iter) {
        const int chunk = std::min(kCgCheck, max_iter - it);
        for (int c = 0; c < chunk; ++c) {
            k_neg_lap<<<nb, kThreads, 0, h->stream>>>(p, q, la, shift, part);
            h->launches++;
            if ((rc = reduce_to(h, part, nb, 1.0, s, S_PQ, S_RRN, S_RR))) return rc;
            k_cg_update<<<nb, kThreads, 0, h->stream>>>(x, r, p, q, n, s, part);
            h->launches++;
            if ((rc = reduce_to(h, part, nb, 1.0, s, S_RRN))) return rc;
            k_cg_direction<<<nb, kThreads, 0, h->stream>>>(r, p, n, s);
            h->launches++;
        }
        HUB_CUDA_TRY(h, cudaGetLastError());
        it += chunk;
        HUB_CUDA_TRY(h, cudaMemcpyAsync(&rr, s + S_RRN, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        if (!std::isfinite(rr)) return fail(h, HUB_ENONFINITE, "non-finite CG residual");
    }
    if (iters) *iters = it;
    if (rr > tol * tol * bb) return fail(h, HUB_ENOCONV, "CG reached its iteration limit");
    return HUB_OK;
}

int density_sum(hub_t h, const double* x, double* out_host) {
    double *part, *s, *r, *p, *q, *b;
    int rc = dens_ws(h, &part, &s, &r, &p, &q, &b);
    if (rc) return rc;
    const unsigned nb = blocks_for(h->Nd);
    k_partial_sum<<<nb, kThreads, 0, h->stream>>>(x, h->Nd, part);
    h->launches++;
    HUB_CUDA_TRY(h, cudaGetLastError());
    if ((rc = reduce_to(h, part, nb, 1.0, s, S_TMP))) return rc;
    HUB_CUDA_TRY(h, cudaMemcpyAsync(out_host, s + S_TMP, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return HUB_OK;
}

int density_dot(hub_t h, const double* x, const double* y, int absdiff, double* out_host) {
    double *part, *s, *r, *p, *q, *b;
    int rc = dens_ws(h, &part, &s, &r, &p, &q, &b);
    if (rc) return rc;
    const unsigned nb = blocks_for(h->Nd);
    if (absdiff) k_partial_absdiff<<<nb, kThreads, 0, h->stream>>>(x, y, h->Nd, part);
    else k_partial_dot<<<nb, kThreads, 0, h->stream>>>(x, y, h->Nd, part);
    h->launches++;
    HUB_CUDA_TRY(h, cudaGetLastError());
    if ((rc = reduce_to(h, part, nb, 1.0, s, S_TMP))) return rc;
    HUB_CUDA_TRY(h, cudaMemcpyAsync(out_host, s + S_TMP, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return HUB_OK;
}

int density_lincomb(hub_t h, double* y, int k, const double* const* v, const double* c,
                    const double* z, double beta) {
    if (k < 0 || k > kMaxLin) return fail(h, HUB_EINVAL, "at most 8 vectors per combination");
    LinArgs a{};
    a.k = k;
    for (int i = 0; i < k; ++i) { a.v[i] = v[i]; a.c[i] = c[i]; }
    k_lincomb<<<blocks_for(h->Nd), kThreads, 0, h->stream>>>(y, h->Nd, a, z, beta);
    h->launches++;
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

__global__ void k_fill(double* __restrict__ y, long n, double v) {
    const long g = (long)blockIdx.x * 256 + threadIdx.x;
    if (g < n) y[g] = v;
}

int density_fill(hub_t h, double* y, double value) {
    k_fill<<<blocks_for(h->Nd), 256, 0, h->stream>>>(y, h->Nd, value);
    h->launches++;
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int density_add3(hub_t h, double* y, const double* a, const double* b, const double* c) {
    k_add3<<<blocks_for(h->Nd), kThreads, 0, h->stream>>>(y, a, b, c, h->Nd);
    h->launches++;
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

}  // namespace hub

using namespace hub;

extern "C" {

int hub_density(hub_t h, const void* X, int ncol, int ld, const double* f_host, double scale,
                double* rho_dev) {
    if (!h) return HUB_EINVAL;
    if (ncol < 0) return fail(h, HUB_EINVAL, "ncol must be >= 0");
    if ((long)ld < h->Nd) return fail(h, HUB_EINVAL, "ld must be >= n1*n2*n3");
    if (!rho_dev) return fail(h, HUB_EINVAL, "NULL density");
    if (ncol == 0) return HUB_OK;
    if (!X || !f_host) return fail(h, HUB_EINVAL, "NULL block or occupations");
    int rc;
    const size_t need = (size_t)ncol * sizeof(double);
    if ((rc = ensure(h, &h->d_aux, &h->aux_bytes, std::max(need, h->aux_bytes)))) return rc;
    double* f_dev = (double*)h->d_aux;
    HUB_CUDA_TRY(h, cudaMemcpyAsync(f_dev, f_host, need, cudaMemcpyHostToDevice, h->stream));
    const unsigned nb = blocks_for(h->Nd);
    ProfScope ps(h, HUB_K_DENSITY);
    if (h->esize == 8) {
        if (h->cplx) k_density<double2><<<nb, kThreads, 0, h->stream>>>((const double2*)X, ld, ncol, h->Nd, f_dev, scale, rho_dev);
        else k_density<double><<<nb, kThreads, 0, h->stream>>>((const double*)X, ld, ncol, h->Nd, f_dev, scale, rho_dev);
    } else {
        if (h->cplx) k_density<float2><<<nb, kThreads, 0, h->stream>>>((const float2*)X, ld, ncol, h->Nd, f_dev, scale, rho_dev);
        else k_density<float><<<nb, kThreads, 0, h->stream>>>((const float*)X, ld, ncol, h->Nd, f_dev, scale, rho_dev);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int hub_hartree(hub_t h, const double* rho_dev, double* V_dev, double tol, int max_iter,
                int* iters_out, double* EH_out) {
    hub::NvtxRange nvtx_("hub_hartree");
    if (!h) return HUB_EINVAL;
    if (!rho_dev || !V_dev) return fail(h, HUB_EINVAL, "NULL density or potential");
    if (!(tol > 0.0) || max_iter < 1) return fail(h, HUB_EINVAL, "tol must be > 0 and max_iter >= 1");
    double *part, *s, *r, *p, *q, *b;
    int rc = dens_ws(h, &part, &s, &r, &p, &q, &b);
    if (rc) return rc;
    const long n = h->Nd;
    const unsigned nb = blocks_for(n);
    {
        ProfScope ps(h, HUB_K_DENSITY);
        k_partial_sum<<<nb, kThreads, 0, h->stream>>>(rho_dev, n, part);
        HUB_CUDA_TRY(h, cudaGetLastError());
    }
    if ((rc = reduce_to(h, part, nb, 1.0, s, S_TMP))) return rc;
    k_center_scale<<<nb, kThreads, 0, h->stream>>>(rho_dev, b, n, 4.0 * M_PI, s, S_TMP);
    h->launches++;
    HUB_CUDA_TRY(h, cudaGetLastError());
    if ((rc = cg_solve(h, 0.0, b, V_dev, tol, max_iter, iters_out))) return rc;
    // remove the constant the singular operator leaves undetermined: V <- V - sum(V) / n
    k_partial_sum<<<nb, kThreads, 0, h->stream>>>(V_dev, n, part);
    h->launches++;
    HUB_CUDA_TRY(h, cudaGetLastError());
    if ((rc = reduce_to(h, part, nb, 1.0, s, S_TMP))) return rc;
    k_center_scale<<<nb, kThreads, 0, h->stream>>>(V_dev, V_dev, n, 1.0, s, S_TMP);
    h->launches++;
    HUB_CUDA_TRY(h, cudaGetLastError());
    if (EH_out) {
        double d = 0.0;
        if ((rc = density_dot(h, rho_dev, V_dev, 0, &d))) return rc;
        *EH_out = 0.5 * h->dV * d;
    }
    return HUB_OK;
}

int hub_lda_exchange(hub_t h, int nchan, const double* rho0, const double* rho1, double* vx0,
                     double* vx1, double* Ex_out) {
    if (!h) return HUB_EINVAL;
    if (nchan != 1 && nchan != 2) return fail(h, HUB_EINVAL, "one or two channels");
    if (!rho0 || !vx0 || (nchan == 2 && (!rho1 || !vx1))) return fail(h, HUB_EINVAL, "NULL density or potential");
    double *part, *s, *r, *p, *q, *b;
    int rc = dens_ws(h, &part, &s, &r, &p, &q, &b);
    if (rc) return rc;
    const long n = h->Nd;
    const unsigned nb = blocks_for(n);
    const double k = 0.75 * std::cbrt(3.0 / M_PI) * (nchan == 2 ? std::cbrt(2.0) : 1.0);
    double E = 0.0;
    for (int c = 0; c < nchan; ++c) {
        {
            ProfScope ps(h, HUB_K_DENSITY);
            k_lda_x<<<nb, kThreads, 0, h->stream>>>(c ? rho1 : rho0, c ? vx1 : vx0, n, k, part);
            HUB_CUDA_TRY(h, cudaGetLastError());
        }
        if ((rc = reduce_to(h, part, nb, h->dV, s, S_TMP))) return rc;
        double e = 0.0;
        HUB_CUDA_TRY(h, cudaMemcpyAsync(&e, s + S_TMP, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        E += e;
    }
    if (Ex_out) *Ex_out = E;
    return HUB_OK;
}

int hub_kerker(hub_t h, const double* r_dev, double* z_dev, double kappa, double tol, int max_iter,
               int* iters_out) {
    hub::NvtxRange nvtx_("hub_kerker");
    if (!h) return HUB_EINVAL;
    if (!r_dev || !z_dev) return fail(h, HUB_EINVAL, "NULL residual or output");
    if (!(kappa >= 0.0) || !(tol > 0.0) || max_iter < 1) return fail(h, HUB_EINVAL, "bad kappa, tol or max_iter");
    double *part, *s, *r, *p, *q, *b;
    int rc = dens_ws(h, &part, &s, &r, &p, &q, &b);
    if (rc) return rc;
    const unsigned nb = blocks_for(h->Nd);
    {
        ProfScope ps(h, HUB_K_DENSITY);
        k_neg_lap<<<nb, kThreads, 0, h->stream>>>(r_dev, b, lap_args(h), 0.0, nullptr);   // b = -Lap r
        HUB_CUDA_TRY(h, cudaGetLastError());
    }
    HUB_CUDA_TRY(h, cudaMemsetAsync(z_dev, 0, h->Nd * sizeof(double), h->stream));
    return cg_solve(h, kappa * kappa, b, z_dev, tol, max_iter, iters_out);
}

}  // extern "C"
