// Small device helpers: potential conversion, block copies, deterministic dot products and
// the Lanczos bound estimator used to place the Chebyshev filter interval (CheFSI, Sec. II.B).
#include <algorithm>
#include <vector>
#include <cmath>

#include "hub_internal.cuh"
#include "cplx.cuh"

namespace hub {

namespace {

template <typename R>
__global__ void k_convert(const double* __restrict__ src, R* __restrict__ dst, long n) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = (R)src[t];
}

template <typename T>
__global__ void k_copy_block(const T* __restrict__ src, int lds, T* __restrict__ dst, int ldd, long Nd) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < Nd) dst[(size_t)blockIdx.y * ldd + t] = src[(size_t)blockIdx.y * lds + t];
}

constexpr int RBLK = 512;     // blocks of the first reduction stage

// partial[b] = sum over a grid-stride slice of conj(x) y (double accumulation)
template <typename R, bool CPLX>
__global__ void k_dot_partial(const typename VT<R, CPLX>::T* __restrict__ x,
                              const typename VT<R, CPLX>::T* __restrict__ y, long n,
                              double* __restrict__ part) {
    double acc = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        if constexpr (CPLX) acc += (double)x[i].x * (double)y[i].x + (double)x[i].y * (double)y[i].y;
        else acc += (double)x[i] * (double)y[i];
    }
    __shared__ double s[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        part[blockIdx.x] = t;
    }
}

// out = sum(part[0..n)) [op]: 0 plain, 1 sqrt
__global__ void k_dot_final(const double* __restrict__ part, int n, double* out, int op) {
    __shared__ double s[RBLK];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = op == 1 ? sqrt(s[0]) : s[0];
}

// Lanczos vector updates with scalars read from device memory (no host round trip)
//   mode 0: v = x / scal[ia]
//   mode 1: w = w - scal[ia] * v - scal[ib] * vprev     (ib < 0: no vprev term)
template <typename R, bool CPLX>
__global__ void k_lanczos_axpy(int mode, typename VT<R, CPLX>::T* __restrict__ out,
                               const typename VT<R, CPLX>::T* __restrict__ v,
                               const typename VT<R, CPLX>::T* __restrict__ vprev, long n,
                               const double* __restrict__ scal, int ia, int ib) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (mode == 0) {
        const double inv = 1.0 / scal[ia];
        out[i] = mulr((R)inv, v[i]);
    } else {
        auto w = out[i];
        w = fmar((R)(-scal[ia]), v[i], w);
        if (ib >= 0) w = fmar((R)(-scal[ib]), vprev[i], w);
        out[i] = w;
    }
}

// Extreme eigenvalues of the k x k symmetric tridiagonal T (diagonal alpha, off-diagonal
// beta) on the host, by bisection on the Sturm count: the number of eigenvalues below x is
// the number of negative pivots of the LDL^T factorisation of T - x I.
int tridiag_count_below(const double* alpha, const double* beta, int k, double x) {
    int neg = 0;
    double q = 1.0;
    for (int i = 0; i < k; ++i) {
        const double b2 = i > 0 ? beta[i - 1] * beta[i - 1] : 0.0;
        q = (alpha[i] - x) - (i > 0 ? b2 / q : 0.0);
        if (q == 0.0) q = -1e-300;       // x on an eigenvalue of a leading block: count it below
        neg += q < 0.0;
    }
    return neg;
}

double tridiag_eigenvalue(const double* alpha, const double* beta, int k, int idx) {
    // Gershgorin interval, then bisection on count(x) > idx
    double lo = alpha[0], hi = alpha[0];
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? std::fabs(beta[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(beta[i]) : 0.0);
        lo = std::min(lo, alpha[i] - r);
        hi = std::max(hi, alpha[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 4e-16 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (tridiag_count_below(alpha, beta, k, mid) > idx) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

template <typename R, bool CPLX>
int dot_t(hub_t h, const void* x, const void* y, double* out, int op) {
    using T = typename VT<R, CPLX>::T;
    double* part = h->d_scal + 1024;   // d_scal holds 4096 doubles
    { ProfScope ps(h, HUB_K_LANCZOS); k_dot_partial<R, CPLX><<<RBLK, 256, 0, h->stream>>>((const T*)x, (const T*)y, h->Nd, part); }
    HUB_CUDA_TRY(h, cudaGetLastError());
    { ProfScope ps(h, HUB_K_LANCZOS); k_dot_final<<<1, RBLK, 0, h->stream>>>(part, RBLK, out, op); }
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

template <typename R, bool CPLX>
int lanczos_t(hub_t h, int spin, int steps, const void* v0, double* lo, double* up) {
    using T = typename VT<R, CPLX>::T;
    const size_t vb = (size_t)h->Nd * sizeof(T);
    int rc;
    if ((rc = ensure(h, &h->d_work, &h->work_bytes, std::max(h->work_bytes, 3 * vb)))) return rc;
    T* v = (T*)h->d_work;
    T* vp = v + h->Nd;
    T* w = vp + h->Nd;
    double* sc = h->d_scal;            // [0..63] alpha, [64..128] beta, [200..201] bounds, [210] norm
    const unsigned nb = (unsigned)((h->Nd + 255) / 256);
    if ((rc = dot_t<R, CPLX>(h, v0, v0, sc + 210, 1))) return rc;
    { ProfScope ps(h, HUB_K_LANCZOS);
    k_lanczos_axpy<R, CPLX><<<nb, 256, 0, h->stream>>>(0, v, (const T*)v0, nullptr, h->Nd, sc, 210, -1); }
    HUB_CUDA_TRY(h, cudaGetLastError());
    for (int j = 0; j < steps; ++j) {
        if ((rc = apply_H_internal(h, spin, v, (int)h->Nd, w, 1, 1.0, 0.0, nullptr, 0.0))) return rc;
        if ((rc = dot_t<R, CPLX>(h, v, w, sc + j, 0))) return rc;                    // alpha_j
        { ProfScope ps(h, HUB_K_LANCZOS);
        k_lanczos_axpy<R, CPLX><<<nb, 256, 0, h->stream>>>(1, w, v, vp, h->Nd, sc, j, j > 0 ? 64 + j - 1 : -1); }
        HUB_CUDA_TRY(h, cudaGetLastError());
        if ((rc = dot_t<R, CPLX>(h, w, w, sc + 64 + j, 1))) return rc;             // beta_{j+1}
        // vprev <- v ; v <- w / beta
        HUB_CUDA_TRY(h, cudaMemcpyAsync(vp, v, vb, cudaMemcpyDeviceToDevice, h->stream));
        { ProfScope ps(h, HUB_K_LANCZOS);
        k_lanczos_axpy<R, CPLX><<<nb, 256, 0, h->stream>>>(0, v, w, nullptr, h->Nd, sc, 64 + j, -1); }
        HUB_CUDA_TRY(h, cudaGetLastError());
    }
    // bounds from the k x k tridiagonal: lowest Ritz value, highest + |beta_k|
    double ab[128];
    HUB_CUDA_TRY(h, cudaMemcpyAsync(ab, sc, 128 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    *lo = tridiag_eigenvalue(ab, ab + 64, steps, 0);
    *up = tridiag_eigenvalue(ab, ab + 64, steps, steps - 1) + std::fabs(ab[64 + steps - 1]);
    return HUB_OK;
}

}  // namespace

int launch_copy_convert_veff(hub_t h, const double* src, void* dst) {
    const unsigned nb = (unsigned)((h->Nd + 255) / 256);
    ProfScope ps(h, HUB_K_COPY);
    if (h->esize == 8) k_convert<double><<<nb, 256, 0, h->stream>>>(src, (double*)dst, h->Nd);
    else k_convert<float><<<nb, 256, 0, h->stream>>>(src, (float*)dst, h->Nd);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int launch_copy_block(hub_t h, const void* src, int lds, void* dst, int ldd, int ncol) {
    if (ncol == 0) return HUB_OK;
    dim3 grid((unsigned)((h->Nd + 255) / 256), ncol);
    const int es = h->esize * (h->cplx ? 2 : 1);
    ProfScope ps(h, HUB_K_COPY);
    if (es == 16)
        k_copy_block<double2><<<grid, 256, 0, h->stream>>>((const double2*)src, lds, (double2*)dst, ldd, h->Nd);
    else if (es == 8)
        k_copy_block<double><<<grid, 256, 0, h->stream>>>((const double*)src, lds, (double*)dst, ldd, h->Nd);
    else
        k_copy_block<float><<<grid, 256, 0, h->stream>>>((const float*)src, lds, (float*)dst, ldd, h->Nd);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int launch_lanczos(hub_t h, int spin, int steps, const void* v0, double* lo, double* up) {
    if (h->esize == 8) return h->cplx ? lanczos_t<double, true>(h, spin, steps, v0, lo, up)
                                      : lanczos_t<double, false>(h, spin, steps, v0, lo, up);
    return h->cplx ? lanczos_t<float, true>(h, spin, steps, v0, lo, up)
                   : lanczos_t<float, false>(h, spin, steps, v0, lo, up);
}

}  // namespace hub

// ---------------------------------------------------------------------------- ALU peaks
// Throughput probe for the roofline denominators of ALU-bound kernels: eight independent
// FMA chains per thread (enough to cover the pipe latency), a full grid of 256-thread CTAs.
namespace {
template <typename T>
__global__ void k_fma_probe(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x & 7) * (T)1e-3 + (T)i;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == (T)-1.2345) out[0] = s;          // keeps the chains alive; never true
}
}  // namespace

extern "C" int hub_alu_peaks(double* fp64_gflops, double* fp32_gflops, void* cuda_stream) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HUB_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HUB_ECUDA;
    double* buf = nullptr;
    if (cudaMalloc(&buf, 16) != cudaSuccess) return HUB_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256;
    int rc = HUB_OK;
    for (int kind = 0; kind < 2 && rc == HUB_OK; ++kind) {
        const int iters = kind == 0 ? 2048 : 65536;
        float best = 1e30f;
        for (int r = 0; r < 6; ++r) {
            cudaEventRecord(e0, st);
            if (kind == 0) k_fma_probe<double><<<blocks, threads, 0, st>>>(buf, iters, 0.9999999, 1e-9);
            else k_fma_probe<float><<<blocks, threads, 0, st>>>((float*)buf, iters, 0.9999999f, 1e-9f);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = HUB_ECUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) best = std::min(best, ms);              // first launch is the warm-up
        }
        const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
        if (rc == HUB_OK) {
            if (kind == 0 && fp64_gflops) *fp64_gflops = flops / (best * 1e-3) / 1e9;
            if (kind == 1 && fp32_gflops) *fp32_gflops = flops / (best * 1e-3) / 1e9;
        }
    }
    if (cudaGetLastError() != cudaSuccess) rc = HUB_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return rc;
}

// ---------------------------------------------------------------------------- MD extrapolation
extern "C" int hub_extrapolate_occupations(int n, int nhist, const double* D_hist, const double* D_atomic,
                                           int natoms, const double* R_hist, double* coef_out, double* D_out) {
    if (n < 0 || nhist < 0 || nhist > 3 || natoms < 0) return HUB_EINVAL;
    if (n > 0 && (!D_atomic || !D_out || (nhist > 0 && !D_hist))) return HUB_EINVAL;
    if (natoms > 0 && nhist >= 2 && !R_hist) return HUB_EINVAL;
    // coefficients from the positions: nhist + 1 sets, the last one the new step
    double alpha = 0.0, beta = 0.0;
    const long m = (long)natoms * 3;
    const int npos = nhist + 1;
    if (npos >= 3 && m > 0) {
        const double* Rn = R_hist + (long)(npos - 1) * m;    // t + dt
        const double* R0 = R_hist + (long)(npos - 2) * m;    // t
        const double* R1 = R_hist + (long)(npos - 3) * m;    // t - dt
        double g11 = 0.0, g12 = 0.0, g22 = 0.0, b1 = 0.0, b2 = 0.0;
        for (long i = 0; i < m; ++i) {
            const double t = Rn[i] - R0[i], d1 = R0[i] - R1[i];
            g11 += d1 * d1;
            b1 += d1 * t;
            if (npos >= 4) {
                const double d2 = R1[i] - R_hist[(long)(npos - 4) * m + i];
                g12 += d1 * d2;
                g22 += d2 * d2;
                b2 += d2 * t;
            }
        }
        const double det = g11 * g22 - g12 * g12;
        if (npos >= 4 && det > 1e-12 * g11 * g22) {
            alpha = (g22 * b1 - g12 * b2) / det;
            beta = (g11 * b2 - g12 * b1) / det;
        } else {
            alpha = g11 > 0.0 ? b1 / g11 : 0.0;
            beta = 0.0;
        }
    }
    if (coef_out) { coef_out[0] = alpha; coef_out[1] = beta; }
    for (long q = 0; q < n; ++q) {
        const double da = D_atomic[q];
        if (nhist == 0) { D_out[q] = da; continue; }
        const double d0 = D_hist[(long)(nhist - 1) * n + q] - da;
        double v = d0;
        if (nhist >= 2) v += alpha * (d0 - (D_hist[(long)(nhist - 2) * n + q] - da));
        if (nhist >= 3) v += beta * ((D_hist[(long)(nhist - 2) * n + q] - da) - (D_hist[(long)(nhist - 3) * n + q] - da));
        D_out[q] = da + v;
    }
    return HUB_OK;
}

// ---------------------------------------------------------------------------- truncation
extern "C" int hub_cutoff_radius(int l, double rs, double tau, double* rc_out) {
    if (l < 0 || l > 2 || !(rs > 0.0) || !(tau > 0.0) || !rc_out) return HUB_EINVAL;
    const double N = std::sqrt(2.0 / (std::tgamma(l + 1.5) * std::pow(rs, 2 * l + 3)));
    auto R = [&](double r) { return N * std::pow(r, l) * std::exp(-r * r / (2.0 * rs * rs)); };
    const double rmax = rs * std::sqrt((double)l);       // R rises to here, falls after
    if (R(rmax) <= tau) { *rc_out = 0.0; return HUB_OK; }
    double lo = rmax, hi = rmax + rs;
    for (int k = 0; k < 10000 && R(hi) > tau; ++k) hi += rs;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (R(mid) > tau) lo = mid; else hi = mid;
    }
    *rc_out = 0.5 * (lo + hi);
    return HUB_OK;
}

// ---------------------------------------------------------------------------- Fermi level
extern "C" int hub_fermi_dirac(int n, const double* eig, const double* w, double kT, double n_elec,
                               double degeneracy, double* f_out, double* mu_out) {
    if (n < 1 || !eig || !w || !f_out || !(kT >= 0.0) || !(degeneracy > 0.0)) return HUB_EINVAL;
    double cap = 0.0;
    for (int i = 0; i < n; ++i) cap += w[i] * degeneracy;
    if (!(n_elec >= 0.0) || n_elec > cap * (1.0 + 1e-12)) return HUB_EINVAL;
    if (kT == 0.0) {
        // lowest states first until n_elec is reached
        std::vector<int> ord(n);
        for (int i = 0; i < n; ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return eig[a] < eig[b]; });
        double left = n_elec, mu = eig[ord[0]];
        for (int i = 0; i < n; ++i) f_out[i] = 0.0;
        for (int j = 0; j < n && left > 1e-12; ++j) {
            f_out[ord[j]] = 1.0;
            left -= w[ord[j]] * degeneracy;
            mu = eig[ord[j]];
        }
        if (mu_out) *mu_out = mu;
        return HUB_OK;
    }
    auto count = [&](double m) {
        double c = 0.0;
        for (int i = 0; i < n; ++i) c += w[i] * degeneracy * 0.5 * (1.0 - std::tanh((eig[i] - m) / (2.0 * kT)));
        return c;
    };
    double lo = eig[0], hi = eig[0];
    for (int i = 1; i < n; ++i) { lo = std::min(lo, eig[i]); hi = std::max(hi, eig[i]); }
    lo -= 50.0 * kT;
    hi += 50.0 * kT;
    for (int it = 0; it < 200; ++it) {
        const double m = 0.5 * (lo + hi);
        if (count(m) < n_elec) lo = m; else hi = m;
        if (hi - lo < 1e-15) break;
    }
    const double mu = 0.5 * (lo + hi);
    for (int i = 0; i < n; ++i) f_out[i] = 0.5 * (1.0 - std::tanh((eig[i] - mu) / (2.0 * kT)));
    if (mu_out) *mu_out = mu;
    return HUB_OK;
}

