// Warm-start model: per-atom local-environment descriptors and a SiLU multilayer
// perceptron that maps them to occupation matrices D, with hand-written forward, backward
// and Adam kernels.  (The paper has no learned component; its SCF, with D updated and mixed
// every iteration, stays the arbiter: the model only supplies the starting D.)
//
// Layers: h0 = (x - mu_in) / sd_in; h_l = silu(W_l h_{l-1} + b_l) for the hidden layers;
// y = (W_L h_{L-1} + b_L) * sd_out + mu_out.  Weights are kept in FP32 (master, Adam state)
// and, with weight_fp16, the forward and input-gradient products read an FP16 copy;
// every product accumulates in FP32.  Loss: mean of ((y - t) / sd_out)^2.
#include <cuda_fp16.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hub_internal.cuh"

struct hub_mlp_ctx {
    int n_in = 0, n_hidden = 0, n_layers = 0, n_out = 0, fp16 = 0;
    cudaStream_t stream = nullptr;
    std::vector<int> in_dim, out_dim;         // per linear layer
    std::vector<long> w_off, b_off;           // offsets into the flat parameter vector
    long nparams = 0;
    float* d_p = nullptr;                     // FP32 parameters (flat)
    __half* d_ph = nullptr;                   // FP16 copy of the parameters
    float* d_g = nullptr;                     // gradients
    float* d_m = nullptr;                     // Adam first moments
    float* d_v = nullptr;                     // Adam second moments
    float* d_norm = nullptr;                  // mu_in, sd_in, mu_out, sd_out
    float* d_act = nullptr;                   // activations and pre-activations
    size_t act_cap = 0;                       // batch capacity of d_act
    float* d_loss = nullptr;
    int adam_t = 0;
    std::string last_error;
};

namespace hub {
namespace {

constexpr int MT = 64, KT = 16;

// C[M x N] = opA(A) opB(B): A is [M x K] (lda) or, with TA, stored [K x M]; B is [K x N]
// or, with TB, stored [N x K]; B elements of type BT.  Epilogue mode:
//   0: C = acc;  1: Z = acc + bias, C = silu(Z);  2: Z = acc + bias, C = Z
template <bool TA, bool TB, typename BT>
__global__ void __launch_bounds__(256)
k_mm(int M, int N, int K, const float* __restrict__ A, int lda, const BT* __restrict__ B, int ldb,
     float* __restrict__ C, int ldc, const float* __restrict__ bias, float* __restrict__ Z, int mode) {
    __shared__ float As[KT][MT + 1], Bs[KT][MT + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * MT, n0 = blockIdx.x * MT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += KT) {
        for (int e = threadIdx.x; e < KT * MT; e += 256) {
            int kk, mm;
            if (TA) { mm = e % MT; kk = e / MT; } else { kk = e % KT; mm = e / KT; }
            const int gm = m0 + mm, gk = k0 + kk;
            float a = 0.f;
            if (gm < M && gk < K) a = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            As[kk][mm] = a;
            int nn;
            if (TB) { kk = e % KT; nn = e / KT; } else { nn = e % MT; kk = e / MT; }
            const int gn = n0 + nn, gk2 = k0 + kk;
            float b = 0.f;
            if (gn < N && gk2 < K) b = (float)(TB ? B[(size_t)gn * ldb + gk2] : B[(size_t)gk2 * ldb + gn]);
            Bs[kk][nn] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) { a[r] = As[kk][ty + 16 * r]; b[r] = Bs[kk][tx + 16 * r]; }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int m = m0 + ty + 16 * r, n = n0 + tx + 16 * c;
            if (m >= M || n >= N) continue;
            float v = acc[r][c];
            if (mode >= 1) {
                v += bias[n];
                Z[(size_t)m * ldc + n] = v;
                if (mode == 1) v = v / (1.f + expf(-v));
            }
            C[(size_t)m * ldc + n] = v;
        }
}

// dZ = dH * silu'(Z)
__global__ void k_silu_bwd(float* __restrict__ dH, const float* __restrict__ Z, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float z = Z[i];
    const float s = 1.f / (1.f + expf(-z));
    dH[i] *= s * (1.f + z * (1.f - s));
}

// db[n] = sum_b dZ[b, n]   (fixed order: deterministic)
__global__ void k_colsum(const float* __restrict__ dZ, int B, int N, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dZ[(size_t)b * N + n];
    db[n] = s;
}

// y = z * sd_out + mu_out
__global__ void k_denorm(const float* __restrict__ z, int B, int N, const float* __restrict__ mu,
                         const float* __restrict__ sd, float* __restrict__ y) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)B * N) return;
    const int n = (int)(i % N);
    y[i] = z[i] * sd[n] + mu[n];
}

// r = z - (t - mu) / sd;  loss = mean r^2;  dz = 2 r / (B N)   (one block, fixed order)
__global__ void k_mse(const float* __restrict__ z, const float* __restrict__ t, int B, int N,
                      const float* __restrict__ mu, const float* __restrict__ sd, float* __restrict__ dz,
                      float* __restrict__ loss) {
    __shared__ double red[1024];
    double acc = 0.0;
    const long tot = (long)B * N;
    for (long i = threadIdx.x; i < tot; i += blockDim.x) {
        const int n = (int)(i % N);
        const float r = z[i] - (t[i] - mu[n]) / sd[n];
        dz[i] = 2.f * r / (float)tot;
        acc += (double)r * r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(red[0] / (double)tot);
}

__global__ void k_adam(float* __restrict__ p, __half* __restrict__ ph, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    ph[i] = __float2half_rn(w);
}

__global__ void k_standardise(const float* __restrict__ X, int B, int N, const float* __restrict__ mu,
                              const float* __restrict__ sd, float* __restrict__ H) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)B * N) return;
    const int n = (int)(i % N);
    H[i] = (X[i] - mu[n]) / sd[n];
}

__global__ void k_to_half(const float* __restrict__ p, __half* __restrict__ ph, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ph[i] = __float2half_rn(p[i]);
}

// column mean and standard deviation (population), sd floored at 1e-6 (one thread per column)
__global__ void k_colstats(const float* __restrict__ X, int rows, int cols, float* __restrict__ mu,
                           float* __restrict__ sd) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0, s2 = 0.0;
    for (int r = 0; r < rows; ++r) {
        const double x = X[(size_t)r * cols + c];
        s += x;
        s2 += x * x;
    }
    const double m = s / rows;
    mu[c] = (float)m;
    sd[c] = (float)fmax(sqrt(fmax(s2 / rows - m * m, 0.0)), 1e-6);
}

__device__ void ylm_unit(double x, double y, double z, double* o) {
    const double PI = 3.14159265358979323846;
    const double k = sqrt(3.0 / (4.0 * PI));
    o[0] = k * y; o[1] = k * z; o[2] = k * x;
    const double k1 = 0.5 * sqrt(15.0 / PI), k0 = 0.25 * sqrt(5.0 / PI), k2 = 0.25 * sqrt(15.0 / PI);
    o[3] = k1 * x * y; o[4] = k1 * y * z; o[5] = k0 * (2 * z * z - x * x - y * y); o[6] = k1 * x * z;
    o[7] = k2 * (x * x - y * y);
}

// one thread per centre atom: radial Gaussians and l = 1, 2 harmonic sums per neighbour
// species over all periodic images within rc, cosine cutoff (double accumulation)
__global__ void k_descriptors(int natoms, const double* __restrict__ pos, const int* __restrict__ species,
                              double L0, double L1, double L2, int ncenter, const int* __restrict__ centers,
                              int nspecies, double rc, int nrad, double eta, int t0, int t1, int t2,
                              float* __restrict__ out) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= ncenter) return;
    const int nf = nrad + 8, F = nspecies * nf;
    const int I = centers[ci];
    double acc[2 * (32 + 8)];
    for (int f = 0; f < F; ++f) acc[f] = 0.0;
    const double PI = 3.14159265358979323846;
    for (int J = 0; J < natoms; ++J) {
        const int s = species[J];
        for (int a = -t0; a <= t0; ++a)
            for (int b = -t1; b <= t1; ++b)
                for (int c = -t2; c <= t2; ++c) {
                    const double dx = pos[3 * J] + a * L0 - pos[3 * I];
                    const double dy = pos[3 * J + 1] + b * L1 - pos[3 * I + 1];
                    const double dz = pos[3 * J + 2] + c * L2 - pos[3 * I + 2];
                    const double r = sqrt(dx * dx + dy * dy + dz * dz);
                    if (r < 1e-8 || r >= rc) continue;
                    const double fc = 0.5 * (cos(PI * r / rc) + 1.0);
                    double* o = acc + s * nf;
                    for (int k = 0; k < nrad; ++k) {
                        const double mu = 0.5 + (rc - 1.0) * k / (nrad > 1 ? nrad - 1 : 1);
                        o[k] += exp(-(r - mu) * (r - mu) / (2.0 * eta * eta)) * fc;
                    }
                    double y[8];
                    ylm_unit(dx / r, dy / r, dz / r, y);
                    for (int q = 0; q < 8; ++q) o[nrad + q] += y[q] * fc;
                }
    }
    for (int f = 0; f < F; ++f) out[(size_t)ci * F + f] = (float)acc[f];
}

int mfail(hub_mlp_t m, int code, const std::string& msg) {
    if (m) m->last_error = msg;
    return code;
}

#define MLP_TRY(m, expr)                                                                    \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) return mfail((m), HUB_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

template <bool TA, bool TB, typename BT>
int mm(hub_mlp_t m, int M, int N, int K, const float* A, int lda, const BT* B, int ldb, float* C, int ldc,
       const float* bias, float* Z, int mode) {
    dim3 grid((N + MT - 1) / MT, (M + MT - 1) / MT);
    k_mm<TA, TB, BT><<<grid, 256, 0, m->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Z, mode);
    MLP_TRY(m, cudaGetLastError());
    return HUB_OK;
}

// activation layout for batch B: the standardised input [B x n_in], then for every linear
// layer l, Z_l and H_l of [B x out_dim[l]], then two scratch blocks [B x max width] for
// gradients
size_t act_floats(hub_mlp_t m, int B) {
    size_t s = (size_t)B * m->n_in;
    int wmax = m->n_in;
    for (size_t l = 0; l < m->out_dim.size(); ++l) {
        s += 2 * (size_t)B * m->out_dim[l];
        wmax = std::max(wmax, m->out_dim[l]);
    }
    return s + 2 * (size_t)B * wmax;
}

int ensure_act(hub_mlp_t m, int B) {
    if ((size_t)B <= m->act_cap && m->d_act) return HUB_OK;
    if (m->d_act) cudaFree(m->d_act);
    m->d_act = nullptr;
    if (cudaMalloc(&m->d_act, act_floats(m, B) * sizeof(float)) != cudaSuccess)
        return mfail(m, HUB_ENOMEM, "activation buffer");
    m->act_cap = B;
    return HUB_OK;
}

// forward pass storing Z_l, H_l; returns pointer to the last layer's Z (normalised output)
int forward(hub_mlp_t m, const float* X, int B, const float** zlast) {
    int rc;
    if ((rc = ensure_act(m, B))) return rc;
    const int nl = (int)m->out_dim.size();
    float* base = m->d_act;
    k_standardise<<<(unsigned)(((long)B * m->n_in + 255) / 256), 256, 0, m->stream>>>(
        X, B, m->n_in, m->d_norm, m->d_norm + m->n_in, base);
    MLP_TRY(m, cudaGetLastError());
    const float* H = base;
    base += (size_t)B * m->n_in;
    int ldh = m->n_in;
    for (int l = 0; l < nl; ++l) {
        const int N = m->out_dim[l], K = m->in_dim[l];
        float* Z = base;
        float* Ho = base + (size_t)B * N;
        base += 2 * (size_t)B * N;
        const int mode = l < nl - 1 ? 1 : 2;
        if (m->fp16)
            rc = mm<false, true, __half>(m, B, N, K, H, ldh, m->d_ph + m->w_off[l], K, Ho, N, m->d_p + m->b_off[l], Z, mode);
        else
            rc = mm<false, true, float>(m, B, N, K, H, ldh, m->d_p + m->w_off[l], K, Ho, N, m->d_p + m->b_off[l], Z, mode);
        if (rc) return rc;
        H = Ho;
        ldh = N;
        if (l == nl - 1) *zlast = Z;
    }
    return HUB_OK;
}

// loss and gradients into d_g (and the loss into d_loss)
int backward(hub_mlp_t m, const float* X, const float* T, int B) {
    int rc;
    const float* zlast = nullptr;
    if ((rc = forward(m, X, B, &zlast))) return rc;
    const int nl = (int)m->out_dim.size();
    std::vector<float*> Z(nl), H(nl);
    float* h0 = m->d_act;                           // standardised input
    float* base = m->d_act + (size_t)B * m->n_in;
    for (int l = 0; l < nl; ++l) {
        Z[l] = base;
        H[l] = base + (size_t)B * m->out_dim[l];
        base += 2 * (size_t)B * m->out_dim[l];
    }
    int wmax = m->n_in;
    for (int l = 0; l < nl; ++l) wmax = std::max(wmax, m->out_dim[l]);
    float* g0 = base;
    float* g1 = base + (size_t)B * wmax;
    const float* mu_out = m->d_norm + 2 * m->n_in;
    const float* sd_out = mu_out + m->n_out;
    k_mse<<<1, 1024, 0, m->stream>>>(zlast, T, B, m->n_out, mu_out, sd_out, g0, m->d_loss);
    MLP_TRY(m, cudaGetLastError());
    // g0 = d loss / d Z_L; walk back
    float* dZ = g0;
    float* other = g1;
    for (int l = nl - 1; l >= 0; --l) {
        const int N = m->out_dim[l], K = m->in_dim[l];
        // dW_l = dZ^T H_{l-1}, H_{-1} = standardised input:
        // C[N x K] = dZ^T [N x B] * Hin [B x K] (A = dZ stored [B x N], transposed)
        const float* Hin = l == 0 ? h0 : H[l - 1];
        if ((rc = mm<true, false, float>(m, N, K, B, dZ, N, Hin, K, m->d_g + m->w_off[l], K, nullptr, nullptr, 0)))
            return rc;
        k_colsum<<<(N + 127) / 128, 128, 0, m->stream>>>(dZ, B, N, m->d_g + m->b_off[l]);
        MLP_TRY(m, cudaGetLastError());
        if (l == 0) break;
        // dH_{l-1} = dZ W_l  ([B x N] x [N x K])
        if (m->fp16)
            rc = mm<false, false, __half>(m, B, K, N, dZ, N, m->d_ph + m->w_off[l], K, other, K, nullptr, nullptr, 0);
        else
            rc = mm<false, false, float>(m, B, K, N, dZ, N, m->d_p + m->w_off[l], K, other, K, nullptr, nullptr, 0);
        if (rc) return rc;
        k_silu_bwd<<<(unsigned)(((long)B * K + 255) / 256), 256, 0, m->stream>>>(other, Z[l - 1], (long)B * K);
        MLP_TRY(m, cudaGetLastError());
        std::swap(dZ, other);
    }
    return HUB_OK;
}

}  // namespace
}  // namespace hub

using namespace hub;

extern "C" {

int hub_mlp_create(hub_mlp_t* out, int n_in, int n_hidden, int n_layers, int n_out, int weight_fp16,
                   unsigned long long seed, void* stream) {
    if (!out || n_in < 1 || n_hidden < 1 || n_layers < 1 || n_out < 1) return HUB_EINVAL;
    hub_mlp_t m = new (std::nothrow) hub_mlp_ctx();
    if (!m) return HUB_ENOMEM;
    m->n_in = n_in; m->n_hidden = n_hidden; m->n_layers = n_layers; m->n_out = n_out;
    m->fp16 = weight_fp16 ? 1 : 0;
    m->stream = (cudaStream_t)stream;
    int prev = n_in;
    for (int l = 0; l <= n_layers; ++l) {
        const int o = l < n_layers ? n_hidden : n_out;
        m->in_dim.push_back(prev);
        m->out_dim.push_back(o);
        m->w_off.push_back(m->nparams);
        m->nparams += (long)o * prev;
        m->b_off.push_back(m->nparams);
        m->nparams += o;
        prev = o;
    }
    // seeded U(-1/sqrt(in), 1/sqrt(in)) initialisation with a counter-based generator
    // (SplitMix64 of seed + index), done once on the host
    std::vector<float> p(m->nparams);
    for (size_t l = 0; l < m->in_dim.size(); ++l) {
        const double k = 1.0 / std::sqrt((double)m->in_dim[l]);
        const long n = (long)m->out_dim[l] * m->in_dim[l] + m->out_dim[l];
        for (long i = 0; i < n; ++i) {
            unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(m->w_off[l] + i + 1);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            const double u = (double)(z >> 11) / 9007199254740992.0;
            p[m->w_off[l] + i] = (float)((2.0 * u - 1.0) * k);
        }
    }
    const size_t pb = m->nparams * sizeof(float);
    cudaError_t e = cudaMalloc(&m->d_p, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_ph, m->nparams * sizeof(__half));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_g, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_m, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_v, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_norm, (2 * n_in + 2 * n_out) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(m->d_p, p.data(), pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, pb);
    if (e == cudaSuccess) {
        std::vector<float> norm(2 * n_in + 2 * n_out);
        for (int i = 0; i < n_in; ++i) { norm[i] = 0.f; norm[n_in + i] = 1.f; }
        for (int i = 0; i < n_out; ++i) { norm[2 * n_in + i] = 0.f; norm[2 * n_in + n_out + i] = 1.f; }
        e = cudaMemcpy(m->d_norm, norm.data(), norm.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        hub_mlp_destroy(m);
        return HUB_ENOMEM;
    }
    k_to_half<<<(unsigned)((m->nparams + 255) / 256), 256, 0, m->stream>>>(m->d_p, m->d_ph, m->nparams);
    *out = m;
    return cudaGetLastError() == cudaSuccess ? HUB_OK : HUB_ECUDA;
}

int hub_mlp_destroy(hub_mlp_t m) {
    if (!m) return HUB_OK;
    cudaStreamSynchronize(m->stream);
    void* ptrs[] = {m->d_p, m->d_ph, m->d_g, m->d_m, m->d_v, m->d_norm, m->d_act, m->d_loss};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete m;
    return HUB_OK;
}

const char* hub_mlp_last_error(hub_mlp_t m) { return m ? m->last_error.c_str() : "NULL model"; }

int hub_mlp_num_params(hub_mlp_t m, long long* n) {
    if (!m || !n) return HUB_EINVAL;
    *n = m->nparams;
    return HUB_OK;
}

int hub_mlp_set_params(hub_mlp_t m, const float* host) {
    if (!m || !host) return HUB_EINVAL;
    MLP_TRY(m, cudaMemcpyAsync(m->d_p, host, m->nparams * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    k_to_half<<<(unsigned)((m->nparams + 255) / 256), 256, 0, m->stream>>>(m->d_p, m->d_ph, m->nparams);
    MLP_TRY(m, cudaGetLastError());
    MLP_TRY(m, cudaMemsetAsync(m->d_m, 0, m->nparams * sizeof(float), m->stream));
    MLP_TRY(m, cudaMemsetAsync(m->d_v, 0, m->nparams * sizeof(float), m->stream));
    m->adam_t = 0;
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    return HUB_OK;
}

int hub_mlp_get_params(hub_mlp_t m, float* host) {
    if (!m || !host) return HUB_EINVAL;
    MLP_TRY(m, cudaMemcpyAsync(host, m->d_p, m->nparams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    return HUB_OK;
}

int hub_mlp_set_normalization(hub_mlp_t m, const float* mu_in, const float* sd_in, const float* mu_out,
                              const float* sd_out) {
    if (!m || !mu_in || !sd_in || !mu_out || !sd_out) return HUB_EINVAL;
    std::vector<float> v(2 * m->n_in + 2 * m->n_out);
    std::copy(mu_in, mu_in + m->n_in, v.begin());
    std::copy(sd_in, sd_in + m->n_in, v.begin() + m->n_in);
    std::copy(mu_out, mu_out + m->n_out, v.begin() + 2 * m->n_in);
    std::copy(sd_out, sd_out + m->n_out, v.begin() + 2 * m->n_in + m->n_out);
    MLP_TRY(m, cudaMemcpyAsync(m->d_norm, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    return HUB_OK;
}

int hub_mlp_fit_normalization(hub_mlp_t m, const float* X, const float* T, int B) {
    if (!m || !X || !T || B < 1) return HUB_EINVAL;
    k_colstats<<<(m->n_in + 127) / 128, 128, 0, m->stream>>>(X, B, m->n_in, m->d_norm, m->d_norm + m->n_in);
    k_colstats<<<(m->n_out + 127) / 128, 128, 0, m->stream>>>(T, B, m->n_out, m->d_norm + 2 * m->n_in,
                                                              m->d_norm + 2 * m->n_in + m->n_out);
    MLP_TRY(m, cudaGetLastError());
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    return HUB_OK;
}

int hub_mlp_forward(hub_mlp_t m, const float* X, int B, float* Y) {
    if (!m || !X || !Y || B < 1) return HUB_EINVAL;
    const float* z = nullptr;
    int rc = forward(m, X, B, &z);
    if (rc) return rc;
    k_denorm<<<(unsigned)(((long)B * m->n_out + 255) / 256), 256, 0, m->stream>>>(
        z, B, m->n_out, m->d_norm + 2 * m->n_in, m->d_norm + 2 * m->n_in + m->n_out, Y);
    MLP_TRY(m, cudaGetLastError());
    return HUB_OK;
}

int hub_mlp_loss_grad(hub_mlp_t m, const float* X, const float* T, int B, float* loss, float* grad_host) {
    if (!m || !X || !T || B < 1) return HUB_EINVAL;
    int rc = backward(m, X, T, B);
    if (rc) return rc;
    if (loss) MLP_TRY(m, cudaMemcpyAsync(loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    if (grad_host)
        MLP_TRY(m, cudaMemcpyAsync(grad_host, m->d_g, m->nparams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    return HUB_OK;
}

int hub_mlp_train_step(hub_mlp_t m, const float* X, const float* T, int B, float lr, float* loss) {
    if (!m || !X || !T || B < 1 || !(lr > 0)) return HUB_EINVAL;
    int rc = backward(m, X, T, B);
    if (rc) return rc;
    m->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
    k_adam<<<(unsigned)((m->nparams + 255) / 256), 256, 0, m->stream>>>(m->d_p, m->d_ph, m->d_g, m->d_m, m->d_v,
                                                                       m->nparams, lr, b1, b2, 1e-8f, c1, c2);
    MLP_TRY(m, cudaGetLastError());
    if (loss) {
        MLP_TRY(m, cudaMemcpyAsync(loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        MLP_TRY(m, cudaStreamSynchronize(m->stream));
    }
    return HUB_OK;
}

int hub_descriptors(int natoms, const double* pos, const int* species, const double* L, int ncenter,
                    const int* centers, int nspecies, double rc, int nrad, double eta, float* out_dev,
                    void* stream) {
    if (natoms < 1 || !pos || !species || !L || ncenter < 0 || (ncenter > 0 && (!centers || !out_dev)) ||
        nspecies < 1 || nspecies > 2 || nrad < 1 || nrad > 32 || !(rc > 0) || !(eta > 0))
        return HUB_EINVAL;
    if (ncenter == 0) return HUB_OK;
    for (int i = 0; i < natoms; ++i)
        if (species[i] < 0 || species[i] >= nspecies) return HUB_EINVAL;
    for (int i = 0; i < ncenter; ++i)
        if (centers[i] < 0 || centers[i] >= natoms) return HUB_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    double* dpos = nullptr;
    int* dsp = nullptr;
    int* dc = nullptr;
    cudaError_t e = cudaMallocAsync(&dpos, natoms * 3 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dsp, natoms * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dc, ncenter * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dpos, pos, natoms * 3 * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dsp, species, natoms * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dc, centers, ncenter * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const int t0 = (int)std::ceil(rc / L[0]) + 1, t1 = (int)std::ceil(rc / L[1]) + 1, t2 = (int)std::ceil(rc / L[2]) + 1;
        k_descriptors<<<(ncenter + 63) / 64, 64, 0, st>>>(natoms, dpos, dsp, L[0], L[1], L[2], ncenter, dc, nspecies,
                                                         rc, nrad, eta, t0, t1, t2, out_dev);
        e = cudaGetLastError();
    }
    if (dpos) cudaFreeAsync(dpos, st);
    if (dsp) cudaFreeAsync(dsp, st);
    if (dc) cudaFreeAsync(dc, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? HUB_OK : HUB_ECUDA;
}

}  // extern "C"
