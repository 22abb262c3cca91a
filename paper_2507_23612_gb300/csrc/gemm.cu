// Rayleigh-Ritz block products (CheFSI, Sec. II.B) on CUDA cores:
//   Gram / projected Hamiltonian  G = alpha * A^H B   (A, B tall: Nd x m, Nd x n)
//   rotation                      Y = X Q             (X tall: Nd x k, Q small k x n)
// Real blocks (Gamma point) and complex blocks (Bloch orbitals, interleaved re/im; G and Q
// then complex double2) share the kernels.  The tall dimension is split over CTAs (split-K);
// every CTA writes a double partial tile and a second kernel sums the partials in a fixed
// order (deterministic).
#include <mutex>
#include <type_traits>

#include "hub_internal.cuh"
#include "cplx.cuh"

namespace hub {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// the double type a working-type element accumulates into across splits
template <typename T> struct Wide { using type = double; };
template <> struct Wide<float2> { using type = double2; };
template <> struct Wide<double2> { using type = double2; };
__device__ __forceinline__ double widen(float a) { return (double)a; }
__device__ __forceinline__ double widen(double a) { return a; }
__device__ __forceinline__ double2 widen(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 widen(double2 a) { return a; }
// a double (complex) coefficient in the working type
template <typename T> __device__ __forceinline__ T narrow(double a) { return (T)a; }
template <typename T> __device__ __forceinline__ T narrow(double2 a);
template <> __device__ __forceinline__ float2 narrow<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 narrow<double2>(double2 a) { return a; }

// partial[z][i][j] = sum_{k in chunk z} conj(A[k, i]) B[k, j] over TB x TB tiles; (TB/4)^2
// threads, 4 x 4 outputs each.  Smaller tiles waste less on the ragged edge and on the
// diagonal tiles of a symmetric product.
template <typename T, int TB>
__global__ void __launch_bounds__((TB / 4) * (TB / 4))
k_gram_partial(const T* __restrict__ A, int lda, const T* __restrict__ B, int ldb, long K, int m,
               int n, long chunk, int tn, int sym, typename Wide<T>::type* __restrict__ part) {
    constexpr int TT = TB / 4, NTH = TT * TT;
    __shared__ T As[BK][TB + 1];
    __shared__ T Bs[BK][TB + 1];
    const int bi = blockIdx.x / tn, bj = blockIdx.x % tn;
    if (sym && bi > bj) return;          // mirrored by the reduction
    const int i0 = bi * TB, j0 = bj * TB;
    const long k0 = (long)blockIdx.y * chunk;
    const long k1 = min(K, k0 + chunk);
    const int tx = threadIdx.x % TT, ty = threadIdx.x / TT;
    const T zero = zero_of(T());
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = zero;
    for (long kb = k0; kb < k1; kb += BK) {
        // TB columns x 16 rows of each operand; k is the contiguous index
        for (int e = threadIdx.x; e < BK * TB; e += NTH) {
            const int kk = e % BK, ii = e / BK;
            const long k = kb + kk;
            const int i = i0 + ii, j = j0 + ii;
            As[kk][ii] = (k < k1 && i < m) ? A[(size_t)i * lda + k] : zero;
            Bs[kk][ii] = (k < k1 && j < n) ? B[(size_t)j * ldb + k] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) { a[r] = As[kk][ty + TT * r]; b[r] = Bs[kk][tx + TT * r]; }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = cfma_conj(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
    typename Wide<T>::type* P = part + (size_t)blockIdx.y * m * n;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = i0 + ty + TT * r, j = j0 + tx + TT * c;
            if (i < m && j < n) P[(size_t)i * n + j] = widen(acc[r][c]);
        }
}

// G = alpha * sum of the partials; a symmetric (Hermitian) product mirrors the lower blocks
template <typename PT>
__global__ void k_gram_reduce(const PT* __restrict__ part, int splits, int m, int n, double alpha,
                              int sym, int tb, PT* __restrict__ G) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)m * n) return;
    int i = (int)(t / n), j = (int)(t % n);
    const bool mirror = sym && (i / tb) > (j / tb);
    if (mirror) {                        // lower blocks were not computed
        const int tmp = i; i = j; j = tmp;
    }
    PT s = zero_of(PT());
    for (int z = 0; z < splits; ++z) s = add(s, part[(size_t)z * m * n + (size_t)i * n + j]);
    G[t] = mulr(alpha, mirror ? cconj(s) : s);
}

// Y[r, j] = sum_kk X[r, kk] Q[kk, j]; Q row-major double (complex: double2) [k x n]
template <typename T>
__global__ void __launch_bounds__(256)
k_rotate(const T* __restrict__ X, int ldx, const typename Wide<T>::type* __restrict__ Q, int k, int n, long K,
         T* __restrict__ Y, int ldy) {
    __shared__ T Xs[BK][BM + 1];
    __shared__ T Qs[BK][BN + 1];
    const long r0 = (long)blockIdx.x * BM;
    const int j0 = blockIdx.y * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const T zero = zero_of(T());
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = zero;
    for (int kb = 0; kb < k; kb += BK) {
        for (int e = threadIdx.x; e < BK * BM; e += 256) {
            const int rr = e % BM, kk = e / BM;
            const long r = r0 + rr;
            Xs[kk][rr] = (r < K && kb + kk < k) ? X[(size_t)(kb + kk) * ldx + r] : zero;
            const int jj = e % BN, kq = e / BN;
            Qs[kq][jj] = (kb + kq < k && j0 + jj < n) ? narrow<T>(Q[(size_t)(kb + kq) * n + j0 + jj]) : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) { a[r] = Xs[kk][tx + 16 * r]; b[r] = Qs[kk][ty + 16 * r]; }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = cfma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int j = j0 + ty + 16 * c;
        if (j >= n) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const long row = r0 + tx + 16 * r;
            if (row < K) Y[(size_t)j * ldy + row] = acc[r][c];
        }
    }
}

// Real float rotation Y = X Q with 8 x 8 outputs per thread: 128 rows x 64 columns per CTA
// of 128 threads; 16-deep slices of X (16-byte loads along the rows) and of Q (double,
// rounded to float) in shared memory.  Requires 16-byte aligned X and Y with ldx, ldy
// multiples of 4.
constexpr int R8_BM = 128, R8_BN = 64, R8_BK = 16;
__global__ void __launch_bounds__(128)
k_rotate_f32x8(const float* __restrict__ X, int ldx, const double* __restrict__ Q, int k, int n, long K,
               float* __restrict__ Y, int ldy) {
    __shared__ __align__(16) float Xs[R8_BK][R8_BM + 4];
    __shared__ __align__(16) float Qs[R8_BK][R8_BN + 4];
    const long r0 = (long)blockIdx.x * R8_BM;
    const int j0 = blockIdx.y * R8_BN;
    const int t = threadIdx.x, tx = t % 8, ty = t / 8;
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
    // the next k-slice's loads fly while the current one is multiplied
    float4 xv[4];
    float qv[8];
    auto load = [&](int kb) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = t + 128 * q;
            const int kk = e / 32, rv = e % 32;
            const long r = r0 + 4 * rv;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kb + kk < k) {
                const float* src = X + (size_t)(kb + kk) * ldx;
                if (r + 3 < K) v = *reinterpret_cast<const float4*>(src + r);
                else {
                    if (r < K) v.x = src[r];
                    if (r + 1 < K) v.y = src[r + 1];
                    if (r + 2 < K) v.z = src[r + 2];
                }
            }
            xv[q] = v;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = t + 128 * q;
            const int kq = e / 64, jj = e % 64;
            qv[q] = (kb + kq < k && j0 + jj < n) ? (float)Q[(size_t)(kb + kq) * n + j0 + jj] : 0.f;
        }
    };
    if (k > 0) load(0);
    for (int kb = 0; kb < k; kb += R8_BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = t + 128 * q;
            *reinterpret_cast<float4*>(&Xs[e / 32][4 * (e % 32)]) = xv[q];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = t + 128 * q;
            Qs[e / 64][e % 64] = qv[q];
        }
        __syncthreads();
        if (kb + R8_BK < k) load(kb + R8_BK);
#pragma unroll
        for (int kk = 0; kk < R8_BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Xs[kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Xs[kk][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Qs[kk][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Qs[kk][tx * 8 + 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
    const long rb = r0 + ty * 8;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int j = j0 + tx * 8 + c;
        if (j >= n) continue;
        float* dst = Y + (size_t)j * ldy + rb;
        if (rb + 7 < K) {
            *reinterpret_cast<float4*>(dst) = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
            *reinterpret_cast<float4*>(dst + 4) = make_float4(acc[4][c], acc[5][c], acc[6][c], acc[7][c]);
        } else {
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (rb + r < K) dst[r] = acc[r][c];
        }
    }
}

template <typename T, int TB>
int gram_tiles(hub_t h, const void* A, int lda, const void* B, int ldb, int m, int n, double alpha,
               bool sym, double* G) {
    using PT = typename Wide<T>::type;
    const int tm = (m + TB - 1) / TB, tn = (n + TB - 1) / TB;
    const long ntiles = sym ? (long)tm * (tm + 1) / 2 : (long)tm * tn;
    const long K = h->Nd;
    constexpr int per_sm = 4 * 256 / ((TB / 4) * (TB / 4));      // resident CTAs of this shape
    int splits = (int)((per_sm * (long)h->num_sms + ntiles - 1) / ntiles);
    long chunk = (K + splits - 1) / splits;
    chunk = ((chunk + BK - 1) / BK) * BK;
    if (chunk < 4 * BK) chunk = 4 * BK;
    splits = (int)((K + chunk - 1) / chunk);
    int rc;
    if ((rc = ensure(h, &h->d_gpart, &h->gpart_bytes, (size_t)splits * m * n * sizeof(PT))))
        return rc;
    PT* part = (PT*)h->d_gpart;
    dim3 grid((unsigned)(tm * tn), splits);
    { ProfScope ps(h, HUB_K_GRAM);
    k_gram_partial<T, TB><<<grid, (TB / 4) * (TB / 4), 0, h->stream>>>((const T*)A, lda, (const T*)B, ldb, K, m, n,
                                                                       chunk, tn, sym ? 1 : 0, part); }
    HUB_CUDA_TRY(h, cudaGetLastError());
    const long tot = (long)m * n;
    { ProfScope ps(h, HUB_K_GRAM_REDUCE);
    k_gram_reduce<PT><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(part, splits, m, n, alpha,
                                                                            sym ? 1 : 0, TB, (PT*)G); }
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

// Real float Gram product with 8 x 8 outputs per thread: 64 x 64 tiles, 64 threads, the
// 16-deep k-slices of both operands staged in shared memory (each thread copies one column
// of each tile in 16-byte loads), every k step two 16-byte shared loads per operand for 64
// FMAs (the 4 x 4 kernel needs one shared load per two FMAs and was bound by them).
// Requires 16-byte aligned operands with lda, ldb multiples of 4.
constexpr int G8_TB = 64, G8_BK = 16;
__global__ void __launch_bounds__(64)
k_gram_f32x8(const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb, long K, int m, int n,
             long chunk, int tn, int sym, double* __restrict__ part) {
    __shared__ __align__(16) float As[G8_BK][G8_TB + 4];
    __shared__ __align__(16) float Bs[G8_BK][G8_TB + 4];
    const int bi = blockIdx.x / tn, bj = blockIdx.x % tn;
    if (sym && bi > bj) return;          // mirrored by the reduction
    const int i0 = bi * G8_TB, j0 = bj * G8_TB;
    const long k0 = (long)blockIdx.y * chunk;
    const long k1 = min(K, k0 + chunk);
    const int t = threadIdx.x, tx = t % 8, ty = t / 8;
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
    const float* Ac = (i0 + t < m) ? A + (size_t)(i0 + t) * lda : nullptr;   // this thread's columns
    const float* Bc = (j0 + t < n) ? B + (size_t)(j0 + t) * ldb : nullptr;
    // the next k-slice's loads fly while the current one is multiplied
    float av[G8_BK], bv[G8_BK];
    auto load = [&](long kb) {
        if (kb + G8_BK <= k1) {
#pragma unroll
            for (int q = 0; q < G8_BK / 4; ++q) {
                const float4 x = Ac ? *reinterpret_cast<const float4*>(Ac + kb + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 y = Bc ? *reinterpret_cast<const float4*>(Bc + kb + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
                av[4 * q] = x.x; av[4 * q + 1] = x.y; av[4 * q + 2] = x.z; av[4 * q + 3] = x.w;
                bv[4 * q] = y.x; bv[4 * q + 1] = y.y; bv[4 * q + 2] = y.z; bv[4 * q + 3] = y.w;
            }
        } else {
#pragma unroll
            for (int kk = 0; kk < G8_BK; ++kk) {
                av[kk] = (Ac && kb + kk < k1) ? Ac[kb + kk] : 0.f;
                bv[kk] = (Bc && kb + kk < k1) ? Bc[kb + kk] : 0.f;
            }
        }
    };
    if (k0 < k1) load(k0);
    for (long kb = k0; kb < k1; kb += G8_BK) {
#pragma unroll
        for (int kk = 0; kk < G8_BK; ++kk) {
            As[kk][t] = av[kk];
            Bs[kk][t] = bv[kk];
        }
        __syncthreads();
        if (kb + G8_BK < k1) load(kb + G8_BK);
#pragma unroll
        for (int kk = 0; kk < G8_BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
    double* P = part + (size_t)blockIdx.y * m * n;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int i = i0 + ty * 8 + r;
        if (i >= m) continue;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int j = j0 + tx * 8 + c;
            if (j < n) P[(size_t)i * n + j] = (double)acc[r][c];
        }
    }
}

int gram_f32x8(hub_t h, const float* A, int lda, const float* B, int ldb, int m, int n, double alpha, bool sym,
               double* G) {
    const int tm = (m + G8_TB - 1) / G8_TB, tn = (n + G8_TB - 1) / G8_TB;
    const long ntiles = sym ? (long)tm * (tm + 1) / 2 : (long)tm * tn;
    const long K = h->Nd;
    int splits = (int)((8L * h->num_sms + ntiles - 1) / ntiles);
    long chunk = (K + splits - 1) / splits;
    chunk = ((chunk + G8_BK - 1) / G8_BK) * G8_BK;
    if (chunk < 4 * G8_BK) chunk = 4 * G8_BK;
    splits = (int)((K + chunk - 1) / chunk);
    int rc;
    if ((rc = ensure(h, &h->d_gpart, &h->gpart_bytes, std::max(h->gpart_bytes, (size_t)splits * m * n * sizeof(double)))))
        return rc;
    double* part = (double*)h->d_gpart;
    dim3 grid((unsigned)(tm * tn), splits);
    { ProfScope ps(h, HUB_K_GRAM);
    k_gram_f32x8<<<grid, 64, 0, h->stream>>>(A, lda, B, ldb, K, m, n, chunk, tn, sym ? 1 : 0, part); }
    HUB_CUDA_TRY(h, cudaGetLastError());
    const long tot = (long)m * n;
    { ProfScope ps(h, HUB_K_GRAM_REDUCE);
    k_gram_reduce<double><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(part, splits, m, n, alpha,
                                                                                sym ? 1 : 0, G8_TB, G); }
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

// 32 x 32 tiles: on the 348-orbital rutile block the 64-wide tiles computed 42 % more
// elements than the symmetric product needs (ragged edge, full diagonal tiles), the 32-wide
// ones 11 %; the FP64 Gram product went from 112 to 81 ms
template <typename T>
int gram_t(hub_t h, const void* A, int lda, const void* B, int ldb, int m, int n, double alpha,
           bool sym, double* G) {
    return gram_tiles<T, 32>(h, A, lda, B, ldb, m, n, alpha, sym, G);
}

}  // namespace

int launch_gram(hub_t h, const void* A, int lda, const void* B, int ldb, int m, int n,
                double alpha, bool sym, double* G) {
    if (m == 0 || n == 0) return HUB_OK;
    if (h->cplx) {
        if (h->esize == 8) return gram_t<double2>(h, A, lda, B, ldb, m, n, alpha, sym, G);
        return gram_t<float2>(h, A, lda, B, ldb, m, n, alpha, sym, G);
    }
    if (h->esize == 8) return gram_t<double>(h, A, lda, B, ldb, m, n, alpha, sym, G);
    if (lda % 4 == 0 && ldb % 4 == 0 && (uintptr_t)A % 16 == 0 && (uintptr_t)B % 16 == 0)
        return gram_f32x8(h, (const float*)A, lda, (const float*)B, ldb, m, n, alpha, sym, G);
    return gram_t<float>(h, A, lda, B, ldb, m, n, alpha, sym, G);
}

int launch_rotate(hub_t h, const void* X, int ldx, const double* Q, int k, int n, void* Y, int ldy) {
    if (n == 0) return HUB_OK;
    dim3 grid((unsigned)((h->Nd + BM - 1) / BM), (n + BN - 1) / BN);
    ProfScope ps(h, HUB_K_ROTATE);
    const double2* Qz = (const double2*)Q;
    if (h->cplx && h->esize == 8)
        k_rotate<double2><<<grid, 256, 0, h->stream>>>((const double2*)X, ldx, Qz, k, n, h->Nd, (double2*)Y, ldy);
    else if (h->cplx)
        k_rotate<float2><<<grid, 256, 0, h->stream>>>((const float2*)X, ldx, Qz, k, n, h->Nd, (float2*)Y, ldy);
    else if (h->esize == 8)
        k_rotate<double><<<grid, 256, 0, h->stream>>>((const double*)X, ldx, Q, k, n, h->Nd, (double*)Y, ldy);
    else if (ldx % 4 == 0 && ldy % 4 == 0 && (uintptr_t)X % 16 == 0 && (uintptr_t)Y % 16 == 0)
        k_rotate_f32x8<<<dim3((unsigned)((h->Nd + R8_BM - 1) / R8_BM), (n + R8_BN - 1) / R8_BN), 128, 0, h->stream>>>(
            (const float*)X, ldx, Q, k, n, h->Nd, (float*)Y, ldy);
    else
        k_rotate<float><<<grid, 256, 0, h->stream>>>((const float*)X, ldx, Q, k, n, h->Nd, (float*)Y, ldy);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

}  // namespace hub

// ---------------------------------------------------------------------------- no-alloc
// hub_gram_noalloc: the split-K Gram product without any allocation.  Its split-K partial
// tiles live in one file-scope device array that every GPU loading this library holds for
// the life of the process.  The host code obtains the array's device address once per
// device with cudaGetSymbolAddress (the array's name in host code is only a stand-in, not a
// device address) and passes that address to the same kernels hub_gram uses.
namespace hub {
namespace {

constexpr size_t kNoAllocDoubles = (size_t)4 << 20;     // 4 Mi doubles = 32 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocDoubles];

std::mutex g_noalloc_mutex;
double* g_noalloc_addr[kNoAllocMaxDevices] = {};

int noalloc_scratch(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return HUB_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return HUB_ECUDA;
        g_noalloc_addr[dev] = (double*)p;
    }
    *out = g_noalloc_addr[dev];
    return HUB_OK;
}

template <typename T>
int gram_noalloc_t(const void* A, int lda, const void* B, int ldb, long K, int m, int n,
                   double alpha, bool sym, double* G, cudaStream_t stream) {
    const size_t mn = (size_t)m * n;
    if (mn > kNoAllocDoubles) return HUB_EINVAL;
    double* part = nullptr;
    int rc = noalloc_scratch(&part);
    if (rc) return rc;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HUB_ECUDA;
    const int tm = (m + BM - 1) / BM, tn = (n + BN - 1) / BN;
    const long ntiles = sym ? (long)tm * (tm + 1) / 2 : (long)tm * tn;
    long splits = (4L * sms + ntiles - 1) / ntiles;
    splits = std::min<long>(splits, (long)(kNoAllocDoubles / mn));   // partials must fit
    splits = std::max<long>(splits, 1);
    long chunk = (K + splits - 1) / splits;
    chunk = ((chunk + BK - 1) / BK) * BK;
    if (chunk < 4 * BK) chunk = 4 * BK;
    splits = (K + chunk - 1) / chunk;
    if ((size_t)splits * mn > kNoAllocDoubles) return HUB_EINVAL;
    dim3 grid((unsigned)(tm * tn), (unsigned)splits);
    k_gram_partial<T, BM><<<grid, 256, 0, stream>>>((const T*)A, lda, (const T*)B, ldb, K, m, n, chunk, tn,
                                                    sym ? 1 : 0, part);
    if (cudaGetLastError() != cudaSuccess) return HUB_ECUDA;
    const long tot = (long)m * n;
    k_gram_reduce<double><<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(part, (int)splits, m, n, alpha,
                                                                             sym ? 1 : 0, BM, G);
    if (cudaGetLastError() != cudaSuccess) return HUB_ECUDA;
    return HUB_OK;
}

}  // namespace

}  // namespace hub

extern "C" int hub_gram_noalloc(const void* A, int ncol_a, const void* B, int ncol_b, long long nrows,
                                int ld, int prec, double alpha, double* G_dev, void* cuda_stream) {
    if (ncol_a < 0 || ncol_b < 0 || nrows < 0 || (long long)ld < nrows) return HUB_EINVAL;
    if (prec != HUB_F64 && prec != HUB_F32) return HUB_EINVAL;
    if (ncol_a == 0 || ncol_b == 0 || nrows == 0) return HUB_OK;
    if (!A || !B || !G_dev) return HUB_EINVAL;
    const bool sym = (A == B) && (ncol_a == ncol_b);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (prec == HUB_F64)
        return hub::gram_noalloc_t<double>(A, ld, B, ld, (long)nrows, ncol_a, ncol_b, alpha, sym, G_dev, st);
    return hub::gram_noalloc_t<float>(A, ld, B, ld, (long)nrows, ncol_a, ncol_b, alpha, sym, G_dev, st);
}
