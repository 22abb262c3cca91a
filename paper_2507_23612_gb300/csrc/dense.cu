// Dense FP64 steps of the Rayleigh-Ritz projection (CheFSI, Sec. II.B) on n x n matrices
// (n = number of orbitals, up to ~1100), all row-major in device memory, real (double) at
// the Gamma point and complex Hermitian (double2, interleaved re/im) for Bloch orbitals:
//   Cholesky S = L L^H (blocked, right-looking), L^-1, small GEMMs with optional adjoint
//   operands, and a Hermitian eigensolver by parallel cyclic Jacobi (round-robin pairing:
//   n/2 disjoint rotations per step) in one cooperative kernel.  Every device-wide wait in
//   this file is a bounded software barrier: after its iteration limit it raises
//   FLAG_TIMEOUT and the kernel returns, so a wait can never hang the GPU.
#include <algorithm>

#include "hub_internal.cuh"
#include "cplx.cuh"

namespace hub {

namespace {

constexpr int NB = 32;   // Cholesky block

// factor the jb x jb diagonal block at (j0, j0) in place (one CTA, NB x NB in shared memory);
// the diagonal of a Hermitian matrix is real, so is L's
template <typename T>
__global__ void k_potf2(T* A, int lda, int j0, int jb, int* flags) {
    __shared__ T s[NB][NB + 1];
    const int t = threadIdx.x;
    for (int e = t; e < jb * jb; e += blockDim.x) {
        const int i = e / jb, j = e % jb;
        s[i][j] = A[(size_t)(j0 + i) * lda + j0 + j];
    }
    __syncthreads();
    for (int k = 0; k < jb; ++k) {
        if (t == 0) {
            const double d = re_of(s[k][k]);
            if (!(d > 0.0) || !isfinite(d)) {
                flags[FLAG_NOTSPD] = 1;
                s[k][k] = from_real<T>(1.0);
            } else {
                s[k][k] = from_real<T>(sqrt(d));
            }
        }
        __syncthreads();
        const double dkk = re_of(s[k][k]);
        for (int i = k + 1 + t; i < jb; i += blockDim.x) s[i][k] = divr(s[i][k], dkk);
        __syncthreads();
        for (int e = t; e < jb * jb; e += blockDim.x) {
            const int i = e / jb, j = e % jb;
            if (i > k && j > k && j <= i) s[i][j] = csub(s[i][j], cmul(s[i][k], cconj(s[j][k])));
        }
        __syncthreads();
    }
    for (int e = t; e < jb * jb; e += blockDim.x) {
        const int i = e / jb, j = e % jb;
        A[(size_t)(j0 + i) * lda + j0 + j] = (j <= i) ? s[i][j] : zero_of(T());
    }
}

// rows below the diagonal block: L21 = A21 L11^-H (each thread solves one row)
template <typename T>
__global__ void k_trsm_rows(T* A, int lda, int j0, int jb, int n) {
    __shared__ T L[NB][NB + 1];
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
        const int i = e / jb, j = e % jb;
        L[i][j] = A[(size_t)(j0 + i) * lda + j0 + j];
    }
    __syncthreads();
    const int r = j0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    T x[NB];
    T* row = A + (size_t)r * lda + j0;
    for (int c = 0; c < jb; ++c) {
        T v = row[c];
        for (int cc = 0; cc < c; ++cc) v = csub(v, cmul(x[cc], cconj(L[c][cc])));
        x[c] = divr(v, re_of(L[c][c]));
    }
    for (int c = 0; c < jb; ++c) row[c] = x[c];
}

// C = alpha op(A) op(B) + beta C, row-major, 32 x 32 tiles; op = identity or the adjoint
// (conjugate transpose; the transpose for real matrices); alpha, beta real
template <typename T>
__global__ void k_dgemm(int ta, int tb, int m, int n, int k, double alpha, const T* __restrict__ A,
                        int lda, const T* __restrict__ B, int ldb, double beta, T* C, int ldc) {
    __shared__ T As[32][33], Bs[32][33];
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8 threads
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    T acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = zero_of(T());
    for (int k0 = 0; k0 < k; k0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int i = i0 + r, kk = k0 + tx;
            T a = zero_of(T());
            if (i < m && kk < k) a = ta ? cconj(A[(size_t)kk * lda + i]) : A[(size_t)i * lda + kk];
            As[r][tx] = a;
            const int kb = k0 + r, j = j0 + tx;
            T b = zero_of(T());
            if (kb < k && j < n) b = tb ? cconj(B[(size_t)j * ldb + kb]) : B[(size_t)kb * ldb + j];
            Bs[r][tx] = b;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const T b = Bs[kk][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = cfma(As[ty + 8 * q][kk], b, acc[q]);
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty + 8 * q, j = j0 + tx;
        if (i < m && j < n) {
            T* c = C + (size_t)i * ldc + j;
            *c = beta != 0.0 ? add(mulr(alpha, acc[q]), mulr(beta, *c)) : mulr(alpha, acc[q]);
        }
    }
}

// Linv = L^-1: one warp per column j solves L x = e_j by forward substitution
template <typename T>
__global__ void k_tri_inverse(const T* __restrict__ L, T* __restrict__ Linv, int n) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int j = warp;
    T* x = Linv;   // column j of Linv: x[i*n + j]
    for (int i = lane; i < j; i += 32) x[(size_t)i * n + j] = zero_of(T());
    for (int i = j; i < n; ++i) {
        T s = zero_of(T());
        for (int l = j + lane; l < i; l += 32) s = cfma(L[(size_t)i * n + l], x[(size_t)l * n + j], s);
        for (int o = 16; o > 0; o >>= 1) s = add(s, shfl_down(s, o));
        if (lane == 0)
            x[(size_t)i * n + j] = divr(csub(from_real<T>(i == j ? 1.0 : 0.0), s), re_of(L[(size_t)i * n + i]));
        __syncwarp();
    }
}

// A <- (A + A^H) / 2 (the diagonal of a Hermitian matrix is real)
template <typename T>
__global__ void k_symmetrize(T* A, int n) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    if (j < i) return;
    if (j == i) { A[(size_t)i * n + i] = from_real<T>(re_of(A[(size_t)i * n + i])); return; }
    const T v = mulr(0.5, add(A[(size_t)i * n + j], cconj(A[(size_t)j * n + i])));
    A[(size_t)i * n + j] = v;
    A[(size_t)j * n + i] = cconj(v);
}

// ---------------------------------------------------------------------------- Jacobi
constexpr long kSpinLimit = 1L << 22;

// bounded grid barrier for a cooperative launch; returns false once any wait ran out
__device__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, int* flags) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = bar + 1;
        const unsigned int gen = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(bar, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long it = 0;
            while (*vgen == gen) {
                if (++it > kSpinLimit) { atomicExch(flags + FLAG_TIMEOUT, 1); break; }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *((volatile int*)(flags + FLAG_TIMEOUT)) == 0;
}

__device__ __forceinline__ void pair_of(int step, int k, int N, int& p, int& q) {
    // round-robin ("circle") schedule: player N-1 fixed, players 0..N-2 rotate
    if (k == 0) { p = N - 1; q = step; }
    else {
        p = (step + k) % (N - 1);
        q = (step - k + (N - 1)) % (N - 1);
    }
    if (p > q) { const int t = p; p = q; q = t; }
}

// Parallel cyclic Jacobi with the round-robin pair schedule.  Each step applies n/2
// disjoint rotations.  Every CTA computes all rotation angles of a step itself from the
// current matrix (identical inputs and operations, so all copies agree), and the step
// writes the rotated matrix into the other of two buffers: nothing the step reads is
// written during it, so one grid barrier per step suffices.  V is rotated in place (only
// the step's own rotations touch a given V element).
// The rotation of a pair (p, q) is J = [[c, sg], [-conj(sg), c]] with c real and
// sg = s exp(i arg a_pq): the phase makes the pivot real, then the real Jacobi angle of
// (a_pp, |a_pq|, a_qq) zeroes it; for real matrices sg = +-s and J is the plain rotation.
// With nmat = 2 the grid solves two independent matrices of the same size at once: each
// half of the CTAs owns one matrix, its buffers, its barrier counters and its reduction
// slots, and only the error flags are shared (a timeout in one half ends both).
template <typename T>
__global__ void k_jacobi(T* A0, T* Ab0, T* V0, T* A1, T* Ab1, T* V1, int nmat,
                         int n, int N, int max_sweeps, double tol, unsigned int* bar, int* flags,
                         unsigned long long* red0, unsigned long long* red1, int* sweeps_out) {
    constexpr bool CPLX = sizeof(T) == 2 * sizeof(double);
    constexpr int RS = CPLX ? 3 : 2;              // doubles per pair: c, sg (re[, im])
    extern __shared__ double rot[];               // [RS * N / 2]
    auto sg_of = [&](int k) -> T {
        if constexpr (CPLX) return make_double2(rot[RS * k + 1], rot[RS * k + 2]);
        else return rot[RS * k + 1];
    };
    const int grp = (nmat == 2 && blockIdx.x >= gridDim.x / 2) ? 1 : 0;
    const unsigned int nb = nmat == 2 ? gridDim.x / 2 : gridDim.x;
    T* A = grp ? A1 : A0;
    T* Ab = grp ? Ab1 : Ab0;
    T* V = grp ? V1 : V0;
    unsigned long long* red = grp ? red1 : red0;
    bar += 2 * grp;
    sweeps_out += grp;
    const long tid = (long)(blockIdx.x - grp * nb) * blockDim.x + threadIdx.x;
    const long nthr = (long)nb * blockDim.x;
    const int H = N / 2;
    T* cur = A;
    T* nxt = Ab;
    const T zero = zero_of(T());
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // convergence: max |a_ij| (i != j) against max |a_ii|
        unsigned long long* acc = red + 2 * (sweep & 1);
        double off = 0.0, dia = 0.0;
        for (long e = tid; e < (long)n * n; e += nthr) {
            const int i = (int)(e / n), j = (int)(e % n);
            const double v = cabs_of(cur[e]);
            if (i == j) dia = fmax(dia, v); else off = fmax(off, v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            off = fmax(off, __shfl_down_sync(0xffffffffu, off, o));
            dia = fmax(dia, __shfl_down_sync(0xffffffffu, dia, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMax(acc, (unsigned long long)__double_as_longlong(off));
            atomicMax(acc + 1, (unsigned long long)__double_as_longlong(dia));
        }
        if (!grid_barrier(bar, nb, flags)) return;
        const double goff = __longlong_as_double((long long)*((volatile unsigned long long*)acc));
        const double gdia = __longlong_as_double((long long)*((volatile unsigned long long*)(acc + 1)));
        if (tid == 0) {                          // the group's first thread
            unsigned long long* other = red + 2 * ((sweep + 1) & 1);
            other[0] = 0ull;
            other[1] = 0ull;
        }
        if (goff <= tol * fmax(gdia, 1e-300)) break;
        if (sweep == max_sweeps - 1) {
            if (tid == 0) flags[FLAG_NOCONV] = 1;
            break;
        }
        // pairs whose coupling is below this are left alone (threshold Jacobi)
        const double skip = 1e-3 * tol * fmax(gdia, 1e-300);
        for (int step = 0; step < N - 1; ++step) {
            // phase 1 (per CTA): the n/2 disjoint rotations of this step
            for (int k = threadIdx.x; k < H; k += blockDim.x) {
                int p, q;
                pair_of(step, k, N, p, q);
                double c = 1.0, sr = 0.0, si = 0.0;
                if (q < n) {
                    const T apq = cur[(size_t)p * n + q];
                    const double mag = cabs_of(apq);
                    if (mag > skip) {
                        const double app = re_of(cur[(size_t)p * n + p]), aqq = re_of(cur[(size_t)q * n + q]);
                        const double theta = (aqq - app) / (2.0 * mag);
                        double t;
                        if (fabs(theta) > 1e150) t = 0.5 / theta;
                        else t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        const double s = t * c;
                        if constexpr (CPLX) { sr = s * (apq.x / mag); si = s * (apq.y / mag); }
                        else sr = apq >= 0.0 ? s : -s;
                    }
                }
                rot[RS * k] = c;
                rot[RS * k + 1] = sr;
                if constexpr (CPLX) rot[RS * k + 2] = si;
            }
            __syncthreads();
            // phase 2: every 2x2 block (P, Q) of the next matrix <- J_P^H B J_Q (blocks of two
            // identity rotations are copied), and V <- V J in place
            // the matrix stays Hermitian: only the blocks P <= Q are computed, and each
            // writes its adjoint too
            const long nblk = (long)H * (H + 1) / 2;
            for (long e = tid; e < nblk + (long)n * H; e += nthr) {
                if (e < nblk) {
                    // row P of the upper triangle holds H - P blocks; S(P) = P (2H - P + 1) / 2
                    // (estimate in float arithmetic: the FP64 pipe is the scarce one; the two
                    // loops below correct the estimate)
                    const float h2 = 2.0f * H + 1.0f;
                    int P = (int)((h2 - sqrtf(fmaxf(h2 * h2 - 8.0f * (float)e, 0.0f))) * 0.5f);
                    P = max(0, min(P, H - 1));
                    auto S = [&](long r) { return r * (2L * H - r + 1) / 2; };
                    while (P > 0 && S(P) > e) --P;
                    while (P < H - 1 && S(P + 1) <= e) ++P;
                    const int Q = P + (int)(e - S(P));
                    const T g1 = sg_of(P), g2 = sg_of(Q);
                    const double c1 = rot[RS * P], c2 = rot[RS * Q];
                    const bool r1 = cabs_of(g1) != 0.0, r2 = cabs_of(g2) != 0.0;
                    int p1, q1, p2, q2;
                    pair_of(step, P, N, p1, q1);
                    pair_of(step, Q, N, p2, q2);
                    auto ld = [&](int i, int j) { return (i < n && j < n) ? cur[(size_t)i * n + j] : zero; };
                    const T b00 = ld(p1, p2), b01 = ld(p1, q2), b10 = ld(q1, p2), b11 = ld(q1, q2);
                    T n00 = b00, n01 = b01, n10 = b10, n11 = b11;
                    if (r1 || r2) {
                        const T r00 = csub(mulr(c1, b00), cmul(g1, b10));
                        const T r01 = csub(mulr(c1, b01), cmul(g1, b11));
                        const T r10 = cfma(cconj(g1), b00, mulr(c1, b10));
                        const T r11 = cfma(cconj(g1), b01, mulr(c1, b11));
                        n00 = csub(mulr(c2, r00), cmul(cconj(g2), r01));
                        n01 = cfma(g2, r00, mulr(c2, r01));
                        n10 = csub(mulr(c2, r10), cmul(cconj(g2), r11));
                        n11 = cfma(g2, r10, mulr(c2, r11));
                        if (P == Q && q1 < n) {
                            // the rotated pair: exact zero off-diagonal, diagonal by the t-update
                            // (t |a_pq| = Re(conj(sg) a_pq) / c)
                            const double ta = re_of(cmul(cconj(g1), b01)) / c1;
                            n00 = from_real<T>(re_of(b00) - ta);
                            n11 = from_real<T>(re_of(b11) + ta);
                            n01 = zero;
                            n10 = zero;
                        }
                    }
                    if (p1 < n && p2 < n) { nxt[(size_t)p1 * n + p2] = n00; nxt[(size_t)p2 * n + p1] = cconj(n00); }
                    if (p1 < n && q2 < n) { nxt[(size_t)p1 * n + q2] = n01; nxt[(size_t)q2 * n + p1] = cconj(n01); }
                    if (q1 < n && p2 < n) { nxt[(size_t)q1 * n + p2] = n10; nxt[(size_t)p2 * n + q1] = cconj(n10); }
                    if (q1 < n && q2 < n) { nxt[(size_t)q1 * n + q2] = n11; nxt[(size_t)q2 * n + q1] = cconj(n11); }
                } else {
                    const long f = e - nblk;
                    const int r = (int)(f / H), P = (int)(f % H);
                    const T g = sg_of(P);
                    if (cabs_of(g) == 0.0) continue;
                    int p, q;
                    pair_of(step, P, N, p, q);
                    if (q >= n) continue;
                    const double c = rot[RS * P];
                    const T vp = V[(size_t)r * n + p], vq = V[(size_t)r * n + q];
                    V[(size_t)r * n + p] = csub(mulr(c, vp), cmul(cconj(g), vq));
                    V[(size_t)r * n + q] = cfma(g, vp, mulr(c, vq));
                }
            }
            if (!grid_barrier(bar, nb, flags)) return;
            T* t = cur; cur = nxt; nxt = t;
        }
    }
    if (cur != A)
        for (long e = tid; e < (long)n * n; e += nthr) A[e] = cur[e];
    if (tid == 0) *sweeps_out = sweep;
}

template <typename T>
__global__ void k_eye(T* V, int n) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    V[t] = from_real<T>(((t / n) == (t % n)) ? 1.0 : 0.0);
}

// ascending order: rank by (value, index); V columns follow
template <typename T>
__global__ void k_sort_eig(const T* __restrict__ A, const T* __restrict__ V, int n,
                           double* __restrict__ eig, T* __restrict__ Vs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ai = re_of(A[(size_t)i * n + i]);
    int rank = 0;
    for (int j = 0; j < n; ++j) {
        const double aj = re_of(A[(size_t)j * n + j]);
        rank += (aj < ai) || (aj == ai && j < i);
    }
    eig[rank] = ai;
    for (int r = 0; r < n; ++r) Vs[(size_t)r * n + rank] = V[(size_t)r * n + i];
}

}  // namespace

// The host entry points take double pointers; on a complex handle every matrix is n x n
// double2 (interleaved re/im, 2 n^2 doubles) and the same memory is read as such.
namespace {

template <typename T>
int gemm_t(hub_t h, bool ta, bool tb, int m, int n, int k, double alpha, const T* A, int lda, const T* B,
           int ldb, double beta, T* C, int ldc) {
    if (m == 0 || n == 0) return HUB_OK;
    dim3 grid((n + 31) / 32, (m + 31) / 32);
    ProfScope ps(h, HUB_K_DGEMM);
    k_dgemm<T><<<grid, 256, 0, h->stream>>>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

template <typename T>
int cholesky_t(hub_t h, T* A, int n) {
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = std::min(NB, n - j0);
        { ProfScope ps(h, HUB_K_CHOLESKY); k_potf2<T><<<1, 256, 0, h->stream>>>(A, n, j0, jb, h->d_flags); }
        HUB_CUDA_TRY(h, cudaGetLastError());
        const int rest = n - j0 - jb;
        if (rest <= 0) continue;
        { ProfScope ps(h, HUB_K_CHOLESKY); k_trsm_rows<T><<<(rest + 127) / 128, 128, 0, h->stream>>>(A, n, j0, jb, n); }
        HUB_CUDA_TRY(h, cudaGetLastError());
        T* A21 = A + (size_t)(j0 + jb) * n + j0;
        T* A22 = A + (size_t)(j0 + jb) * n + (j0 + jb);
        int rc = gemm_t<T>(h, false, true, rest, rest, jb, -1.0, A21, n, A21, n, 1.0, A22, n);
        if (rc) return rc;
    }
    return HUB_OK;
}

template <typename T>
int jacobi_t(hub_t h, int nmat, T* const* A, T* const* V, double* const* eig, int n) {
    const int N = n + (n & 1);
    const size_t nn = (size_t)n * n;
    constexpr int CW = sizeof(T) / sizeof(double);
    const size_t per = 2 * CW * nn + 8;                         // doubles of workspace per matrix
    int rc;
    if ((rc = ensure(h, &h->d_work2, &h->work2_bytes, std::max(nmat * per * sizeof(double), h->work2_bytes))))
        return rc;
    T* Vt[2];
    T* Ab[2];
    unsigned long long* red[2];
    for (int g = 0; g < 2; ++g) {
        const int m = g < nmat ? g : 0;
        double* base = (double*)h->d_work2 + m * per;
        Vt[g] = (T*)base;
        Ab[g] = Vt[g] + nn;                                     // second matrix buffer
        red[g] = (unsigned long long*)(base + 2 * CW * nn);     // 4 slots
    }
    int* sweeps = h->d_flags + 6;                               // slots 6 and 7
    for (int g = 0; g < nmat; ++g) {
        {
            ProfScope ps(h, HUB_K_EIG_MISC);
            k_eye<T><<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(Vt[g], n);
        }
        HUB_CUDA_TRY(h, cudaGetLastError());
        HUB_CUDA_TRY(h, cudaMemsetAsync(red[g], 0, 4 * sizeof(unsigned long long), h->stream));
    }
    HUB_CUDA_TRY(h, cudaMemsetAsync(h->d_bar, 0, 4 * sizeof(unsigned int), h->stream));
    HUB_CUDA_TRY(h, cudaMemsetAsync(sweeps, 0, 2 * sizeof(int), h->stream));
    int per_sm = 0;
    const size_t rot_bytes = (size_t)(N / 2) * (CW + 1) * sizeof(double);
    if (rot_bytes > 48 * 1024) return fail(h, HUB_EINVAL, "subspace too large for the Jacobi solver");
    HUB_CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi<T>, 256, rot_bytes));
    int blocks = std::max(1, std::min(per_sm, 1)) * h->num_sms / nmat;   // per matrix
    const long work = (long)(N / 2) * (N / 2 + 1) / 2 + (long)n * (N / 2);
    blocks = (int)std::min<long>(blocks, std::max<long>(1, (work + 255) / 256));
    blocks = std::max(1, blocks) * nmat;
    int max_sweeps = 60;
    double tol = 1e-13;
    unsigned int* bar = h->d_bar;
    int* flags = h->d_flags;
    T* A0 = A[0];
    T* A1 = nmat > 1 ? A[1] : A[0];
    void* args[] = {&A0, &Ab[0], &Vt[0], &A1, &Ab[1], &Vt[1], &nmat, &n, (void*)&N, &max_sweeps, &tol, &bar,
                    &flags, &red[0], &red[1], &sweeps};
    {
        ProfScope ps(h, HUB_K_JACOBI);
        HUB_CUDA_TRY(h, cudaLaunchCooperativeKernel((void*)k_jacobi<T>, dim3(blocks), dim3(256), args, rot_bytes,
                                                    h->stream));
    }
    for (int g = 0; g < nmat; ++g) {
        ProfScope ps(h, HUB_K_EIG_MISC);
        k_sort_eig<T><<<(n + 127) / 128, 128, 0, h->stream>>>(A[g], Vt[g], n, eig[g], V[g]);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

}  // namespace

int dense_gemm(hub_t h, bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
               int lda, const double* B, int ldb, double beta, double* C, int ldc) {
    if (h->cplx)
        return gemm_t<double2>(h, ta, tb, m, n, k, alpha, (const double2*)A, lda, (const double2*)B, ldb, beta,
                               (double2*)C, ldc);
    return gemm_t<double>(h, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

int dense_cholesky(hub_t h, double* A, int n) {
    return h->cplx ? cholesky_t<double2>(h, (double2*)A, n) : cholesky_t<double>(h, A, n);
}

int dense_tri_inverse(hub_t h, const double* L, double* Linv, int n) {
    const int threads = 256;
    const long warps = n;
    const unsigned blocks = (unsigned)((warps * 32 + threads - 1) / threads);
    ProfScope ps(h, HUB_K_TRI_INVERSE);
    if (h->cplx) k_tri_inverse<double2><<<blocks, threads, 0, h->stream>>>((const double2*)L, (double2*)Linv, n);
    else k_tri_inverse<double><<<blocks, threads, 0, h->stream>>>(L, Linv, n);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int dense_symmetrize(hub_t h, double* A, int n) {
    const long tot = (long)n * n;
    ProfScope ps(h, HUB_K_EIG_MISC);
    if (h->cplx) k_symmetrize<double2><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>((double2*)A, n);
    else k_symmetrize<double><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(A, n);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

// A (n x n Hermitian, destroyed) -> eig ascending (device [n]) and V (device n x n row-major,
// column j = eigenvector j).  Uses 2 n x n matrices + 8 doubles of scratch per matrix.
int dense_jacobi_eigh_multi(hub_t h, int nmat, double* const* A, double* const* V, double* const* eig, int n) {
    if (n == 0) return HUB_OK;
    if (nmat < 1 || nmat > 2) return fail(h, HUB_EINVAL, "one or two matrices per Jacobi launch");
    if (h->cplx) {
        double2* Az[2] = {(double2*)A[0], (double2*)A[nmat - 1]};
        double2* Vz[2] = {(double2*)V[0], (double2*)V[nmat - 1]};
        return jacobi_t<double2>(h, nmat, Az, Vz, eig, n);
    }
    return jacobi_t<double>(h, nmat, A, V, eig, n);
}

int dense_jacobi_eigh(hub_t h, double* A, double* V, double* eig, int n) {
    return dense_jacobi_eigh_multi(h, 1, &A, &V, &eig, n);
}

}  // namespace hub
