// Dense FP64 steps of the Rayleigh-Ritz projection (CheFSI, Sec. II.B) on n x n matrices
// (n = number of orbitals, up to ~1100), all row-major in device memory:
//   Cholesky S = L L^T (blocked, right-looking), L^-1, small GEMMs, and a symmetric
//   eigensolver by parallel cyclic Jacobi (round-robin pairing: n/2 disjoint rotations per
//   step) in one cooperative kernel.  Every device-wide wait in this file is a bounded
//   software barrier: after its iteration limit it raises FLAG_TIMEOUT and the kernel
//   returns, so a wait can never hang the GPU.
#include <algorithm>

#include "hub_internal.cuh"

namespace hub {

namespace {

constexpr int NB = 32;   // Cholesky block

// factor the jb x jb diagonal block at (j0, j0) in place (one CTA, NB x NB in shared memory)
__global__ void k_potf2(double* A, int lda, int j0, int jb, int* flags) {
    __shared__ double s[NB][NB + 1];
    const int t = threadIdx.x;
    for (int e = t; e < jb * jb; e += blockDim.x) {
        const int i = e / jb, j = e % jb;
        s[i][j] = A[(size_t)(j0 + i) * lda + j0 + j];
    }
    __syncthreads();
    for (int k = 0; k < jb; ++k) {
        if (t == 0) {
            const double d = s[k][k];
            if (!(d > 0.0) || !isfinite(d)) {
                flags[FLAG_NOTSPD] = 1;
                s[k][k] = 1.0;
            } else {
                s[k][k] = sqrt(d);
            }
        }
        __syncthreads();
        const double dkk = s[k][k];
        for (int i = k + 1 + t; i < jb; i += blockDim.x) s[i][k] /= dkk;
        __syncthreads();
        for (int e = t; e < jb * jb; e += blockDim.x) {
            const int i = e / jb, j = e % jb;
            if (i > k && j > k && j <= i) s[i][j] -= s[i][k] * s[j][k];
        }
        __syncthreads();
    }
    for (int e = t; e < jb * jb; e += blockDim.x) {
        const int i = e / jb, j = e % jb;
        A[(size_t)(j0 + i) * lda + j0 + j] = (j <= i) ? s[i][j] : 0.0;
    }
}

// rows below the diagonal block: L21 = A21 L11^-T (each thread solves one row)
__global__ void k_trsm_rows(double* A, int lda, int j0, int jb, int n) {
    __shared__ double L[NB][NB + 1];
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
        const int i = e / jb, j = e % jb;
        L[i][j] = A[(size_t)(j0 + i) * lda + j0 + j];
    }
    __syncthreads();
    const int r = j0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double x[NB];
    double* row = A + (size_t)r * lda + j0;
    for (int c = 0; c < jb; ++c) {
        double v = row[c];
        for (int cc = 0; cc < c; ++cc) v -= x[cc] * L[c][cc];
        x[c] = v / L[c][c];
    }
    for (int c = 0; c < jb; ++c) row[c] = x[c];
}

// C = alpha op(A) op(B) + beta C, row-major, 32 x 32 tiles
__global__ void k_dgemm(int ta, int tb, int m, int n, int k, double alpha, const double* __restrict__ A,
                        int lda, const double* __restrict__ B, int ldb, double beta, double* C, int ldc) {
    __shared__ double As[32][33], Bs[32][33];
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8 threads
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    double acc[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < k; k0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int i = i0 + r, kk = k0 + tx;
            double a = 0.0;
            if (i < m && kk < k) a = ta ? A[(size_t)kk * lda + i] : A[(size_t)i * lda + kk];
            As[r][tx] = a;
            const int kb = k0 + r, j = j0 + tx;
            double b = 0.0;
            if (kb < k && j < n) b = tb ? B[(size_t)j * ldb + kb] : B[(size_t)kb * ldb + j];
            Bs[r][tx] = b;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const double b = Bs[kk][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(As[ty + 8 * q][kk], b, acc[q]);
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty + 8 * q, j = j0 + tx;
        if (i < m && j < n) {
            double* c = C + (size_t)i * ldc + j;
            *c = alpha * acc[q] + (beta != 0.0 ? beta * *c : 0.0);
        }
    }
}

// Linv = L^-1: one warp per column j solves L x = e_j by forward substitution
__global__ void k_tri_inverse(const double* __restrict__ L, double* __restrict__ Linv, int n) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int j = warp;
    double* x = Linv;   // column j of Linv: x[i*n + j]
    for (int i = lane; i < j; i += 32) x[(size_t)i * n + j] = 0.0;
    for (int i = j; i < n; ++i) {
        double s = 0.0;
        for (int l = j + lane; l < i; l += 32) s += L[(size_t)i * n + l] * x[(size_t)l * n + j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) x[(size_t)i * n + j] = ((i == j ? 1.0 : 0.0) - s) / L[(size_t)i * n + i];
        __syncwarp();
    }
}

__global__ void k_symmetrize(double* A, int n) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    if (j <= i) return;
    const double v = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
    A[(size_t)i * n + j] = v;
    A[(size_t)j * n + i] = v;
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
// With nmat = 2 the grid solves two independent matrices of the same size at once: each
// half of the CTAs owns one matrix, its buffers, its barrier counters and its reduction
// slots, and only the error flags are shared (a timeout in one half ends both).
__global__ void k_jacobi(double* A0, double* Ab0, double* V0, double* A1, double* Ab1, double* V1, int nmat,
                         int n, int N, int max_sweeps, double tol, unsigned int* bar, int* flags,
                         unsigned long long* red0, unsigned long long* red1, int* sweeps_out) {
    extern __shared__ double rot[];               // [N]: cosine and sine of each pair
    const int grp = (nmat == 2 && blockIdx.x >= gridDim.x / 2) ? 1 : 0;
    const unsigned int nb = nmat == 2 ? gridDim.x / 2 : gridDim.x;
    double* A = grp ? A1 : A0;
    double* Ab = grp ? Ab1 : Ab0;
    double* V = grp ? V1 : V0;
    unsigned long long* red = grp ? red1 : red0;
    bar += 2 * grp;
    sweeps_out += grp;
    const long tid = (long)(blockIdx.x - grp * nb) * blockDim.x + threadIdx.x;
    const long nthr = (long)nb * blockDim.x;
    const int H = N / 2;
    double* cur = A;
    double* nxt = Ab;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // convergence: max |a_ij| (i != j) against max |a_ii|
        unsigned long long* acc = red + 2 * (sweep & 1);
        double off = 0.0, dia = 0.0;
        for (long e = tid; e < (long)n * n; e += nthr) {
            const int i = (int)(e / n), j = (int)(e % n);
            const double v = fabs(cur[e]);
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
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = cur[(size_t)p * n + q];
                    if (fabs(apq) > skip) {
                        const double app = cur[(size_t)p * n + p], aqq = cur[(size_t)q * n + q];
                        const double theta = (aqq - app) / (2.0 * apq);
                        double t;
                        if (fabs(theta) > 1e150) t = 0.5 / theta;
                        else t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                }
                rot[2 * k] = c;
                rot[2 * k + 1] = s;
            }
            __syncthreads();
            // phase 2: every 2x2 block (P, Q) of the next matrix <- J_P^T B J_Q (blocks of two
            // identity rotations are copied), and V <- V J in place
            // the matrix stays symmetric: only the blocks P <= Q are computed, and each
            // writes its transpose too
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
                    const double s1 = rot[2 * P + 1], s2 = rot[2 * Q + 1];
                    const double c1 = rot[2 * P], c2 = rot[2 * Q];
                    int p1, q1, p2, q2;
                    pair_of(step, P, N, p1, q1);
                    pair_of(step, Q, N, p2, q2);
                    auto ld = [&](int i, int j) { return (i < n && j < n) ? cur[(size_t)i * n + j] : 0.0; };
                    const double b00 = ld(p1, p2), b01 = ld(p1, q2), b10 = ld(q1, p2), b11 = ld(q1, q2);
                    double n00 = b00, n01 = b01, n10 = b10, n11 = b11;
                    if (s1 != 0.0 || s2 != 0.0) {
                        const double r00 = c1 * b00 - s1 * b10, r01 = c1 * b01 - s1 * b11;
                        const double r10 = s1 * b00 + c1 * b10, r11 = s1 * b01 + c1 * b11;
                        n00 = c2 * r00 - s2 * r01; n01 = s2 * r00 + c2 * r01;
                        n10 = c2 * r10 - s2 * r11; n11 = s2 * r10 + c2 * r11;
                        if (P == Q && q1 < n) {
                            // the rotated pair: exact zero off-diagonal, diagonal by the t-update
                            const double t = s1 / c1;
                            n00 = b00 - t * b01;
                            n11 = b11 + t * b01;
                            n01 = 0.0;
                            n10 = 0.0;
                        }
                    }
                    if (p1 < n && p2 < n) { nxt[(size_t)p1 * n + p2] = n00; nxt[(size_t)p2 * n + p1] = n00; }
                    if (p1 < n && q2 < n) { nxt[(size_t)p1 * n + q2] = n01; nxt[(size_t)q2 * n + p1] = n01; }
                    if (q1 < n && p2 < n) { nxt[(size_t)q1 * n + p2] = n10; nxt[(size_t)p2 * n + q1] = n10; }
                    if (q1 < n && q2 < n) { nxt[(size_t)q1 * n + q2] = n11; nxt[(size_t)q2 * n + q1] = n11; }
                } else {
                    const long f = e - nblk;
                    const int r = (int)(f / H), P = (int)(f % H);
                    const double s = rot[2 * P + 1];
                    if (s == 0.0) continue;
                    int p, q;
                    pair_of(step, P, N, p, q);
                    if (q >= n) continue;
                    const double c = rot[2 * P];
                    const double vp = V[(size_t)r * n + p], vq = V[(size_t)r * n + q];
                    V[(size_t)r * n + p] = c * vp - s * vq;
                    V[(size_t)r * n + q] = s * vp + c * vq;
                }
            }
            if (!grid_barrier(bar, nb, flags)) return;
            double* t = cur; cur = nxt; nxt = t;
        }
    }
    if (cur != A)
        for (long e = tid; e < (long)n * n; e += nthr) A[e] = cur[e];
    if (tid == 0) *sweeps_out = sweep;
}

__global__ void k_eye(double* V, int n) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    V[t] = ((t / n) == (t % n)) ? 1.0 : 0.0;
}

// ascending order: rank by (value, index); V columns follow
__global__ void k_sort_eig(const double* __restrict__ A, const double* __restrict__ V, int n,
                           double* __restrict__ eig, double* __restrict__ Vs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ai = A[(size_t)i * n + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
        const double aj = A[(size_t)j * n + j];
        rank += (aj < ai) || (aj == ai && j < i);
    }
    eig[rank] = ai;
    for (int r = 0; r < n; ++r) Vs[(size_t)r * n + rank] = V[(size_t)r * n + i];
}

}  // namespace

int dense_gemm(hub_t h, bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
               int lda, const double* B, int ldb, double beta, double* C, int ldc) {
    if (m == 0 || n == 0) return HUB_OK;
    dim3 grid((n + 31) / 32, (m + 31) / 32);
    ProfScope ps(h, HUB_K_DGEMM);
    k_dgemm<<<grid, 256, 0, h->stream>>>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int dense_cholesky(hub_t h, double* A, int n) {
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = std::min(NB, n - j0);
        { ProfScope ps(h, HUB_K_CHOLESKY); k_potf2<<<1, 256, 0, h->stream>>>(A, n, j0, jb, h->d_flags); }
        HUB_CUDA_TRY(h, cudaGetLastError());
        const int rest = n - j0 - jb;
        if (rest <= 0) continue;
        { ProfScope ps(h, HUB_K_CHOLESKY); k_trsm_rows<<<(rest + 127) / 128, 128, 0, h->stream>>>(A, n, j0, jb, n); }
        HUB_CUDA_TRY(h, cudaGetLastError());
        double* A21 = A + (size_t)(j0 + jb) * n + j0;
        double* A22 = A + (size_t)(j0 + jb) * n + (j0 + jb);
        int rc = dense_gemm(h, false, true, rest, rest, jb, -1.0, A21, n, A21, n, 1.0, A22, n);
        if (rc) return rc;
    }
    return HUB_OK;
}

int dense_tri_inverse(hub_t h, const double* L, double* Linv, int n) {
    const int threads = 256;
    const long warps = n;
    ProfScope ps(h, HUB_K_TRI_INVERSE);
    k_tri_inverse<<<(unsigned)((warps * 32 + threads - 1) / threads), threads, 0, h->stream>>>(L, Linv, n);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int dense_symmetrize(hub_t h, double* A, int n) {
    const long tot = (long)n * n;
    ProfScope ps(h, HUB_K_EIG_MISC);
    k_symmetrize<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(A, n);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

// A (n x n symmetric, destroyed) -> eig ascending (device [n]) and V (device n x n row-major,
// column j = eigenvector j).  Uses 2 n x n + n scratch from the handle.
int dense_jacobi_eigh_multi(hub_t h, int nmat, double* const* A, double* const* V, double* const* eig, int n) {
    if (n == 0) return HUB_OK;
    if (nmat < 1 || nmat > 2) return fail(h, HUB_EINVAL, "one or two matrices per Jacobi launch");
    const int N = n + (n & 1);
    const size_t nn = (size_t)n * n;
    const size_t per = 2 * nn + 8;                               // doubles of workspace per matrix
    int rc;
    if ((rc = ensure(h, &h->d_work2, &h->work2_bytes, std::max(nmat * per * sizeof(double), h->work2_bytes))))
        return rc;
    double* Vt[2];
    double* Ab[2];
    unsigned long long* red[2];
    for (int g = 0; g < 2; ++g) {
        const int m = g < nmat ? g : 0;
        Vt[g] = (double*)h->d_work2 + m * per;
        Ab[g] = Vt[g] + nn;                                     // second matrix buffer
        red[g] = (unsigned long long*)(Ab[g] + nn);             // 4 slots
    }
    int* sweeps = h->d_flags + 6;                               // slots 6 and 7
    for (int g = 0; g < nmat; ++g) {
        {
            ProfScope ps(h, HUB_K_EIG_MISC);
            k_eye<<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(Vt[g], n);
        }
        HUB_CUDA_TRY(h, cudaGetLastError());
        HUB_CUDA_TRY(h, cudaMemsetAsync(red[g], 0, 4 * sizeof(unsigned long long), h->stream));
    }
    HUB_CUDA_TRY(h, cudaMemsetAsync(h->d_bar, 0, 4 * sizeof(unsigned int), h->stream));
    HUB_CUDA_TRY(h, cudaMemsetAsync(sweeps, 0, 2 * sizeof(int), h->stream));
    int per_sm = 0;
    const size_t rot_bytes = (size_t)N * sizeof(double);
    if (rot_bytes > 48 * 1024) return fail(h, HUB_EINVAL, "subspace too large for the Jacobi solver");
    HUB_CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, 256, rot_bytes));
    int blocks = std::max(1, std::min(per_sm, 1)) * h->num_sms / nmat;   // per matrix
    const long work = (long)(N / 2) * (N / 2 + 1) / 2 + (long)n * (N / 2);
    blocks = (int)std::min<long>(blocks, std::max<long>(1, (work + 255) / 256));
    blocks = std::max(1, blocks) * nmat;
    int max_sweeps = 60;
    double tol = 1e-13;
    unsigned int* bar = h->d_bar;
    int* flags = h->d_flags;
    double* A0 = A[0];
    double* A1 = nmat > 1 ? A[1] : A[0];
    void* args[] = {&A0, &Ab[0], &Vt[0], &A1, &Ab[1], &Vt[1], &nmat, &n, (void*)&N, &max_sweeps, &tol, &bar,
                    &flags, &red[0], &red[1], &sweeps};
    {
        ProfScope ps(h, HUB_K_JACOBI);
        HUB_CUDA_TRY(h, cudaLaunchCooperativeKernel((void*)k_jacobi, dim3(blocks), dim3(256), args, rot_bytes,
                                                    h->stream));
    }
    for (int g = 0; g < nmat; ++g) {
        ProfScope ps(h, HUB_K_EIG_MISC);
        k_sort_eig<<<(n + 127) / 128, 128, 0, h->stream>>>(A[g], Vt[g], n, eig[g], V[g]);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int dense_jacobi_eigh(hub_t h, double* A, double* V, double* eig, int n) {
    return dense_jacobi_eigh_multi(h, 1, &A, &V, &eig, n);
}

}  // namespace hub
