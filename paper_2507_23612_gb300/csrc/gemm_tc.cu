// BF16 tensor-core Rayleigh-Ritz products (CheFSI, Sec. II.B) on tcgen05 (sm_103a):
//
//   projected Hamiltonian  G = alpha * A^T B      A, B: float blocks Nd x m, Nd x n
//   rotation               Y = X Q                X: float block Nd x k, Q: double k x n
//
// Both are written as one "TN" product D[M x N] = sum_K A[M x K] B[N x K]^T with K-major
// operands: for the projected Hamiltonian M, N are orbitals and K the grid (split over
// CTAs, FP32 partial tiles reduced in double); for the rotation M is the grid (X is
// transposed into a K-major copy), N the orbitals, K the subspace.
//
// Operands are rounded to BF16 in a conversion pass.  With TERMS = 3 each float x is split
// as x = hi + lo (hi = bf16(x), lo = bf16(x - hi)) and the product is hi*hi + hi*lo + lo*hi
// (about 16 significand bits); with TERMS = 1 it is hi*hi.  Accumulation is FP32 in TMEM.
//
// Kernel: 128 threads.  Thread 0 issues TMA loads (cp.async.bulk.tensor, SWIZZLE_128B,
// 128 rows x 64 BF16 per tile) into an S-stage shared ring guarded by mbarriers; thread 32
// issues tcgen05.mma (M = 128, N = 128, K = 16 per instruction) into TMEM and releases
// stages with tcgen05.commit; then all four warps read their 32 TMEM lanes with tcgen05.ld
// and write the tile.  Every mbarrier wait is bounded: after kSpinLimit polls the kernel
// raises FLAG_TIMEOUT, stops issuing, waits (bounded) for the work it issued, frees TMEM
// and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <mutex>

#include "hub_internal.cuh"
#include "tcgen05.cuh"

namespace hub {

namespace {

constexpr int TM = 128;                 // rows of A per tile (TMEM lanes)
constexpr int TN = 128;                 // rows of B per tile (TMEM columns per n-tile)
constexpr int TKC = 64;                 // K elements per stage (128 bytes of BF16)
constexpr int TILE_BYTES = TM * TKC * 2;  // 16 KB
struct TcArgs {
    int m, n;              // valid rows of A-side (M) and B-side (N) of the product
    int kchunks_total;     // K / 64 rounded up
    int kchunks_per;       // chunks per split
    int ntiles;            // n-tiles handled by one CTA (<= NT)
    int mode;              // 0: partial tiles part[split][m][n]; 1: Y[row + col*ldy]
    float* part;
    float* Y;
    long ldy;
    int* flags;
};

// grid: x = m-tiles, y = n-tile groups, z = K splits
template <int NT, int TERMS, int S>
__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap mapA_hi, const __grid_constant__ CUtensorMap mapA_lo,
          const __grid_constant__ CUtensorMap mapB_hi, const __grid_constant__ CUtensorMap mapB_lo, TcArgs a) {
    constexpr int NA = TERMS == 1 ? 1 : 2;                // A tiles per stage (hi, lo)
    constexpr int NB = (TERMS == 1 ? 1 : 2) * NT;         // B tiles per stage
    constexpr int STAGE = (NA + NB) * TILE_BYTES;
    constexpr int TCOLS = NT * TN <= 32 ? 32 : (NT * TN <= 64 ? 64 : (NT * TN <= 128 ? 128 : (NT * TN <= 256 ? 256 : 512)));
    extern __shared__ __align__(1024) unsigned char dsm[];
    unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    __shared__ int issued_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x;
    const int nt0 = blockIdx.y * NT;
    const int ntl = min(NT, a.ntiles - nt0);                // n-tiles of this CTA
    const int split = blockIdx.z;
    const int kc0 = split * a.kchunks_per;
    const int kc1 = min(a.kchunks_total, kc0 + a.kchunks_per);

    if (threadIdx.x == 0) {
        abort_flag = 0;
        issued_sh = 0;
        for (int s = 0; s < S; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        mbar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)), "r"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int nk = kc1 - kc0;

    if (threadIdx.x == 0 && nk > 0) {
        // producer
        int issued = 0;
        for (int i = 0; i < nk; ++i) {
            const int s = i % S;
            if (i >= S && !mbar_wait(&empty_bar[s], ((i / S) - 1) & 1, &abort_flag)) break;
            unsigned char* st = ring + (size_t)s * STAGE;
            mbar_expect_tx(&full_bar[s], (uint32_t)((NA + (TERMS == 1 ? 1 : 2) * ntl) * TILE_BYTES));
            const int kx = (kc0 + i) * TKC;
            tma_load_2d(st, &mapA_hi, kx, mt * TM, &full_bar[s]);
            if (TERMS != 1) tma_load_2d(st + TILE_BYTES, &mapA_lo, kx, mt * TM, &full_bar[s]);
            for (int j = 0; j < ntl; ++j) {
                unsigned char* bt = st + (size_t)(NA + j * (TERMS == 1 ? 1 : 2)) * TILE_BYTES;
                tma_load_2d(bt, &mapB_hi, kx, (nt0 + j) * TN, &full_bar[s]);
                if (TERMS != 1) tma_load_2d(bt + TILE_BYTES, &mapB_lo, kx, (nt0 + j) * TN, &full_bar[s]);
            }
            issued = i + 1;
        }
        issued_sh = issued;
    } else if (threadIdx.x == 32 && nk > 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc_bf16(TM, TN);
        for (int i = 0; i < nk; ++i) {
            const int s = i % S;
            if (!mbar_wait(&full_bar[s], (i / S) & 1, &abort_flag)) break;
            tc_fence_after();
            unsigned char* st = ring + (size_t)s * STAGE;
            for (int j = 0; j < ntl; ++j) {
                unsigned char* bt = st + (size_t)(NA + j * (TERMS == 1 ? 1 : 2)) * TILE_BYTES;
                const uint32_t dcol = tmem + (uint32_t)(j * TN);
#pragma unroll
                for (int kk = 0; kk < TKC / 16; ++kk) {
                    const uint64_t koff = (uint64_t)(kk * 32) >> 4;    // 16 BF16 = 32 bytes
                    const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
                    mma_bf16(dcol, smem_desc(st) + koff, smem_desc(bt) + koff, idesc, acc);
                    if (TERMS != 1) {
                        mma_bf16(dcol, smem_desc(st) + koff, smem_desc(bt + TILE_BYTES) + koff, idesc, 1u);
                        mma_bf16(dcol, smem_desc(st + TILE_BYTES) + koff, smem_desc(bt) + koff, idesc, 1u);
                    }
                }
            }
            mma_commit(&empty_bar[s]);       // stage free once these MMAs complete
        }
        mma_commit(&done_bar);               // accumulators final once everything completes
    } else if (threadIdx.x == 32) {
        mma_commit(&done_bar);
    }
    __syncwarp();

    // epilogue: all 128 threads, warp w owns TMEM lanes 32w .. 32w+31 (rows of the tile);
    // the done barrier completes once every issued MMA has (waited on even after an abort)
    const bool ok = mbar_drain(&done_bar, 0);
    if (!ok) abort_flag = 1;
    tc_fence_after();
    if (ok && nk > 0 && !abort_flag) {
        const int row = mt * TM + warp * 32 + lane;
        for (int j = 0; j < ntl; ++j) {
            for (int c = 0; c < TN; c += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * TN + c), v);
                const int col0 = (nt0 + j) * TN + c;
                if (a.mode == 0) {
                    if (row < a.m) {
                        float* dst = a.part + ((size_t)split * a.m + row) * a.n;
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (col0 + q < a.n) dst[col0 + q] = v[q];
                    }
                } else {
                    if (row < a.m) {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (col0 + q < a.n) a.Y[(size_t)(col0 + q) * a.ldy + row] = v[q];
                    }
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) {
        atomicExch(a.flags + FLAG_TIMEOUT, 1);
        // let the TMA copies still in flight land before shared memory goes away
        const int issued = issued_sh;
        for (int i = issued > S ? issued - S : 0; i < issued; ++i) mbar_drain(&full_bar[i % S], (i / S) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

// ---------------------------------------------------------------------------- conversions
// column-major float block (ld) -> column-major BF16 hi / lo copies (ldb)
__global__ void k_split_bf16(const float* __restrict__ X, long ld, long Nd, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo, long ldb) {
    const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Nd) return;
    const float x = X[(size_t)blockIdx.y * ld + g];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[(size_t)blockIdx.y * ldb + g] = h;
    if (lo) lo[(size_t)blockIdx.y * ldb + g] = __float2bfloat16_rn(x - __bfloat162float(h));
}

// column-major float block (Nd x k, ld) -> row-major BF16 [Nd][kp] hi / lo (a transpose
// through 32 x 32 shared tiles, coalesced on both sides)
__global__ void k_split_bf16_T(const float* __restrict__ X, long ld, long Nd, int k, __nv_bfloat16* __restrict__ hi,
                               __nv_bfloat16* __restrict__ lo, int kp) {
    __shared__ float t[32][33];
    const long g0 = (long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int c = c0 + r;
        const long g = g0 + threadIdx.x;
        t[r][threadIdx.x] = (c < k && g < Nd) ? X[(size_t)c * ld + g] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const long g = g0 + r;
        const int c = c0 + threadIdx.x;
        if (g < Nd && c < kp) {
            const float x = t[threadIdx.x][r];
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            hi[(size_t)g * kp + c] = h;
            if (lo) lo[(size_t)g * kp + c] = __float2bfloat16_rn(x - __bfloat162float(h));
        }
    }
}

// Q (double, row-major k x n) -> Qt BF16 [n][kp]: row j holds column j of Q
__global__ void k_q_bf16_T(const double* __restrict__ Q, int k, int n, __nv_bfloat16* __restrict__ hi,
                           __nv_bfloat16* __restrict__ lo, int kp) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * kp) return;
    const int j = (int)(t / kp), c = (int)(t % kp);
    const float x = c < k ? (float)Q[(size_t)c * n + j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[t] = h;
    if (lo) lo[t] = __float2bfloat16_rn(x - __bfloat162float(h));
}

__global__ void k_reduce_partials(const float* __restrict__ part, int splits, int m, int n, double alpha,
                                  int sym, double* __restrict__ G) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)m * n) return;
    int i = (int)(t / n), j = (int)(t % n);
    if (sym && (i / TN) > (j / TN)) { const int q = i; i = j; j = q; }
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += (double)part[(size_t)z * m * n + (size_t)i * n + j];
    G[t] = alpha * s;
}

// ---------------------------------------------------------------------------- host
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

int get_encoder(hub_t h) {
    std::lock_guard<std::mutex> lk(g_encode_mu);
    if (g_encode) return HUB_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    HUB_CUDA_TRY(h, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (!fn || q != cudaDriverEntryPointSuccess) return fail(h, HUB_ECUDA, "cuTensorMapEncodeTiled unavailable");
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return HUB_OK;
}

// 2-D BF16 map: rows of `inner` contiguous elements (row stride `stride_elems`), 64 x 128 box
int make_map(hub_t h, CUtensorMap* map, const void* base, long inner, long rows, long stride_elems) {
    if ((uintptr_t)base % 16 != 0 || (stride_elems * 2) % 16 != 0)
        return fail(h, HUB_EINVAL, "BF16 operand not 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(stride_elems * 2)};
    cuuint32_t box[2] = {TKC, TM};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, HUB_ECUDA, "cuTensorMapEncodeTiled failed");
    return HUB_OK;
}

template <int NT, int TERMS, int S>
int launch_tc(hub_t h, const CUtensorMap& ahi, const CUtensorMap& alo, const CUtensorMap& bhi,
              const CUtensorMap& blo, const TcArgs& a, dim3 grid) {
    constexpr int NA = TERMS == 1 ? 1 : 2;
    constexpr int NB = (TERMS == 1 ? 1 : 2) * NT;
    constexpr size_t SMEM = (size_t)S * (NA + NB) * TILE_BYTES + 1024;
    static_assert(SMEM <= 227 * 1024, "stage ring exceeds shared memory");
    HUB_CUDA_TRY(h, cudaFuncSetAttribute(k_tc_gemm<NT, TERMS, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
    ProfScope ps(h, a.mode == 0 ? HUB_K_GRAM : HUB_K_ROTATE);
    k_tc_gemm<NT, TERMS, S><<<grid, 128, SMEM, h->stream>>>(ahi, alo, bhi, blo, a);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

}  // namespace

int tensor_map_encoder(hub_t h, PFN_cuTensorMapEncodeTiled_v12000* out) {
    const int rc = get_encoder(h);
    if (rc) return rc;
    *out = g_encode;
    return HUB_OK;
}

// G[m x n] = alpha * A^T B with BF16 tensor-core products (A, B float, column-major)
int launch_gram_bf16(hub_t h, const void* A, int lda, const void* B, int ldb, int m, int n, double alpha,
                     bool sym, double* G) {
    if (h->cplx || h->esize != 4) return fail(h, HUB_EINVAL, "BF16 products take real float blocks");
    if (m == 0 || n == 0) return HUB_OK;
    int rc;
    if ((rc = get_encoder(h))) return rc;
    const int terms = h->bf16_terms;
    const long Nd = h->Nd;
    const long ldh = (Nd + 7) / 8 * 8;
    const bool same = (A == B) && (lda == ldb) && (m == n);
    const size_t per = (size_t)ldh * 2;
    const size_t nA = (size_t)m * per, nB = same ? 0 : (size_t)n * per;
    const size_t bytes = (nA + nB) * (terms == 1 ? 1 : 2) + 256;
    if ((rc = ensure(h, &h->d_bf16, &h->bf16_bytes, std::max(bytes, h->bf16_bytes)))) return rc;
    __nv_bfloat16* ahi = (__nv_bfloat16*)h->d_bf16;
    __nv_bfloat16* alo = terms == 1 ? nullptr : (__nv_bfloat16*)((char*)ahi + nA);
    __nv_bfloat16* bhi = same ? ahi : (__nv_bfloat16*)((char*)h->d_bf16 + nA * (terms == 1 ? 1 : 2));
    __nv_bfloat16* blo = same ? alo : (terms == 1 ? nullptr : (__nv_bfloat16*)((char*)bhi + nB));
    {
        ProfScope ps(h, HUB_K_COPY);
        k_split_bf16<<<dim3((unsigned)((Nd + 255) / 256), m), 256, 0, h->stream>>>((const float*)A, lda, Nd, ahi, alo, ldh);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    if (!same) {
        ProfScope ps(h, HUB_K_COPY);
        k_split_bf16<<<dim3((unsigned)((Nd + 255) / 256), n), 256, 0, h->stream>>>((const float*)B, ldb, Nd, bhi, blo, ldh);
        HUB_CUDA_TRY(h, cudaGetLastError());
    }
    CUtensorMap mA, mAl, mB, mBl;
    if ((rc = make_map(h, &mA, ahi, Nd, m, ldh))) return rc;
    if ((rc = make_map(h, &mB, bhi, Nd, n, ldh))) return rc;
    mAl = mA; mBl = mB;
    if (terms != 1) {
        if ((rc = make_map(h, &mAl, alo, Nd, m, ldh))) return rc;
        if ((rc = make_map(h, &mBl, blo, Nd, n, ldh))) return rc;
    }
    const int mtiles = (m + TM - 1) / TM, ntiles = (n + TN - 1) / TN;
    const int kchunks = (int)((Nd + TKC - 1) / TKC);
    const int tiles = mtiles * ntiles;
    int splits = std::max(1, (h->gemm_split * h->num_sms + tiles - 1) / tiles);
    int per_split = (kchunks + splits - 1) / splits;
    splits = (kchunks + per_split - 1) / per_split;
    if ((rc = ensure(h, &h->d_gpart, &h->gpart_bytes, std::max(h->gpart_bytes, (size_t)splits * m * n * sizeof(float)))))
        return rc;
    TcArgs ta{};
    ta.m = m; ta.n = n; ta.kchunks_total = kchunks; ta.kchunks_per = per_split; ta.ntiles = ntiles;
    ta.mode = 0; ta.part = (float*)h->d_gpart; ta.Y = nullptr; ta.ldy = 0; ta.flags = h->d_flags;
    dim3 grid(mtiles, ntiles, splits);
    if (terms == 1) rc = launch_tc<1, 1, 4>(h, mA, mAl, mB, mBl, ta, grid);
    else rc = launch_tc<1, 3, 3>(h, mA, mAl, mB, mBl, ta, grid);
    if (rc) return rc;
    {
        ProfScope ps(h, HUB_K_GRAM_REDUCE);
        const long tot = (long)m * n;
        k_reduce_partials<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>((const float*)h->d_gpart, splits, m, n,
                                                                                alpha, 0, G);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    (void)sym;
    return HUB_OK;
}

// Y[Nd x n] = X[Nd x k] Q[k x n] with BF16 tensor-core products (X, Y float column-major;
// Q double row-major)
int launch_rotate_bf16(hub_t h, const void* X, int ldx, const double* Q, int k, int n, void* Y, int ldy) {
    if (h->cplx || h->esize != 4) return fail(h, HUB_EINVAL, "BF16 products take real float blocks");
    if (n == 0) return HUB_OK;
    int rc;
    if ((rc = get_encoder(h))) return rc;
    const int terms = h->bf16_terms;
    const long Nd = h->Nd;
    const int kp = (k + TKC - 1) / TKC * TKC;
    const size_t nX = (size_t)Nd * kp * 2, nQ = (size_t)n * kp * 2;
    const size_t bytes = (nX + nQ) * (terms == 1 ? 1 : 2) + 256;
    if ((rc = ensure(h, &h->d_bf16, &h->bf16_bytes, std::max(bytes, h->bf16_bytes)))) return rc;
    __nv_bfloat16* xhi = (__nv_bfloat16*)h->d_bf16;
    __nv_bfloat16* xlo = terms == 1 ? nullptr : (__nv_bfloat16*)((char*)xhi + nX);
    __nv_bfloat16* qhi = (__nv_bfloat16*)((char*)h->d_bf16 + nX * (terms == 1 ? 1 : 2));
    __nv_bfloat16* qlo = terms == 1 ? nullptr : (__nv_bfloat16*)((char*)qhi + nQ);
    {
        ProfScope ps(h, HUB_K_COPY);
        k_split_bf16_T<<<dim3((unsigned)((Nd + 31) / 32), (kp + 31) / 32), dim3(32, 8), 0, h->stream>>>(
            (const float*)X, ldx, Nd, k, xhi, xlo, kp);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    {
        ProfScope ps(h, HUB_K_COPY);
        const long tot = (long)n * kp;
        k_q_bf16_T<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(Q, k, n, qhi, qlo, kp);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    CUtensorMap mA, mAl, mB, mBl;
    if ((rc = make_map(h, &mA, xhi, kp, Nd, kp))) return rc;
    if ((rc = make_map(h, &mB, qhi, kp, n, kp))) return rc;
    mAl = mA; mBl = mB;
    if (terms != 1) {
        if ((rc = make_map(h, &mAl, xlo, kp, Nd, kp))) return rc;
        if ((rc = make_map(h, &mBl, qlo, kp, n, kp))) return rc;
    }
    const int mtiles = (int)((Nd + TM - 1) / TM), ntiles = (n + TN - 1) / TN;
    TcArgs ta{};
    ta.m = (int)Nd; ta.n = n; ta.kchunks_total = kp / TKC; ta.kchunks_per = kp / TKC; ta.ntiles = ntiles;
    ta.mode = 1; ta.part = nullptr; ta.Y = (float*)Y; ta.ldy = ldy; ta.flags = h->d_flags;
    if (terms == 1) {
        dim3 grid(mtiles, (ntiles + 3) / 4, 1);
        return launch_tc<4, 1, 2>(h, mA, mAl, mB, mBl, ta, grid);
    }
    dim3 grid(mtiles, (ntiles + 1) / 2, 1);
    return launch_tc<2, 3, 2>(h, mA, mAl, mB, mBl, ta, grid);
}

}  // namespace hub
