// BF16 / FP16 tensor-core Rayleigh-Ritz products (CheFSI, Sec. II.B) on tcgen05 (sm_103a):
//
//   projected Hamiltonian  G = alpha * A^T B      A, B: float blocks Nd x m, Nd x n
//   rotation               Y = X Q                X: float block Nd x k, Q: double k x n
//
// Both are written as one "TN" product D[M x N] = sum_K A[M x K] B[N x K]^T with K-major
// operands: for the projected Hamiltonian M, N are orbitals and K the grid (split over
// CTAs, FP32 partial tiles reduced in double); for the rotation M is the grid (X is
// transposed into a K-major copy), N the orbitals, K the subspace.
//
// Operands are rounded to a 16-bit type t16 in a conversion pass.  With TERMS = 3 each float
// x is split as x = hi + lo (hi = t16(x), lo = t16(x - hi)) and the product is hi*hi + hi*lo
// + lo*hi (about 16 significand bits with BF16, 22 with FP16); with TERMS = 1 it is hi*hi.
// Accumulation is FP32 in TMEM.  FP16 has 5 exponent bits, so each FP16 operand block is
// first scaled by a power of two 2^s that puts its largest magnitude in [2^14, 2^15)
// (a max-|x| reduction on the device gives s; scaling by 2^s is exact), and the result is
// scaled back by 2^-(sA + sB) in the reduction or in the rotation's epilogue.
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
#include <cuda_fp16.h>
#include <algorithm>
#include <mutex>
#include <type_traits>

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
    const unsigned* maxbits;   // FP16 operands: max |x| bit patterns of A [0] and B [1]
};

// FP16 operand scaling: the exponent s with max * 2^s in [2^14, 2^15) for the largest
// magnitude max (as float bits); s = 0 for an all-zero block
__device__ __forceinline__ int f16_shift(unsigned mbits) {
    if (mbits == 0u) return 0;
    const int e = (int)((mbits >> 23) & 0xffu) - 127;
    return min(120, max(-120, 14 - e));
}
__device__ __forceinline__ float pow2f(int s) { return __int_as_float((s + 127) << 23); }   // |s| <= 126

template <typename T16>
struct Half16;
template <>
struct Half16<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 from(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float to(__nv_bfloat16 x) { return __bfloat162float(x); }
};
template <>
struct Half16<__half> {
    static __device__ __forceinline__ __half from(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float to(__half x) { return __half2float(x); }
};

// grid: x = m-tiles, y = n-tile groups, z = K splits
template <int NT, int TERMS, int S, bool F16>
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
        const uint32_t idesc = F16 ? instr_desc_f16(TM, TN) : instr_desc_bf16(TM, TN);
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
        // FP16 rotation: remove the operand scales 2^(sA + sB) from the tile
        const int unshift = (F16 && a.mode == 1) ? f16_shift(a.maxbits[0]) + f16_shift(a.maxbits[1]) : 0;
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
                            if (col0 + q < a.n)
                                a.Y[(size_t)(col0 + q) * a.ldy + row] = F16 ? ldexpf(v[q], -unshift) : v[q];
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
// largest |x| of a column-major block (rows x cols, ld) as float bits, merged into *out by
// atomicMax (non-negative floats order like their bit patterns); *out starts at 0
template <typename T>
__global__ void k_absmax(const T* __restrict__ X, long ld, long rows, unsigned* __restrict__ out) {
    const T* col = X + (size_t)blockIdx.y * ld;
    float m = 0.f;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < rows; g += (long)gridDim.x * blockDim.x)
        m = fmaxf(m, (float)fabs((double)col[g]));
    unsigned b = __float_as_uint(m);
    b = __reduce_max_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0 && b != 0u) atomicMax(out, b);
}

// scale factor 2^s of an operand: 1 for BF16 (mx == nullptr), else from its max |x|
__device__ __forceinline__ float operand_scale(const unsigned* mx) { return mx ? pow2f(f16_shift(*mx)) : 1.f; }

// column-major float block (ld) -> column-major 16-bit hi / lo copies (ldb)
template <typename T16>
__global__ void k_split16(const float* __restrict__ X, long ld, long Nd, T16* __restrict__ hi, T16* __restrict__ lo,
                          long ldb, const unsigned* __restrict__ mx) {
    const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Nd) return;
    const float x = X[(size_t)blockIdx.y * ld + g] * operand_scale(mx);
    const T16 h = Half16<T16>::from(x);
    hi[(size_t)blockIdx.y * ldb + g] = h;
    if (lo) lo[(size_t)blockIdx.y * ldb + g] = Half16<T16>::from(x - Half16<T16>::to(h));
}

// column-major float block (Nd x k, ld) -> row-major 16-bit [Nd][kp] hi / lo (a transpose
// through 32 x 32 shared tiles, coalesced on both sides)
template <typename T16>
__global__ void k_split16_T(const float* __restrict__ X, long ld, long Nd, int k, T16* __restrict__ hi,
                            T16* __restrict__ lo, int kp, const unsigned* __restrict__ mx) {
    __shared__ float t[32][33];
    const long g0 = (long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    const float sc = operand_scale(mx);
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int c = c0 + r;
        const long g = g0 + threadIdx.x;
        t[r][threadIdx.x] = (c < k && g < Nd) ? X[(size_t)c * ld + g] * sc : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const long g = g0 + r;
        const int c = c0 + threadIdx.x;
        if (g < Nd && c < kp) {
            const float x = t[threadIdx.x][r];
            const T16 h = Half16<T16>::from(x);
            hi[(size_t)g * kp + c] = h;
            if (lo) lo[(size_t)g * kp + c] = Half16<T16>::from(x - Half16<T16>::to(h));
        }
    }
}

// Q (double, row-major k x n) -> Qt 16-bit [n][kp]: row j holds column j of Q
template <typename T16>
__global__ void k_q16_T(const double* __restrict__ Q, int k, int n, T16* __restrict__ hi, T16* __restrict__ lo, int kp,
                        const unsigned* __restrict__ mx) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * kp) return;
    const int j = (int)(t / kp), c = (int)(t % kp);
    const float x = c < k ? (float)Q[(size_t)c * n + j] * operand_scale(mx) : 0.f;
    const T16 h = Half16<T16>::from(x);
    hi[t] = h;
    if (lo) lo[t] = Half16<T16>::from(x - Half16<T16>::to(h));
}

// G = alpha * sum of the split partials; FP16 operands (mx != nullptr): times 2^-(sA + sB)
__global__ void k_reduce_partials(const float* __restrict__ part, int splits, int m, int n, double alpha,
                                  int sym, double* __restrict__ G, const unsigned* __restrict__ mx) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)m * n) return;
    int i = (int)(t / n), j = (int)(t % n);
    if (sym && (i / TN) > (j / TN)) { const int q = i; i = j; j = q; }
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += (double)part[(size_t)z * m * n + (size_t)i * n + j];
    if (mx) s = ldexp(s, -(f16_shift(mx[0]) + f16_shift(mx[1])));
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

// 2-D map of 16-bit elements (BF16 or FP16): rows of `inner` contiguous elements (row stride
// `stride_elems`), 64 x 128 box
int make_map(hub_t h, CUtensorMap* map, const void* base, long inner, long rows, long stride_elems, bool f16) {
    if ((uintptr_t)base % 16 != 0 || (stride_elems * 2) % 16 != 0)
        return fail(h, HUB_EINVAL, "16-bit operand not 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(stride_elems * 2)};
    cuuint32_t box[2] = {TKC, TM};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, HUB_ECUDA, "cuTensorMapEncodeTiled failed");
    return HUB_OK;
}

template <int NT, int TERMS, int S, bool F16>
int launch_tc(hub_t h, const CUtensorMap& ahi, const CUtensorMap& alo, const CUtensorMap& bhi,
              const CUtensorMap& blo, const TcArgs& a, dim3 grid) {
    constexpr int NA = TERMS == 1 ? 1 : 2;
    constexpr int NB = (TERMS == 1 ? 1 : 2) * NT;
    constexpr size_t SMEM = (size_t)S * (NA + NB) * TILE_BYTES + 1024;
    static_assert(SMEM <= 227 * 1024, "stage ring exceeds shared memory");
    HUB_CUDA_TRY(h, cudaFuncSetAttribute(k_tc_gemm<NT, TERMS, S, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
    ProfScope ps(h, a.mode == 0 ? HUB_K_GRAM : HUB_K_ROTATE);
    k_tc_gemm<NT, TERMS, S, F16><<<grid, 128, SMEM, h->stream>>>(ahi, alo, bhi, blo, a);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

// largest |x| of a column-major block into *out (device), FP16 operands only
template <typename T>
int launch_absmax(hub_t h, const T* X, long ld, long rows, int cols, unsigned* out) {
    if (rows <= 0 || cols <= 0) return HUB_OK;
    ProfScope ps(h, HUB_K_COPY);
    const unsigned bx = (unsigned)std::min<long>((rows + 255) / 256, std::max(1L, 4L * h->num_sms / cols + 1));
    k_absmax<T><<<dim3(bx, (unsigned)cols), 256, 0, h->stream>>>(X, ld, rows, out);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

template <typename T16>
int gram16(hub_t h, const void* A, int lda, const void* B, int ldb, int m, int n, double alpha, double* G) {
    constexpr bool F16 = std::is_same<T16, __half>::value;
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
    T16* ahi = (T16*)h->d_bf16;
    T16* alo = terms == 1 ? nullptr : (T16*)((char*)ahi + nA);
    T16* bhi = same ? ahi : (T16*)((char*)h->d_bf16 + nA * (terms == 1 ? 1 : 2));
    T16* blo = same ? alo : (terms == 1 ? nullptr : (T16*)((char*)bhi + nB));
    // FP16: max |x| of A into d_tcmax[0] and of B into d_tcmax[1] (the same slot twice when
    // A is B), read by the conversions and by the reduction
    const unsigned* mxA = nullptr;
    const unsigned* mxB = nullptr;
    if (F16) {
        HUB_CUDA_TRY(h, cudaMemsetAsync(h->d_tcmax, 0, 4 * sizeof(unsigned), h->stream));
        if ((rc = launch_absmax(h, (const float*)A, lda, Nd, m, h->d_tcmax))) return rc;
        if (!same && (rc = launch_absmax(h, (const float*)B, ldb, Nd, n, h->d_tcmax + 1))) return rc;
        if (same) HUB_CUDA_TRY(h, cudaMemcpyAsync(h->d_tcmax + 1, h->d_tcmax, sizeof(unsigned), cudaMemcpyDeviceToDevice, h->stream));
        mxA = h->d_tcmax;
        mxB = h->d_tcmax + 1;
    }
    {
        ProfScope ps(h, HUB_K_COPY);
        k_split16<T16><<<dim3((unsigned)((Nd + 255) / 256), m), 256, 0, h->stream>>>((const float*)A, lda, Nd, ahi, alo,
                                                                                     ldh, mxA);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    if (!same) {
        ProfScope ps(h, HUB_K_COPY);
        k_split16<T16><<<dim3((unsigned)((Nd + 255) / 256), n), 256, 0, h->stream>>>((const float*)B, ldb, Nd, bhi, blo,
                                                                                     ldh, mxB);
        HUB_CUDA_TRY(h, cudaGetLastError());
    }
    CUtensorMap mA, mAl, mB, mBl;
    if ((rc = make_map(h, &mA, ahi, Nd, m, ldh, F16))) return rc;
    if ((rc = make_map(h, &mB, bhi, Nd, n, ldh, F16))) return rc;
    mAl = mA; mBl = mB;
    if (terms != 1) {
        if ((rc = make_map(h, &mAl, alo, Nd, m, ldh, F16))) return rc;
        if ((rc = make_map(h, &mBl, blo, Nd, n, ldh, F16))) return rc;
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
    ta.maxbits = mxA;
    dim3 grid(mtiles, ntiles, splits);
    if (terms == 1) rc = launch_tc<1, 1, 4, F16>(h, mA, mAl, mB, mBl, ta, grid);
    else rc = launch_tc<1, 3, 3, F16>(h, mA, mAl, mB, mBl, ta, grid);
    if (rc) return rc;
    {
        ProfScope ps(h, HUB_K_GRAM_REDUCE);
        const long tot = (long)m * n;
        k_reduce_partials<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>((const float*)h->d_gpart, splits, m, n,
                                                                                alpha, 0, G, mxA);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

template <typename T16>
int rotate16(hub_t h, const void* X, int ldx, const double* Q, int k, int n, void* Y, int ldy) {
    constexpr bool F16 = std::is_same<T16, __half>::value;
    int rc;
    if ((rc = get_encoder(h))) return rc;
    const int terms = h->bf16_terms;
    const long Nd = h->Nd;
    const int kp = (k + TKC - 1) / TKC * TKC;
    const size_t nX = (size_t)Nd * kp * 2, nQ = (size_t)n * kp * 2;
    const size_t bytes = (nX + nQ) * (terms == 1 ? 1 : 2) + 256;
    if ((rc = ensure(h, &h->d_bf16, &h->bf16_bytes, std::max(bytes, h->bf16_bytes)))) return rc;
    T16* xhi = (T16*)h->d_bf16;
    T16* xlo = terms == 1 ? nullptr : (T16*)((char*)xhi + nX);
    T16* qhi = (T16*)((char*)h->d_bf16 + nX * (terms == 1 ? 1 : 2));
    T16* qlo = terms == 1 ? nullptr : (T16*)((char*)qhi + nQ);
    // FP16: max |x| of X into d_tcmax[0] and of Q into d_tcmax[1]
    const unsigned* mxX = nullptr;
    const unsigned* mxQ = nullptr;
    if (F16) {
        HUB_CUDA_TRY(h, cudaMemsetAsync(h->d_tcmax, 0, 4 * sizeof(unsigned), h->stream));
        if ((rc = launch_absmax(h, (const float*)X, ldx, Nd, k, h->d_tcmax))) return rc;
        if ((rc = launch_absmax(h, Q, (long)k * n, (long)k * n, 1, h->d_tcmax + 1))) return rc;
        mxX = h->d_tcmax;
        mxQ = h->d_tcmax + 1;
    }
    {
        ProfScope ps(h, HUB_K_COPY);
        k_split16_T<T16><<<dim3((unsigned)((Nd + 31) / 32), (kp + 31) / 32), dim3(32, 8), 0, h->stream>>>(
            (const float*)X, ldx, Nd, k, xhi, xlo, kp, mxX);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    {
        ProfScope ps(h, HUB_K_COPY);
        const long tot = (long)n * kp;
        k_q16_T<T16><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(Q, k, n, qhi, qlo, kp, mxQ);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    CUtensorMap mA, mAl, mB, mBl;
    if ((rc = make_map(h, &mA, xhi, kp, Nd, kp, F16))) return rc;
    if ((rc = make_map(h, &mB, qhi, kp, n, kp, F16))) return rc;
    mAl = mA; mBl = mB;
    if (terms != 1) {
        if ((rc = make_map(h, &mAl, xlo, kp, Nd, kp, F16))) return rc;
        if ((rc = make_map(h, &mBl, qlo, kp, n, kp, F16))) return rc;
    }
    const int mtiles = (int)((Nd + TM - 1) / TM), ntiles = (n + TN - 1) / TN;
    TcArgs ta{};
    ta.m = (int)Nd; ta.n = n; ta.kchunks_total = kp / TKC; ta.kchunks_per = kp / TKC; ta.ntiles = ntiles;
    ta.mode = 1; ta.part = nullptr; ta.Y = (float*)Y; ta.ldy = ldy; ta.flags = h->d_flags;
    ta.maxbits = mxX;
    if (terms == 1) {
        dim3 grid(mtiles, (ntiles + 3) / 4, 1);
        return launch_tc<4, 1, 2, F16>(h, mA, mAl, mB, mBl, ta, grid);
    }
    dim3 grid(mtiles, (ntiles + 1) / 2, 1);
    return launch_tc<2, 3, 2, F16>(h, mA, mAl, mB, mBl, ta, grid);
}

}  // namespace

int tensor_map_encoder(hub_t h, PFN_cuTensorMapEncodeTiled_v12000* out) {
    const int rc = get_encoder(h);
    if (rc) return rc;
    *out = g_encode;
    return HUB_OK;
}

// G[m x n] = alpha * A^T B with 16-bit tensor-core products (A, B float, column-major); the
// operand type is the handle's (BF16 or FP16)
int launch_gram_bf16(hub_t h, const void* A, int lda, const void* B, int ldb, int m, int n, double alpha,
                     bool sym, double* G) {
    (void)sym;
    if (h->cplx || h->esize != 4) return fail(h, HUB_EINVAL, "16-bit tensor-core products take real float blocks");
    if (m == 0 || n == 0) return HUB_OK;
    if (h->prec == HUB_MIXED_F16) return gram16<__half>(h, A, lda, B, ldb, m, n, alpha, G);
    return gram16<__nv_bfloat16>(h, A, lda, B, ldb, m, n, alpha, G);
}

// Y[Nd x n] = X[Nd x k] Q[k x n] with 16-bit tensor-core products (X, Y float column-major;
// Q double row-major)
int launch_rotate_bf16(hub_t h, const void* X, int ldx, const double* Q, int k, int n, void* Y, int ldy) {
    if (h->cplx || h->esize != 4) return fail(h, HUB_EINVAL, "16-bit tensor-core products take real float blocks");
    if (n == 0) return HUB_OK;
    if (h->prec == HUB_MIXED_F16) return rotate16<__half>(h, X, ldx, Q, k, n, Y, ldy);
    return rotate16<__nv_bfloat16>(h, X, ldx, Q, k, n, Y, ldy);
}

}  // namespace hub
