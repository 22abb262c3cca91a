// Tensor-core form of the projector gather (Sec. II.B: the inner products of all functions
// of an atom are computed together), for real float blocks.  The brick tables group, per
// 8 x 8 x 4 brick of the grid, the functions of the sites that touch it (entries of at most
// 64), and the tensor-core tables pack each brick's entries into groups of at most 64
// functions (one group per brick on average on the rutile workload, against six entries).
// Per group and per tile of 128 orbitals the partial inner products
//
//   part[prow(f), n] = sum_{p in brick} phi_f(p) X[g(p), n]
//
// are one tcgen05 product D[128 orbitals x NP functions] = X_b^T Phi_b over the K = 256
// points of the brick (summed per function over its bricks afterwards, as for the SIMT brick
// gather), so that the brick's X is loaded and split once for all the functions of the
// group.  Both operands are split for TF32: hi = the float rounded to the 10 TF32
// significand bits, lo = value - hi (exact) rounded the same way, and D = hi*hi + (hi*lo +
// lo*hi) with FP32 accumulation in TMEM, about 22 significant bits (the float path's own
// accuracy) and no rounding bias.  The two small correction
// products accumulate apart from hi*hi (the tensor core aligns the addends of a sum to the
// largest, so corrections added to the large accumulator lose their low bits) and the two
// accumulators are added when the result is read out.
//
// Operands are K-major in the 128-byte-swizzled layout of tcgen05 (rows of 128 bytes = 32
// brick points, 8-row groups of 1024 bytes, the 16-byte chunk c of row r stored at chunk
// c XOR (r % 8)).  An X slice (32 brick points = 4 rows of 8 points of one z-plane, for 128
// orbitals: one row per orbital) is copied from global memory by the converter warps with
// 16-byte cp.async (8 lanes per orbital, four slices in flight) into raw slice buffers, read
// back by the same threads and written split into hi and lo; the
// projector values are stored in the same layout when the tables are built (one row per
// function and slice) and copied with cp.async.bulk.
//
// Kernel: persistent CTAs of 320 threads over (group, orbital tile) units.  Warp 0 issues
// the value copies into a three-stage ring, warp 1 issues the MMAs into one of two TMEM
// accumulators, warps 2-5 load and split the X slices, and warps 6-9, once a unit's product
// is complete, read its accumulator (tcgen05.ld) and write the partial rows while the next
// unit is converted and multiplied.  Every mbarrier
// wait is bounded: after its limit the CTA raises FLAG_TIMEOUT, stops issuing, drains the
// copies and MMAs it issued, frees its TMEM and returns.
#include <algorithm>
#include <vector>

#include "hub_internal.cuh"
#include "tcgen05.cuh"

namespace hub {

namespace {

constexpr int GT_M = 128;                     // orbitals per tile (MMA M, TMEM lanes)
constexpr int GT_K = 32;                      // brick points per slice (128 bytes of FP32)
constexpr int GT_SLICES = BRP / GT_K;         // 8 slices per brick
constexpr int GT_NP = BRF;                    // functions per group at most (MMA N)
constexpr int GT_S = 3;                       // ring stages (values and split X)
constexpr int GT_XB = GT_M * GT_K * 4;        // 16 KB: one X slice
constexpr int GT_BB = GT_NP * GT_K * 4;       // 8 KB: one value slice at most
constexpr int GT_STAGE = 2 * GT_XB + 2 * GT_BB;   // X hi, X lo, values hi, values lo
constexpr int GT_THREADS = 320;           // producer, MMA, 4 converter and 4 epilogue warps
constexpr uint32_t GT_TMEM_COLS = 4 * GT_NP;  // two units in flight x (hi*hi, corrections)
constexpr int GT_D = 4;                       // raw X slices in flight per converter thread
constexpr size_t GT_SMEM = (size_t)GT_S * GT_STAGE + (size_t)GT_D * GT_XB + 1024;
constexpr uint32_t kTf32Hi = 0xFFFFE000u;     // sign, exponent and the 10 TF32 significand bits

struct GtcArgs {
    const float* X;       // block, column-major with leading dimension ld
    const int4* grp;      // per group: brick, float offset of its values, slots NP, first slot
    const int* grow;      // per slot: partial row of its function (-1: padding)
    const float* vhi;
    const float* vlo;
    float* part;
    long ld;
    int n1, n2, n3, ncol, nbx, nby, nunits, ctiles;
    int* flags;
};

// TF32 split rounded to nearest (ties away from zero in magnitude): hi = x rounded to the 10
// TF32 significand bits, lo = x - hi (exact in float, |lo| <= 2^-11 |x|) rounded the same
// way.  Rounding both parts to nearest keeps the split unbiased: with truncation (low bits
// cleared) hi and lo both lean towards zero and the dropped lo*lo term has the sign of the
// product, which biased every projector inner product by ~5e-7 of its value towards zero.
__device__ __forceinline__ uint32_t tf32_round(uint32_t u) { return (u + 0x1000u) & kTf32Hi; }
__device__ __forceinline__ uint32_t split_hi(uint32_t u) { return tf32_round(u); }
__device__ __forceinline__ uint32_t split_lo(uint32_t u) {
    return tf32_round(__float_as_uint(__uint_as_float(u) - __uint_as_float(tf32_round(u))));
}

// the 8 16-byte chunks a converter thread copies for slice q of group g and orbital tile ct:
// chunk j = it * 128 + c of the slice is orbital n = j / 8 of the tile, its 4 points
// x % 4 = 0..3 at x / 4 = j % 2, y-row (j / 2) % 4; each lands in the thread's own 16-byte
// slots of a raw slice buffer (chunk it at (it * 128 + c) * 16), zero-filled outside the
// grid and beyond ncol.  cp.async keeps GT_D slices in flight without holding registers.
__device__ __forceinline__ void copy_slice(const GtcArgs& a, int g, int ct, int q, int c, unsigned char* raw) {
    const int brick = a.grp[g].x;
    const int bx = brick % a.nbx, by = (brick / a.nbx) % a.nby, bz = brick / (a.nbx * a.nby);
    const int z = 4 * bz + (q >> 1);
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int j = it * 128 + c;
        const int n = j >> 3, ch = j & 7;
        const int x = 8 * bx + 4 * (ch & 1), y = 8 * by + 4 * (q & 1) + (ch >> 1);
        const int col = ct * GT_M + n;
        const bool in = x < a.n1 && y < a.n2 && z < a.n3 && col < a.ncol;
        const float* src = in ? a.X + (size_t)col * a.ld + x + (size_t)a.n1 * (y + (size_t)a.n2 * z) : a.X;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr(raw + (size_t)j * 16)), "l"(src),
                     "r"(in ? 16 : 0) : "memory");
    }
}

__global__ void __launch_bounds__(GT_THREADS, 1)
k_gather_tc(GtcArgs a) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[GT_S], lo_bar[GT_S], empty_bar[GT_S], tfull_bar[2], tempty_bar[2],
        done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    __shared__ int issued_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nu = (a.nunits - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;   // units of this CTA

    if (threadIdx.x == 0) {
        abort_flag = 0;
        issued_sh = 0;
        for (int s = 0; s < GT_S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&lo_bar[s], 128);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], 128);
        }
        mbar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(GT_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // value slices (hi and lo) by bulk copies
            int i = 0;
            for (int uu = 0; uu < nu && !abort_flag; ++uu) {
                const int u = (int)blockIdx.x + uu * (int)gridDim.x;
                const int4 G = a.grp[u / a.ctiles];
                const uint32_t vb = (uint32_t)G.z * GT_K * 4;
                bool stop = false;
                for (int q = 0; q < GT_SLICES; ++q, ++i) {
                    const int s = i % GT_S;
                    if (i >= GT_S && !mbar_wait(&empty_bar[s], ((i / GT_S) - 1) & 1, &abort_flag)) { stop = true; break; }
                    unsigned char* st = ring + (size_t)s * GT_STAGE;
                    mbar_expect_tx(&full_bar[s], 2 * vb);
                    const size_t off = (size_t)G.y + (size_t)q * GT_K * G.z;
                    bulk_load(st + 2 * GT_XB, a.vhi + off, vb, &full_bar[s]);
                    bulk_load(st + 2 * GT_XB + GT_BB, a.vlo + off, vb, &full_bar[s]);
                    issued_sh = i + 1;
                }
                if (stop) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int i = 0;
            for (int uu = 0; uu < nu && !abort_flag; ++uu) {
                const int u = (int)blockIdx.x + uu * (int)gridDim.x;
                const int4 G = a.grp[u / a.ctiles];
                const int buf = uu & 1;
                // the accumulator's previous unit must have been read out
                if (uu >= 2 && !mbar_wait(&tempty_bar[buf], ((uu >> 1) - 1) & 1, &abort_flag)) break;
                tc_fence_after();
                const uint32_t idesc = instr_desc_tf32(GT_M, G.z);
                const uint32_t dcol = tmem + (uint32_t)(2 * buf * GT_NP);      // hi * hi
                const uint32_t ccol = dcol + (uint32_t)GT_NP;                  // hi * lo + lo * hi
                bool stop = false;
                for (int q = 0; q < GT_SLICES; ++q, ++i) {
                    const int s = i % GT_S;
                    if (!mbar_wait(&full_bar[s], (i / GT_S) & 1, &abort_flag) ||
                        !mbar_wait(&lo_bar[s], (i / GT_S) & 1, &abort_flag)) { stop = true; break; }
                    tc_fence_after();
                    unsigned char* st = ring + (size_t)s * GT_STAGE;
                    const uint64_t ah = smem_desc(st), al = smem_desc(st + GT_XB);
                    const uint64_t bh = smem_desc(st + 2 * GT_XB), bl = smem_desc(st + 2 * GT_XB + GT_BB);
#pragma unroll
                    for (int kk = 0; kk < GT_K / 8; ++kk) {
                        const uint64_t ko = (uint64_t)(kk * 32) >> 4;     // 8 TF32 = 32 bytes along a row
                        const uint32_t acc = (q > 0 || kk > 0) ? 1u : 0u;
                        mma_tf32(dcol, ah + ko, bh + ko, idesc, acc);
                        mma_tf32(ccol, ah + ko, bl + ko, idesc, acc);
                        mma_tf32(ccol, al + ko, bh + ko, idesc, 1u);
                    }
                    mma_commit(&empty_bar[s]);          // stage free once these MMAs complete
                }
                if (stop) break;
                mma_commit(&tfull_bar[buf]);            // the unit's product is complete
            }
            mma_commit(&done_bar);                      // every MMA issued by this thread
        }
    } else if (warp < 6) {
        // warps 2-5: X slices into the stages (hi and lo), slice after slice over the units:
        // slice i's raw copy was issued GT_D - 1 slices earlier into raw buffer i % GT_D; the
        // thread reads back only its own chunks, so its cp.async wait is the only sync needed.
        // Waits on the stages are decided per warp (all lanes leave together).
        const int c = threadIdx.x - 64;
        unsigned char* raw = ring + (size_t)GT_S * GT_STAGE;
        const int nsl = nu * GT_SLICES;
        auto issue = [&](int i) {
            if (i < nsl) {
                const int u = (int)blockIdx.x + (i / GT_SLICES) * (int)gridDim.x;
                copy_slice(a, u / a.ctiles, u % a.ctiles, i % GT_SLICES, c, raw + (size_t)(i % GT_D) * GT_XB);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");     // one group per slice, empty or not
        };
        for (int i = 0; i < GT_D - 1; ++i) issue(i);
        for (int i = 0; i < nsl; ++i) {
            issue(i + GT_D - 1);
            const int s = i % GT_S;
            const bool ok = i < GT_S || mbar_wait(&empty_bar[s], ((i / GT_S) - 1) & 1, &abort_flag);
            if (__any_sync(0xffffffffu, !ok)) break;
            asm volatile("cp.async.wait_group %0;" ::"n"(GT_D - 1) : "memory");   // slice i has landed
            const unsigned char* rs = raw + (size_t)(i % GT_D) * GT_XB;
            unsigned char* xs = ring + (size_t)s * GT_STAGE;
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                const int j = it * 128 + c;
                const int n = j >> 3, ch = j & 7;
                const uint32_t off = (uint32_t)n * 128 + ((uint32_t)(ch ^ (n & 7)) << 4);
                const uint4 v = *reinterpret_cast<const uint4*>(rs + (size_t)j * 16);
                *reinterpret_cast<uint4*>(xs + off) = make_uint4(split_hi(v.x), split_hi(v.y), split_hi(v.z),
                                                                split_hi(v.w));
                *reinterpret_cast<uint4*>(xs + GT_XB + off) =
                    make_uint4(split_lo(v.x), split_lo(v.y), split_lo(v.z), split_lo(v.w));
            }
            fence_proxy_async();
            mbar_arrive(&lo_bar[s]);
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");        // no copy outlives the CTA
    } else {
        // warps 6-9: each unit's partial rows from its accumulator while the converters and
        // the MMAs go on with the next unit; warp w reads TMEM lanes 32 (w % 4) .. + 31
        const int quad = warp & 3;
        const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
        const int row = 32 * quad + lane;
        for (int uu = 0; uu < nu; ++uu) {
            const int u = (int)blockIdx.x + uu * (int)gridDim.x;
            const int e = u / a.ctiles, ct = u - e * a.ctiles;
            const int buf = uu & 1;
            const bool ok = mbar_wait(&tfull_bar[buf], (uu >> 1) & 1, &abort_flag);
            if (__any_sync(0xffffffffu, !ok)) break;
            tc_fence_after();
            const int4 G = a.grp[e];
            const int col = ct * GT_M + row;
            for (int c0 = 0; c0 < G.z; c0 += 16) {
                float v[16], w[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(2 * buf * GT_NP + c0), v);
                tmem_ld16(tmem + lane_base + (uint32_t)(2 * buf * GT_NP + GT_NP + c0), w);
                const int4* gr = reinterpret_cast<const int4*>(a.grow + G.w + c0);   // 16 slots
                int r[16];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int4 q4 = gr[k];
                    r[4 * k] = q4.x; r[4 * k + 1] = q4.y; r[4 * k + 2] = q4.z; r[4 * k + 3] = q4.w;
                }
                if (col < a.ncol) {
#pragma unroll
                    for (int f = 0; f < 16; ++f)
                        if (r[f] >= 0) a.part[(size_t)r[f] * a.ncol + col] = v[f] + w[f];
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty_bar[buf]);
        }
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0) {
        // TMEM must outlive every MMA issued; the copies in flight must land before the CTA's
        // shared memory goes away
        if (!mbar_drain(&done_bar, 0)) abort_flag = 1;
        if (abort_flag) {
            atomicExch(a.flags + FLAG_TIMEOUT, 1);
            const int issued = issued_sh;
            for (int j = issued > GT_S ? issued - GT_S : 0; j < issued; ++j) mbar_drain(&full_bar[j % GT_S], (j / GT_S) & 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GT_TMEM_COLS) : "memory");
    }
}

// tensor-core values of every group from the SIMT brick values: group g's block holds, per
// slice q of 32 points, NP rows of 128 bytes (row r = function slot r, zero for padding),
// point kk of the slice in 16-byte chunk kk / 4 XOR (r % 8), split TF32 hi + lo; slot r takes
// its values from the SIMT brick values at src[first slot + r] (-1: padding)
__global__ void k_fill_tc(const int4* __restrict__ grp, const int* __restrict__ src, const float* __restrict__ phi,
                          float* __restrict__ vhi, float* __restrict__ vlo) {
    const int4 G = grp[blockIdx.x];
    const int np = G.z;
    const int n = np * BRP;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int q = t / (np * GT_K);
        const int r = (t / GT_K) % np;
        const int kk = t % GT_K;
        const int k = q * GT_K + kk;
        const int o = src[G.w + r];
        const float v = o >= 0 ? phi[(size_t)o + brick_slot(k)] : 0.f;
        const uint32_t u = __float_as_uint(v);
        const size_t dst = (size_t)G.y + (size_t)q * GT_K * np + (size_t)r * GT_K + ((((kk >> 2) ^ (r & 7)) << 2) | (kk & 3));
        vhi[dst] = __uint_as_float(split_hi(u));
        vlo[dst] = __uint_as_float(split_lo(u));
    }
}

// ---------------------------------------------------------------------------- scatter
// Y[g(p), n] += alpha sum_f phi_f(p) W[frow(f), n] per brick: one unit per (brick, 128-orbital
// tile) holds every entry of the brick (so one unit writes each Y element it touches), its
// functions concatenated and padded to chunks of 32.  Per chunk:
// A = the values [128 points x 32 functions] of each half of the brick (table layout, bulk
// copies), B = W^T [128 orbitals x 32 functions] gathered from W's rows and split hi / lo by
// four builder warps, and D_half[128 points x 128 orbitals] += A_hi B_hi + A_hi B_lo +
// A_lo B_hi in TMEM (one accumulator per half; the correction terms ride in it: an error of
// the projector term far below the float H bound).  Four epilogue warps read D 16 orbitals
// at a time, write alpha D into a shared tile [16 orbitals][256 points] (the layout of a
// tensor-map box of 8 x 8 x 4 points x 16 orbitals of Y) and one thread adds the tile to Y
// with a TMA reduce-add (the read-modify-write of Y happens in L2; out-of-grid points and
// orbitals beyond ncol are clipped by the tensor map), two tiles alternating, while the MMAs
// of the next unit run in the other TMEM accumulator.
constexpr int ST_KC = 32;                          // functions per chunk
constexpr int ST_AB = 2 * GT_M * ST_KC * 4;        // 32 KB: values of both halves for one chunk
constexpr int ST_BB = GT_M * ST_KC * 4;            // 16 KB: one W^T chunk
constexpr int ST_STAGE = 2 * ST_AB + 2 * ST_BB;    // values hi, lo; W^T hi, lo
constexpr int ST_S = 2;
constexpr int ST_EO = 16;                          // orbitals per epilogue tile
constexpr int ST_EB = ST_EO * BRP * 4;             // 16 KB epilogue tile
constexpr size_t ST_SMEM = (size_t)ST_S * ST_STAGE + 2 * ST_EB + 1024;
constexpr uint32_t ST_TMEM_COLS = 512;             // two units x two halves x 128 orbitals
constexpr int ST_THREADS = 320;                    // load, MMA, 4 builder and 4 epilogue warps

struct StcArgs {
    float* Y;
    long ld;
    const int4* sbrick;   // per used brick: brick, float offset of its values, function slots
                          // K (a multiple of 32), functions (K without the padding)
    const int* sfrow;     // per function slot (value offset / 256): row of W, or -1
    const float* vhi;
    const float* vlo;
    const float* W;       // [nproj x ncol]
    float alpha;
    const double* alpha_dev;
    int ncol, n1, n2, n3, nbx, nby, nbricks, ctiles;
    int* flags;
};

__global__ void __launch_bounds__(ST_THREADS, 1)
k_scatter_tc(const __grid_constant__ CUtensorMap ymap, StcArgs a) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[ST_S], lo_bar[ST_S], empty_bar[ST_S], tfull_bar[2], tempty_bar[2],
        done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    __shared__ int issued_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // units of this CTA: its bricks blockIdx.x, + gridDim.x, ..., each with its orbital tiles
    // one after another (the brick's values, read from memory for the first tile, come from
    // L2 for the others)
    const int nu = (a.nbricks - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x * a.ctiles;
    auto brick_of = [&](int uu) { return (int)blockIdx.x + (uu / a.ctiles) * (int)gridDim.x; };
    const float alpha = a.alpha_dev ? (float)a.alpha_dev[0] : a.alpha;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        issued_sh = 0;
        for (int s = 0; s < ST_S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&lo_bar[s], 128);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], 128);
        }
        mbar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(ST_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int i = 0;
            for (int uu = 0; uu < nu && !abort_flag; ++uu) {
                const int4 B = a.sbrick[brick_of(uu)];
                bool stop = false;
                for (int c = 0; c < B.z / ST_KC; ++c, ++i) {
                    const int s = i % ST_S;
                    if (i >= ST_S && !mbar_wait(&empty_bar[s], ((i / ST_S) - 1) & 1, &abort_flag)) { stop = true; break; }
                    unsigned char* st = ring + (size_t)s * ST_STAGE;
                    mbar_expect_tx(&full_bar[s], 2 * ST_AB);
                    const size_t off = (size_t)B.y + (size_t)c * (ST_AB / 4);
                    bulk_load(st, a.vhi + off, ST_AB, &full_bar[s]);
                    bulk_load(st + ST_AB, a.vlo + off, ST_AB, &full_bar[s]);
                    issued_sh = i + 1;
                }
                if (stop) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc_tf32(GT_M, GT_M);
            int i = 0;
            for (int uu = 0; uu < nu && !abort_flag; ++uu) {
                const int4 B = a.sbrick[brick_of(uu)];
                const int buf = uu & 1;
                if (uu >= 2 && !mbar_wait(&tempty_bar[buf], ((uu >> 1) - 1) & 1, &abort_flag)) break;
                tc_fence_after();
                bool stop = false;
                for (int c = 0; c < B.z / ST_KC; ++c, ++i) {
                    const int s = i % ST_S;
                    if (!mbar_wait(&full_bar[s], (i / ST_S) & 1, &abort_flag) ||
                        !mbar_wait(&lo_bar[s], (i / ST_S) & 1, &abort_flag)) { stop = true; break; }
                    tc_fence_after();
                    unsigned char* st = ring + (size_t)s * ST_STAGE;
                    const int kval = B.w - c * ST_KC;           // functions of this chunk
                    const uint64_t bh = smem_desc(st + 2 * ST_AB), bl = smem_desc(st + 2 * ST_AB + ST_BB);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t dcol = tmem + (uint32_t)(buf * 256 + h * GT_M);
                        const uint64_t ah = smem_desc(st + h * (ST_AB / 2)), al = smem_desc(st + ST_AB + h * (ST_AB / 2));
#pragma unroll
                        for (int kk = 0; kk < ST_KC / 8; ++kk) {
                            if (kk * 8 >= kval) break;      // padding slots of the last chunk: zeros
                            const uint64_t ko = (uint64_t)(kk * 32) >> 4;
                            mma_tf32(dcol, ah + ko, bh + ko, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                            mma_tf32(dcol, ah + ko, bl + ko, idesc, 1u);
                            mma_tf32(dcol, al + ko, bh + ko, idesc, 1u);
                        }
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (stop) break;
                mma_commit(&tfull_bar[buf]);
            }
            mma_commit(&done_bar);
        }
    } else if (warp < 6) {
        // builders: W^T chunks, split hi / lo.  The W values of the next chunk are loaded
        // (32 independent loads per thread) before the wait for this chunk's stage, so their
        // latency overlaps the wait and the stores.
        const int t = threadIdx.x - 64;                 // orbital row of the W^T tile
        auto load = [&](int uu, int c, float (&v)[ST_KC]) {
            const int bi = brick_of(uu), ct = uu % a.ctiles;
            const int4 B = a.sbrick[bi];
            const int col = ct * GT_M + t;
            const int4* fr = reinterpret_cast<const int4*>(a.sfrow + (size_t)B.y / BRP + (size_t)c * ST_KC);
#pragma unroll
            for (int f4 = 0; f4 < ST_KC / 4; ++f4) {
                const int4 r = fr[f4];
                const bool cin = col < a.ncol;
                v[4 * f4 + 0] = (r.x >= 0 && cin) ? a.W[(size_t)r.x * a.ncol + col] : 0.f;
                v[4 * f4 + 1] = (r.y >= 0 && cin) ? a.W[(size_t)r.y * a.ncol + col] : 0.f;
                v[4 * f4 + 2] = (r.z >= 0 && cin) ? a.W[(size_t)r.z * a.ncol + col] : 0.f;
                v[4 * f4 + 3] = (r.w >= 0 && cin) ? a.W[(size_t)r.w * a.ncol + col] : 0.f;
            }
        };
        auto nchunks = [&](int uu) { return a.sbrick[brick_of(uu)].z / ST_KC; };
        if (nu > 0) {
            float cur[ST_KC], nxt[ST_KC];
            int uu = 0, c = 0, i = 0;
            load(0, 0, cur);
            while (true) {
                int nuu = uu, nc = c + 1;
                if (nc == nchunks(uu)) { nuu = uu + 1; nc = 0; }
                const bool more = nuu < nu;
                if (more) load(nuu, nc, nxt);
                const int s = i % ST_S;
                const bool ok = i < ST_S || mbar_wait(&empty_bar[s], ((i / ST_S) - 1) & 1, &abort_flag);
                if (__any_sync(0xffffffffu, !ok)) break;
                unsigned char* st = ring + (size_t)s * ST_STAGE + 2 * ST_AB;
#pragma unroll
                for (int f4 = 0; f4 < ST_KC / 4; ++f4) {
                    const uint32_t v0 = __float_as_uint(cur[4 * f4]), v1 = __float_as_uint(cur[4 * f4 + 1]);
                    const uint32_t v2 = __float_as_uint(cur[4 * f4 + 2]), v3 = __float_as_uint(cur[4 * f4 + 3]);
                    const uint32_t off = (uint32_t)t * 128 + ((uint32_t)(f4 ^ (t & 7)) << 4);
                    *reinterpret_cast<uint4*>(st + off) = make_uint4(split_hi(v0), split_hi(v1), split_hi(v2), split_hi(v3));
                    *reinterpret_cast<uint4*>(st + ST_BB + off) =
                        make_uint4(split_lo(v0), split_lo(v1), split_lo(v2), split_lo(v3));
                }
                fence_proxy_async();
                mbar_arrive(&lo_bar[s]);
                ++i;
                if (!more) break;
#pragma unroll
                for (int k = 0; k < ST_KC; ++k) cur[k] = nxt[k];
                uu = nuu;
                c = nc;
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (points of a half)
        const int t = threadIdx.x - 192;
        const int quad = warp & 3;
        const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
        const int prow = 32 * quad + lane;
        float* tiles = reinterpret_cast<float*>(ring + (size_t)ST_S * ST_STAGE);   // 2 x [16 orbitals][256 points]
        int ep = 0;                                     // tiles written so far
        for (int uu = 0; uu < nu; ++uu) {
            const int bi = brick_of(uu), ct = uu % a.ctiles;
            const int4 B = a.sbrick[bi];
            const int buf = uu & 1;
            // the four epilogue warps go on or stop together (they share named barrier 1, which
            // has no time limit): barrier 1 with an AND of every thread's wait result
            const uint32_t mine = mbar_wait(&tfull_bar[buf], (uu >> 1) & 1, &abort_flag) ? 1u : 0u;
            uint32_t all;
            asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 128, p;\n"
                         " selp.u32 %0, 1, 0, q;\n}" : "=r"(all) : "r"(mine) : "memory");
            if (!all) break;
            tc_fence_after();
            const int bx = B.x % a.nbx, by = (B.x / a.nbx) % a.nby, bz = B.x / (a.nbx * a.nby);
            for (int o0 = 0; B.z > 0 && o0 < GT_M && ct * GT_M + o0 < a.ncol; o0 += ST_EO, ++ep) {
                float v0[16], v1[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(buf * 256 + o0), v0);
                tmem_ld16(tmem + lane_base + (uint32_t)(buf * 256 + GT_M + o0), v1);
                float* tile = tiles + (ep & 1) * (ST_EO * BRP);
                // the tile's previous reduce (two tiles back) has finished reading it
                if (t == 0) bulk_wait_read<1>();
                asm volatile("bar.sync 1, 128;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    tile[q * BRP + prow] = alpha * v0[q];
                    tile[q * BRP + GT_M + prow] = alpha * v1[q];
                }
                fence_proxy_async();
                asm volatile("bar.sync 1, 128;" ::: "memory");      // the tile is complete
                if (t == 0) {
                    tma_reduce_add_4d(&ymap, tile, 8 * bx, 8 * by, 4 * bz, ct * GT_M + o0);
                    bulk_commit();
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty_bar[buf]);
        }
        if (t == 0) bulk_wait_all();
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_drain(&done_bar, 0)) abort_flag = 1;
        if (abort_flag) {
            atomicExch(a.flags + FLAG_TIMEOUT, 1);
            const int issued = issued_sh;
            for (int j = issued > ST_S ? issued - ST_S : 0; j < issued; ++j) mbar_drain(&full_bar[j % ST_S], (j / ST_S) & 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ST_TMEM_COLS) : "memory");
    }
}

// scatter values of every used brick: per 32-slot chunk and brick half, 128 rows (points) of
// 32 functions, 16-byte chunk k / 4 of row p stored at chunk (k / 4) XOR (p % 8); slot k of
// the brick takes its value offset from src (-1: padding)
__global__ void k_fill_tcs(const int4* __restrict__ sbrick, const int* __restrict__ ssrc, const float* __restrict__ phi,
                           float* __restrict__ vhi, float* __restrict__ vlo) {
    const int4 B = sbrick[blockIdx.x];
    const int n = B.z * BRP;
    const int* src = ssrc + (size_t)B.y / BRP;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int k = e / BRP, p = e % BRP;
        const int o = src[k];
        const float v = o >= 0 ? phi[(size_t)o + brick_slot(p)] : 0.f;
        const int c = k / ST_KC, kf = k % ST_KC, h = p / GT_M, row = p % GT_M;
        const size_t dst = (size_t)B.y + ((size_t)(c * 2 + h) * GT_M + row) * ST_KC +
                           ((((kf >> 2) ^ (row & 7)) << 2) | (kf & 3));
        const uint32_t u = __float_as_uint(v);
        vhi[dst] = __uint_as_float(split_hi(u));
        vlo[dst] = __uint_as_float(split_lo(u));
    }
}

}  // namespace

int build_tc_tables(hub_t h, Table& t) {
    t.tc = 0;
    if (!t.dense || h->n1 % 4 != 0 || t.nbent == 0) return HUB_OK;
    std::vector<int4> bent(t.nbent);
    HUB_CUDA_TRY(h, cudaMemcpy(bent.data(), t.d_bent, bent.size() * sizeof(int4), cudaMemcpyDeviceToHost));
    std::vector<int> bfirst(t.nbused + 1), frow(t.npart_rows);
    HUB_CUDA_TRY(h, cudaMemcpy(bfirst.data(), t.d_bfirst, bfirst.size() * sizeof(int), cudaMemcpyDeviceToHost));
    HUB_CUDA_TRY(h, cudaMemcpy(frow.data(), t.d_frow, frow.size() * sizeof(int), cudaMemcpyDeviceToHost));
    // gather groups: the entries of each used brick packed in order into groups of at most
    // GT_NP functions; per function slot its value offset and its partial row
    std::vector<int4> grp;
    std::vector<int> gsrc, grow;
    size_t off = 0;
    for (int bi = 0; bi < t.nbused; ++bi) {
        int e = bfirst[bi];
        while (e < bfirst[bi + 1]) {
            if (bent[e].y > GT_NP) return HUB_OK;            // keep the SIMT forms
            const int first = (int)gsrc.size();
            int nf = 0;
            for (; e < bfirst[bi + 1] && nf + bent[e].y <= GT_NP; ++e) {
                for (int f = 0; f < bent[e].y; ++f) {
                    gsrc.push_back(bent[e].z + f * BRP);
                    grow.push_back(bent[e].w + f);
                }
                nf += bent[e].y;
            }
            const int np = std::max(16, (nf + 15) / 16 * 16);
            for (int f = nf; f < np; ++f) {
                gsrc.push_back(-1);
                grow.push_back(-1);
            }
            grp.push_back(make_int4(bent[bfirst[bi]].x, (int)off, np, first));
            off += (size_t)np * BRP;
            if (off >= (1ull << 31)) return HUB_OK;          // keep the SIMT forms
        }
    }
    t.ntcg = (int)grp.size();
    int* d_gsrc = nullptr;
    HUB_CUDA_TRY(h, cudaMalloc((void**)&t.d_tcg, grp.size() * sizeof(int4)));
    HUB_CUDA_TRY(h, cudaMemcpy(t.d_tcg, grp.data(), grp.size() * sizeof(int4), cudaMemcpyHostToDevice));
    HUB_CUDA_TRY(h, cudaMalloc((void**)&t.d_tcg_row, grow.size() * sizeof(int)));
    HUB_CUDA_TRY(h, cudaMemcpy(t.d_tcg_row, grow.data(), grow.size() * sizeof(int), cudaMemcpyHostToDevice));
    HUB_CUDA_TRY(h, cudaMalloc((void**)&d_gsrc, gsrc.size() * sizeof(int)));
    HUB_CUDA_TRY(h, cudaMemcpy(d_gsrc, gsrc.data(), gsrc.size() * sizeof(int), cudaMemcpyHostToDevice));
    HUB_CUDA_TRY(h, cudaMalloc((void**)&t.d_tchi, off * sizeof(float)));
    HUB_CUDA_TRY(h, cudaMalloc((void**)&t.d_tclo, off * sizeof(float)));
    {
        ProfScope ps(h, HUB_K_TABLE);
        k_fill_tc<<<t.ntcg, 256, 0, h->stream>>>(t.d_tcg, d_gsrc, t.d_phi, t.d_tchi, t.d_tclo);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    cudaFree(d_gsrc);
    // scatter tables: per used brick the functions of its entries one after another in
    // function slots, the brick's count padded to a multiple of 32 (an entry holds 4 to 14
    // functions: padding each entry to 32 would more than double the MMA work)
    std::vector<int4> sbrick(t.nbused);
    std::vector<int> sfrow, ssrc;
    size_t soff = 0;
    for (int bi = 0; bi < t.nbused; ++bi) {
        int K = 0;
        for (int e = bfirst[bi]; e < bfirst[bi + 1]; ++e) {
            const int4& E = bent[e];
            for (int f = 0; f < E.y; ++f) {
                sfrow.push_back(frow[E.w + f]);
                ssrc.push_back(E.z + f * BRP);
            }
            K += E.y;
        }
        const int Kreal = K;
        for (; K % ST_KC != 0; ++K) {
            sfrow.push_back(-1);
            ssrc.push_back(-1);
        }
        sbrick[bi] = make_int4(bent[bfirst[bi]].x, (int)soff, K, Kreal);
        soff += (size_t)K * BRP;
        if (soff >= (1ull << 31)) return HUB_OK;          // keep the SIMT scatter
    }
    int* d_ssrc = nullptr;
    HUB_CUDA_TRY(h, cudaMalloc((void**)&t.d_tcs_brick, sbrick.size() * sizeof(int4)));
    HUB_CUDA_TRY(h, cudaMemcpy(t.d_tcs_brick, sbrick.data(), sbrick.size() * sizeof(int4), cudaMemcpyHostToDevice));
    HUB_CUDA_TRY(h, cudaMalloc((void**)&t.d_tcs_frow, sfrow.size() * sizeof(int)));
    HUB_CUDA_TRY(h, cudaMemcpy(t.d_tcs_frow, sfrow.data(), sfrow.size() * sizeof(int), cudaMemcpyHostToDevice));
    HUB_CUDA_TRY(h, cudaMalloc((void**)&d_ssrc, ssrc.size() * sizeof(int)));
    HUB_CUDA_TRY(h, cudaMemcpy(d_ssrc, ssrc.data(), ssrc.size() * sizeof(int), cudaMemcpyHostToDevice));
    HUB_CUDA_TRY(h, cudaMalloc((void**)&t.d_tcs_hi, soff * sizeof(float)));
    HUB_CUDA_TRY(h, cudaMalloc((void**)&t.d_tcs_lo, soff * sizeof(float)));
    {
        ProfScope ps(h, HUB_K_TABLE);
        k_fill_tcs<<<t.nbused, 256, 0, h->stream>>>(t.d_tcs_brick, d_ssrc, t.d_phi, t.d_tcs_hi, t.d_tcs_lo);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    cudaFree(d_ssrc);
    t.tc = 1;
    return HUB_OK;
}

int launch_gather_tc(hub_t h, const void* X, int ncol, int ld) {
    Table& t = h->proj;
    if (!t.tc) return fail(h, HUB_EINVAL, "no tensor-core brick tables (n1 must be a multiple of 4)");
    if ((uintptr_t)X % 16 != 0 || ld % 4 != 0) return fail(h, HUB_EINVAL, "tensor-core gather: block not 16-byte aligned");
    if (ncol == 0) return HUB_OK;
    GtcArgs a{};
    a.X = (const float*)X;
    a.grp = t.d_tcg;
    a.grow = t.d_tcg_row;
    a.vhi = t.d_tchi;
    a.vlo = t.d_tclo;
    a.part = (float*)h->d_part;
    a.ld = ld;
    a.n1 = h->n1;
    a.n2 = h->n2;
    a.n3 = h->n3;
    a.ncol = ncol;
    a.nbx = t.nbx;
    a.nby = t.nby;
    a.ctiles = (ncol + GT_M - 1) / GT_M;
    a.nunits = t.ntcg * a.ctiles;
    a.flags = h->d_flags;
    const int grid = std::max(1, std::min(a.nunits, h->num_sms));
    HUB_CUDA_TRY(h, cudaFuncSetAttribute(k_gather_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GT_SMEM));
    ProfScope ps(h, HUB_K_GATHER);
    k_gather_tc<<<grid, GT_THREADS, GT_SMEM, h->stream>>>(a);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int launch_scatter_tc(hub_t h, void* Y, int ncol, int ld, double alpha, const double* alpha_dev) {
    Table& t = h->proj;
    if (!t.tc) return fail(h, HUB_EINVAL, "no tensor-core brick tables (n1 must be a multiple of 4)");
    if (ncol == 0 || t.nbused == 0) return HUB_OK;
    StcArgs a{};
    a.Y = (float*)Y;
    a.ld = ld;
    a.sbrick = t.d_tcs_brick;
    a.sfrow = t.d_tcs_frow;
    a.vhi = t.d_tcs_hi;
    a.vlo = t.d_tcs_lo;
    a.W = (const float*)h->d_W;
    a.alpha = (float)alpha;
    a.alpha_dev = alpha_dev;
    a.ncol = ncol;
    a.n1 = h->n1;
    a.n2 = h->n2;
    a.n3 = h->n3;
    a.nbx = t.nbx;
    a.nby = t.nby;
    a.ctiles = (ncol + GT_M - 1) / GT_M;
    a.nbricks = t.nbused;
    a.flags = h->d_flags;
    // Y as a 4-D tensor (x, y, z, orbital) for the reduce-add of 8 x 8 x 4-point, 16-orbital
    // boxes: strides multiples of 16 bytes (n1 and ld multiples of 4), base 16-byte aligned
    if ((uintptr_t)Y % 16 != 0 || ld % 4 != 0 || h->n1 % 4 != 0)
        return fail(h, HUB_EINVAL, "tensor-core scatter: block not 16-byte aligned");
    PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    int rc;
    if ((rc = tensor_map_encoder(h, &enc))) return rc;
    CUtensorMap ymap;
    const cuuint64_t dims[4] = {(cuuint64_t)h->n1, (cuuint64_t)h->n2, (cuuint64_t)h->n3, (cuuint64_t)ncol};
    const cuuint64_t strides[3] = {(cuuint64_t)h->n1 * 4, (cuuint64_t)h->n1 * h->n2 * 4, (cuuint64_t)ld * 4};
    const cuuint32_t box[4] = {8, 8, 4, (cuuint32_t)ST_EO};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(&ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Y, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(h, HUB_ECUDA, "tensor-core scatter: cuTensorMapEncodeTiled failed");
    const int grid = std::max(1, std::min(a.nbricks, h->num_sms));
    HUB_CUDA_TRY(h, cudaFuncSetAttribute(k_scatter_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ST_SMEM));
    ProfScope ps(h, HUB_K_SCATTER);
    k_scatter_tc<<<grid, ST_THREADS, ST_SMEM, h->stream>>>(ymap, a);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

}  // namespace hub
