// Fused finite-difference stencil: Laplacian (2*n0-th order, Sec. II.B) + local potential
// + Chebyshev three-term recurrence update, with the Bloch-periodic index wrap.
//
//   Yout = alpha * (-1/2 Lap_h Y + V .* Y - shift * Y) + beta * Yprev
//
// Layout: Y[g + col*ld], g = x + n1*(y + n2*z).  One CTA owns a TX x TY tile of the x-y
// plane for one column and marches along z over a chunk of planes.
//
// Pipeline: shared memory holds a ring of S stages; stage p % S holds plane p of Y with an
// NH-wide x/y halo, plus the tile's interior of V and Yprev for that plane.  Stages are
// filled with cp.async P planes ahead of use, so HBM/L2 latency overlaps the arithmetic.
// Each thread owns a fixed list of halo slots whose in-plane offsets (wrapped into the cell)
// are computed once.  The z-neighbours of a thread's point live in a register queue of
// 2*NH+1 values fed from the ring, the x/y neighbours are read from the current stage.
// Slots that wrapped across a cell face get the Bloch factor exp(i k_a L_a)^wraps (only
// for complex elements; real Gamma-point data is copied untouched).  Yprev may alias Yout:
// each element is read (through the ring) before the same thread writes it.
#include <algorithm>
#include <cmath>

#include "hub_internal.cuh"
#include "cplx.cuh"

namespace hub {

template <typename R>
struct StencilDev {
    const void* Y;
    const void* Yprev;
    void* Yout;
    const R* V;
    int n1, n2, n3, ld;
    R w[3][6];
    R center, alpha, beta;    // float: centre without the kinetic part (difference form)
    double ph[3][2];
    int zchunk, nzc;
    // batched / graph form: when coef != nullptr the recurrence coefficients are read on the
    // device, coef = {alpha, beta, shift}, and w = alpha * wbase, centre = alpha * (cen_kin -
    // shift) (double) or alpha * (-shift) (float)
    const double* coef;
    R wbase[3][6];
    double cen_kin;
};

template <typename R>
struct Coef {
    R w[3][6];
    R center, alpha, beta;
};

template <typename R>
__device__ __forceinline__ Coef<R> resolve_coef(const StencilDev<R>& a) {
    Coef<R> c;
    if (a.coef) {
        const double al = a.coef[0], be = a.coef[1], sh = a.coef[2];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
#pragma unroll
            for (int p = 0; p < 6; ++p) c.w[ax][p] = (R)(al * (double)a.wbase[ax][p]);
        c.center = (R)(sizeof(R) == 4 ? al * (-sh) : al * (a.cen_kin - sh));
        c.alpha = (R)al;
        c.beta = (R)be;
    } else {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
#pragma unroll
            for (int p = 0; p < 6; ++p) c.w[ax][p] = a.w[ax][p];
        c.center = a.center;
        c.alpha = a.alpha;
        c.beta = a.beta;
    }
    return c;
}

// Rounded weights and the centre coefficient.  Double uses the summation form
//   c f0 + sum_p w_p (f+p + f-p),   c = alpha(-1/2 c0 sum h^-2 - shift).
// Float uses the difference form
//   alpha(-shift) f0 + sum_p w_p ((f+p + f-p) - 2 f0)
// whose terms are small for smooth orbitals: the large kinetic centre (~100 Ha at h = 0.2)
// never enters a partial sum, so rounding does not bias the Rayleigh quotients (with the
// summation form float rounding shifted every low eigenvalue by ~1e-5 ||H|| eps-scaled),
// and constants are annihilated for any rounded weights.
template <typename R>
static void fill_coefficients(const StencilArgs& s, StencilDev<R>& d) {
    double wsum = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int p = 0; p < 6; ++p) {
            const double w = p < s.n0 ? s.w[a][p] : 0.0;
            d.w[a][p] = (R)w;
            wsum += w;
        }
    // the kinetic centre is -2 sum w; the float form carries it inside the differences
    d.center = sizeof(R) == 4 ? (R)(s.center + 2.0 * wsum) : (R)s.center;
    d.alpha = (R)s.alpha;
    d.beta = (R)s.beta;
    d.coef = s.coef;
    double wb = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int p = 0; p < 6; ++p) {
            const double w = p < s.n0 ? s.wbase[a][p] : 0.0;
            d.wbase[a][p] = (R)w;
            wb += w;
        }
    d.cen_kin = -2.0 * wb;
}

__device__ __forceinline__ int floordiv(int a, int n) {
    int q = a / n;
    return (a % n != 0 && a < 0) ? q - 1 : q;
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename R, bool CPLX, int TX, int TY, int P>
struct StencilCfg {
    static constexpr int NH = 6;
    static constexpr int SX = TX + 2 * NH, SY = TY + 2 * NH;
    static constexpr int NT = TX * TY;
    static constexpr int S = P + 8;                       // ring stages
    static constexpr int SLOTS = SX * SY;
    static constexpr int PER = (SLOTS + NT - 1) / NT;     // halo'd slots per thread
    using T = typename VT<R, CPLX>::T;
    // stage layout: Y plane with halo, then interior V (R), then interior Yprev (T)
    static constexpr size_t YB = sizeof(T) * SLOTS;
    static constexpr size_t VB = sizeof(R) * NT;
    static constexpr size_t PB = sizeof(T) * NT;
    static constexpr size_t STAGE = ((YB + VB + PB + 127) / 128) * 128;
    static constexpr size_t SMEM = STAGE * S;
};

template <typename R, bool CPLX, int TX, int TY, int P>
__global__ void __launch_bounds__(TX * TY)
k_stencil(StencilDev<R> a) {
    const Coef<R> cf = resolve_coef(a);
    using C = StencilCfg<R, CPLX, TX, TY, P>;
    using T = typename C::T;
    constexpr int NH = C::NH, SX = C::SX, S = C::S, NT = C::NT, PER = C::PER;
    extern __shared__ __align__(128) unsigned char smem[];

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int col = blockIdx.z / a.nzc;
    const int zc = blockIdx.z - col * a.nzc;
    const int z0 = zc * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.n3);
    const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
    const long plane = (long)n1 * n2;
    const int gx0 = blockIdx.x * TX, gy0 = blockIdx.y * TY;

    const T* __restrict__ Y = reinterpret_cast<const T*>(a.Y) + (size_t)col * a.ld;
    const T* Yp = a.Yprev ? reinterpret_cast<const T*>(a.Yprev) + (size_t)col * a.ld : nullptr;
    T* Yo = reinterpret_cast<T*>(a.Yout) + (size_t)col * a.ld;

    // this thread's halo'd slots: shared index, wrapped in-plane offset, Bloch factor
    int s_idx[PER];
    int s_off[PER];
    T s_ph[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NT;
        s_idx[k] = -1;
        s_off[k] = 0;
        s_ph[k] = phase_pow<T>(1.0, 0.0, 0);
        if (i < C::SLOTS) {
            const int ix = i % SX, iy = i / SX;
            const int gx = gx0 - NH + ix, gy = gy0 - NH + iy;
            const int wx = floordiv(gx, n1), wy = floordiv(gy, n2);
            s_idx[k] = i;
            s_off[k] = (gy - wy * n2) * n1 + (gx - wx * n1);
            if constexpr (CPLX)
                s_ph[k] = cmul(phase_pow<T>(a.ph[0][0], a.ph[0][1], wx), phase_pow<T>(a.ph[1][0], a.ph[1][1], wy));
        }
    }
    const bool active = (gx0 + tx < n1) && (gy0 + ty < n2);
    const long own = (long)(gy0 + ty) * n1 + (gx0 + tx);

    auto stage_Y = [&](int p) { return reinterpret_cast<T*>(smem + C::STAGE * (size_t)(((p % S) + S) % S)); };
    auto stage_V = [&](int p) { return reinterpret_cast<R*>(reinterpret_cast<unsigned char*>(stage_Y(p)) + C::YB); };
    auto stage_P = [&](int p) { return reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(stage_Y(p)) + C::YB + C::VB); };

    // issue the copies of plane p (wrapped along z); interior V / Yprev only for planes
    // that will be computed
    auto issue = [&](int p) {
        const int wz = floordiv(p, n3);
        const long zoff = (long)(p - wz * n3) * plane;
        T* ys = stage_Y(p);
#pragma unroll
        for (int k = 0; k < PER; ++k)
            if (s_idx[k] >= 0) cp_async<sizeof(T)>(ys + s_idx[k], Y + zoff + s_off[k]);
        if (active && p >= z0 && p < z1) {
            cp_async<sizeof(R)>(stage_V(p) + tid, a.V + zoff + own);
            if (Yp) cp_async<sizeof(T)>(stage_P(p) + tid, Yp + zoff + own);
        }
    };
    // Bloch factors of this thread's wrapped slots of plane p (complex only)
    auto fix = [&](int p) {
        if constexpr (CPLX) {
            const T pz = phase_pow<T>(a.ph[2][0], a.ph[2][1], floordiv(p, n3));
            T* ys = stage_Y(p);
#pragma unroll
            for (int k = 0; k < PER; ++k)
                if (s_idx[k] >= 0) ys[s_idx[k]] = cmul(ys[s_idx[k]], cmul(s_ph[k], pz));
        }
    };

    // prologue: the z-queue of planes z0-NH .. z0+NH straight from global memory (active
    // threads own a point inside the cell, so only the z wrap carries a Bloch factor), and
    // ring planes z0 .. z0+NH+P in flight
    const int ctr = (ty + NH) * SX + (tx + NH);
    T q[2 * NH + 1];
#pragma unroll
    for (int j = 0; j < 2 * NH + 1; ++j) {
        q[j] = zero_of(T());
        if (active) {
            const int p = z0 - NH + j;
            const int wz = floordiv(p, n3);
            q[j] = Y[(long)(p - wz * n3) * plane + own];
            if constexpr (CPLX) q[j] = cmul(q[j], phase_pow<T>(a.ph[2][0], a.ph[2][1], wz));
        }
    }
    const int last_needed = z1 + NH - 1;      // highest plane any step reads
#pragma unroll 1
    for (int p = z0; p <= z0 + NH + P; ++p) {
        if (p <= last_needed) issue(p);
        cp_async_commit();
    }
    cp_async_wait<P>();                        // planes z0 .. z0+NH have landed
#pragma unroll 1
    for (int p = z0; p <= z0 + NH; ++p)
        if (p <= last_needed) fix(p);
    __syncthreads();

#pragma unroll 1
    for (int z = z0; z < z1; ++z) {
        if (active) {
            const T* ys = stage_Y(z);
            T acc = mulr(cf.center + cf.alpha * stage_V(z)[tid], q[NH]);
            const T c0 = q[NH];
#pragma unroll
            for (int p = 1; p <= NH; ++p) {
                T sz = add(q[NH + p], q[NH - p]);
                T sx = add(ys[ctr + p], ys[ctr - p]);
                T sy = add(ys[ctr + p * SX], ys[ctr - p * SX]);
                if constexpr (sizeof(R) == 4) {
                    sz = fmar((R)-2, c0, sz);
                    sx = fmar((R)-2, c0, sx);
                    sy = fmar((R)-2, c0, sy);
                }
                acc = fmar(cf.w[2][p - 1], sz, acc);
                acc = fmar(cf.w[0][p - 1], sx, acc);
                acc = fmar(cf.w[1][p - 1], sy, acc);
            }
            if (Yp) acc = fmar(cf.beta, stage_P(z)[tid], acc);
            Yo[(long)z * plane + own] = acc;
        }
        if (z + 1 == z1) break;
        __syncthreads();                       // every thread is done with stage z
        const int nxt = z + NH + 1 + P;         // reuses the stage of plane z - 1
        if (nxt <= last_needed) issue(nxt);
        cp_async_commit();
        cp_async_wait<P>();                    // plane z + NH + 1 has landed
        fix(z + NH + 1);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 2 * NH; ++j) q[j] = q[j + 1];
        q[2 * NH] = stage_Y(z + NH + 1)[ctr];
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------- vector form
// Same pipeline with VEC = 16 bytes / element consecutive x-points per thread: the halo'd
// plane is copied as 16-byte vectors (the x-halo is padded to HX, a multiple of VEC), the
// x-neighbours of a thread's VEC points come from (VEC + 2 HX) / VEC vector loads, each
// y-neighbour row from one vector load, and the z-queue holds vectors.  Requires
// n1 % VEC == 0, ld % VEC == 0 and 16-byte aligned blocks, so a vector never straddles
// a row end or a cell face (its VEC points share one Bloch factor).
template <typename T, int VEC>
struct alignas(sizeof(T) * VEC) VecT {      // natural size: 16 B for Y vectors, 8 B for a
    T v[VEC];                               // pair of float potentials
};

template <typename R, bool CPLX, int VEC, int TXT, int TY, int P>
struct VecCfg {
    static constexpr int NH = 6;
    static constexpr int HX = ((NH + VEC - 1) / VEC) * VEC;
    static constexpr int TXP = TXT * VEC;
    static constexpr int SXP = TXP + 2 * HX;
    static constexpr int SXV = SXP / VEC;                  // vectors per smem row
    static constexpr int SY = TY + 2 * NH;
    static constexpr int NT = TXT * TY;
    static constexpr int S = P + 8;
    static constexpr int NVS = SXV * SY;
    static constexpr int PER = (NVS + NT - 1) / NT;
    using T = typename VT<R, CPLX>::T;
    using V = VecT<T, VEC>;
    using VR = VecT<R, VEC>;
    static constexpr size_t YB = sizeof(T) * SXP * SY;
    static constexpr size_t VB = sizeof(R) * TXP * TY;
    static constexpr size_t PB = sizeof(T) * TXP * TY;
    static constexpr size_t STAGE = ((YB + VB + PB + 127) / 128) * 128;
    static constexpr size_t SMEM = STAGE * S;
};

template <typename R, bool CPLX, int VEC, int TXT, int TY, int P>
__global__ void __launch_bounds__(TXT * TY)
k_stencil_vec(StencilDev<R> a) {
    const Coef<R> cf = resolve_coef(a);
    using C = VecCfg<R, CPLX, VEC, TXT, TY, P>;
    static_assert(sizeof(typename C::V) == 16, "Y vectors are 16-byte copies");
    static_assert(sizeof(typename C::VR) == sizeof(R) * VEC, "potential vectors are unpadded");
    static_assert(C::YB % 16 == 0 && C::VB % 16 == 0, "stage regions stay 16-byte aligned");
    using T = typename C::T;
    using V = typename C::V;
    using VR = typename C::VR;
    constexpr int NH = C::NH, HX = C::HX, SXP = C::SXP, SXV = C::SXV, S = C::S, NT = C::NT, PER = C::PER;
    constexpr int NXV = (VEC + 2 * HX) / VEC;              // x-neighbour vectors per thread
    extern __shared__ __align__(128) unsigned char smem[];

    const int tid = threadIdx.x;
    const int tx = tid % TXT, ty = tid / TXT;
    const int col = blockIdx.z / a.nzc;
    const int zc = blockIdx.z - col * a.nzc;
    const int z0 = zc * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.n3);
    const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
    const long plane = (long)n1 * n2;
    const int gx0 = blockIdx.x * C::TXP, gy0 = blockIdx.y * TY;

    const T* __restrict__ Y = reinterpret_cast<const T*>(a.Y) + (size_t)col * a.ld;
    const T* Yp = a.Yprev ? reinterpret_cast<const T*>(a.Yprev) + (size_t)col * a.ld : nullptr;
    T* Yo = reinterpret_cast<T*>(a.Yout) + (size_t)col * a.ld;

    int s_idx[PER];                 // vector slot in the stage
    const T* s_src[PER];            // source of the slot in plane 0 (wrapped x/y)
    T s_ph[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NT;
        s_idx[k] = -1;
        s_src[k] = Y;
        s_ph[k] = phase_pow<T>(1.0, 0.0, 0);
        if (i < C::NVS) {
            const int cx = i % SXV, iy = i / SXV;
            const int gx = gx0 - HX + cx * VEC, gy = gy0 - NH + iy;
            const int wx = floordiv(gx, n1), wy = floordiv(gy, n2);
            s_idx[k] = i;
            s_src[k] = Y + (long)(gy - wy * n2) * n1 + (gx - wx * n1);
            if constexpr (CPLX)
                s_ph[k] = cmul(phase_pow<T>(a.ph[0][0], a.ph[0][1], wx), phase_pow<T>(a.ph[1][0], a.ph[1][1], wy));
        }
    }
    const bool active = (gx0 + tx * VEC < n1) && (gy0 + ty < n2);
    const long own = (long)(gy0 + ty) * n1 + (gx0 + tx * VEC);

    auto stY = [&](int st) { return reinterpret_cast<V*>(smem + C::STAGE * (size_t)st); };
    auto stV = [&](int st) { return reinterpret_cast<VR*>(smem + C::STAGE * (size_t)st + C::YB); };
    auto stP = [&](int st) { return reinterpret_cast<V*>(smem + C::STAGE * (size_t)st + C::YB + C::VB); };

    // copies of plane p (z index already wrapped to zw) into stage st
    auto issue = [&](int st, int zw, bool interior) {
        const long zoff = (long)zw * plane;
        V* ys = stY(st);
#pragma unroll
        for (int k = 0; k < PER; ++k)
            if (s_idx[k] >= 0) cp_async<16>(ys + s_idx[k], s_src[k] + zoff);
        if (active && interior) {
            cp_async<sizeof(VR)>(stV(st) + tid, a.V + zoff + own);
            if (Yp) cp_async<16>(stP(st) + tid, Yp + zoff + own);
        }
    };
    auto fix = [&](int st, int wz) {
        if constexpr (CPLX) {
            const T pz = phase_pow<T>(a.ph[2][0], a.ph[2][1], wz);
            V* ys = stY(st);
#pragma unroll
            for (int k = 0; k < PER; ++k)
                if (s_idx[k] >= 0) {
                    const T f = cmul(s_ph[k], pz);
                    V v = ys[s_idx[k]];
#pragma unroll
                    for (int e = 0; e < VEC; ++e) v.v[e] = cmul(v.v[e], f);
                    ys[s_idx[k]] = v;
                }
        }
    };

    const int last_needed = z1 + NH - 1;
    // z-queue of planes z0-NH .. z0+NH from global memory
    V q[2 * NH + 1];
#pragma unroll
    for (int j = 0; j < 2 * NH + 1; ++j) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) q[j].v[e] = zero_of(T());
        if (active) {
            const int p = z0 - NH + j;
            const int wz = floordiv(p, n3);
            q[j] = *reinterpret_cast<const V*>(Y + (long)(p - wz * n3) * plane + own);
            if constexpr (CPLX) {
                const T f = phase_pow<T>(a.ph[2][0], a.ph[2][1], wz);
#pragma unroll
                for (int e = 0; e < VEC; ++e) q[j].v[e] = cmul(q[j].v[e], f);
            }
        }
    }
    // ring: planes z0 .. z0+NH+P; issue cursor (plane, stage, wrapped z, wraps)
    int ip = z0, ist = 0, izw = z0 % n3, iwz = z0 / n3;
#pragma unroll 1
    for (int j = 0; j <= NH + P; ++j) {
        if (ip <= last_needed) issue(ist, izw, ip < z1);
        cp_async_commit();
        ++ip; if (++ist == S) ist = 0; if (++izw == n3) { izw = 0; ++iwz; }
    }
    cp_async_wait<P>();
    {
        int st = 0, zw = z0 % n3, wz = z0 / n3;
#pragma unroll 1
        for (int p = z0; p <= z0 + NH; ++p) {
            if (p <= last_needed) fix(st, wz);
            if (++st == S) st = 0;
            if (++zw == n3) { zw = 0; ++wz; }
        }
    }
    __syncthreads();
    // stage of plane z and of plane z + NH + 1, and the wrap count of plane z + NH + 1
    int sz = 0;
    int sf = (NH + 1) % S;
    int fwz = (z0 + NH + 1) / n3;
    int fzw = (z0 + NH + 1) % n3;
    constexpr int ctr_row = NH;                 // smem row of the thread's own y, minus ty
#pragma unroll 1
    for (int z = z0; z < z1; ++z) {
        if (active) {
            const V* ys = stY(sz);
            const int rbase = (ty + ctr_row) * SXV;          // vector index of the own row
            // own row: vectors covering x - HX .. x + VEC - 1 + HX
            T xr[VEC + 2 * HX];
#pragma unroll
            for (int j = 0; j < NXV; ++j) {
                const V v = ys[rbase + tx + j];
#pragma unroll
                for (int e = 0; e < VEC; ++e) xr[j * VEC + e] = v.v[e];
            }
            const VR vv = stV(sz)[tid];
            V pv;
            if (Yp) pv = stP(sz)[tid];
            V out;
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                T acc = mulr(cf.center + cf.alpha * vv.v[e], q[NH].v[e]);
                const T c0 = q[NH].v[e];
#pragma unroll
                for (int p = 1; p <= NH; ++p) {
                    T sz = add(q[NH + p].v[e], q[NH - p].v[e]);
                    T sx = add(xr[HX + e + p], xr[HX + e - p]);
                    if constexpr (sizeof(R) == 4) {
                        sz = fmar((R)-2, c0, sz);
                        sx = fmar((R)-2, c0, sx);
                    }
                    acc = fmar(cf.w[2][p - 1], sz, acc);
                    acc = fmar(cf.w[0][p - 1], sx, acc);
                }
                out.v[e] = acc;
            }
#pragma unroll
            for (int p = 1; p <= NH; ++p) {
                const V up = ys[rbase + p * SXV + tx + HX / VEC];
                const V dn = ys[rbase - p * SXV + tx + HX / VEC];
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    T sy = add(up.v[e], dn.v[e]);
                    if constexpr (sizeof(R) == 4) sy = fmar((R)-2, q[NH].v[e], sy);
                    out.v[e] = fmar(cf.w[1][p - 1], sy, out.v[e]);
                }
            }
            if (Yp) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) out.v[e] = fmar(cf.beta, pv.v[e], out.v[e]);
            }
            *reinterpret_cast<V*>(Yo + (long)z * plane + own) = out;
        }
        if (z + 1 == z1) break;
        __syncthreads();
        if (ip <= last_needed) issue(ist, izw, ip < z1);
        cp_async_commit();
        ++ip; if (++ist == S) ist = 0; if (++izw == n3) { izw = 0; ++iwz; }
        cp_async_wait<P>();
        fix(sf, fwz);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 2 * NH; ++j) q[j] = q[j + 1];
        q[2 * NH] = stY(sf)[(ty + ctr_row) * SXV + tx + HX / VEC];
        if (++sz == S) sz = 0;
        if (++sf == S) sf = 0;
        if (++fzw == n3) { fzw = 0; ++fwz; }
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------- packed float pairs
// Blackwell f32x2 instructions (add.rn.f32x2, fma.rn.f32x2, mul.rn.f32x2): two lanes of
// ordinary IEEE float arithmetic per instruction, the same rounding as scalar code.
typedef unsigned long long u64;
__device__ __forceinline__ u64 pk2(float a, float b) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float lo2(u64 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi2(u64 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---------------------------------------------------------------------------- float x4 form
// Real float, 4 consecutive x-points per thread held as two packed pairs, so that every add
// and FMA is one f32x2 instruction; the z-loop is unrolled 2*NH+1 times so that the
// register queue rotates by static indexing.  A stage holds the halo'd plane z only (the x/y
// neighbours), plus three per-thread interior slots: the plane z + NH + 1 that enters the
// z register queue after plane z, and V and Yprev of plane z.  Stages are filled PH planes
// ahead; with RS = PH + 2 stages the copy into a stage starts two planes after its last
// reader, so one barrier per plane suffices (the interior slots are written and read by the
// same thread and need none).  The three axes accumulate in separate registers (six
// independent FMA chains per thread instead of two).
template <int TXT, int TY, int PH>
struct SplitCfg {
    static constexpr int NH = 6, HX = 8;
    static constexpr int TXP = TXT * 4;
    static constexpr int SXV = (TXP + 2 * HX) / 4;     // float4 vectors per halo row
    static constexpr int SY = TY + 2 * NH;
    static constexpr int NT = TXT * TY;
    static constexpr int RS = PH + 2;
    static constexpr int NVS = SXV * SY;
    static constexpr int PER = (NVS + NT - 1) / NT;
    static constexpr size_t YB = 16 * (size_t)NVS;     // halo plane
    static constexpr size_t IB = 16 * (size_t)NT;      // one float4 per thread
    static constexpr size_t STAGE = YB + 3 * IB;       // halo | feed | V | Yprev
    static constexpr size_t SMEM = STAGE * RS;
};

template <int TXT, int TY, int PH>
__global__ void __launch_bounds__(TXT * TY)
k_stencil_f32s(StencilDev<float> a) {
    const Coef<float> cf = resolve_coef(a);
    using C = SplitCfg<TXT, TY, PH>;
    constexpr int NH = C::NH, HX = C::HX, SXV = C::SXV, RS = C::RS, NT = C::NT, PER = C::PER;
    constexpr int Q = 2 * NH + 1;
    static_assert(C::YB % 16 == 0 && C::STAGE % 16 == 0, "stage regions stay 16-byte aligned");
    extern __shared__ __align__(128) unsigned char smem[];

    const int tid = threadIdx.x;
    const int tx = tid % TXT, ty = tid / TXT;
    const int col = blockIdx.z / a.nzc;
    const int zc = blockIdx.z - col * a.nzc;
    const int z0 = zc * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.n3);
    const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
    const long plane = (long)n1 * n2;
    const int gx0 = blockIdx.x * C::TXP, gy0 = blockIdx.y * TY;

    const float* __restrict__ Y = reinterpret_cast<const float*>(a.Y) + (size_t)col * a.ld;
    const float* Yp = a.Yprev ? reinterpret_cast<const float*>(a.Yprev) + (size_t)col * a.ld : nullptr;
    float* Yo = reinterpret_cast<float*>(a.Yout) + (size_t)col * a.ld;

    int s_idx[PER];
    const float* s_src[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NT;
        s_idx[k] = -1;
        s_src[k] = Y;
        if (i < C::NVS) {
            const int cx = i % SXV, iy = i / SXV;
            const int gx = gx0 - HX + cx * 4, gy = gy0 - NH + iy;
            const int wx = floordiv(gx, n1), wy = floordiv(gy, n2);
            s_idx[k] = i;
            s_src[k] = Y + (long)(gy - wy * n2) * n1 + (gx - wx * n1);
        }
    }
    const bool active = (gx0 + tx * 4 < n1) && (gy0 + ty < n2);
    const long own = (long)(gy0 + ty) * n1 + (gx0 + tx * 4);

    auto stY = [&](int st) { return reinterpret_cast<ulonglong2*>(smem + C::STAGE * (size_t)st); };
    auto stI = [&](int st, int k) {            // k = 0 feed, 1 V, 2 Yprev
        return reinterpret_cast<ulonglong2*>(smem + C::STAGE * (size_t)st + C::YB + C::IB * (size_t)k);
    };
    // copy group j: halo, V and Yprev of plane z0 + j, and the queue feed plane z0 + j + NH + 1.
    // Groups are issued in order; the plane of the next group and the offsets of its planes
    // advance by additions (no multiply or modulo per plane).
    int ip = z0;                                // plane of the next group
    long ioff = (long)z0 * plane;               // its offset (ip < z1 <= n3: no wrap)
    int fz = z0 + NH + 1;                       // its feed plane, wrapped into the cell
    while (fz >= n3) fz -= n3;
    long foff = (long)fz * plane;
    const float* Yown = Y + own;
    const float* Vown = a.V + own;
    const float* Pown = Yp ? Yp + own : nullptr;
    auto issue = [&](int st) {
        if (ip < z1) {
            ulonglong2* ys = stY(st);
#pragma unroll
            for (int k = 0; k < PER; ++k)
                if (s_idx[k] >= 0) cp_async<16>(ys + s_idx[k], s_src[k] + ioff);
            if (active) {
                cp_async<16>(stI(st, 1) + tid, Vown + ioff);
                if (Pown) cp_async<16>(stI(st, 2) + tid, Pown + ioff);
            }
        }
        if (active && ip + 1 < z1) cp_async<16>(stI(st, 0) + tid, Yown + foff);
        ++ip;
        ioff += plane;
        if (++fz == n3) { fz = 0; foff = 0; } else foff += plane;
    };

    u64 wx[NH], wy[NH], wz[NH];
#pragma unroll
    for (int p = 0; p < NH; ++p) {
        wx[p] = pk2(cf.w[0][p], cf.w[0][p]);
        wy[p] = pk2(cf.w[1][p], cf.w[1][p]);
        wz[p] = pk2(cf.w[2][p], cf.w[2][p]);
    }
    const u64 cen2 = pk2(cf.center, cf.center), alp2 = pk2(cf.alpha, cf.alpha), bet2 = pk2(cf.beta, cf.beta);
    const u64 m2 = pk2(-2.0f, -2.0f);

    u64 ql[Q], qh[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        ql[j] = 0ull;
        qh[j] = 0ull;
        if (active) {
            const int p = z0 - NH + j;
            const int wz_ = floordiv(p, n3);
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(Y + (long)(p - wz_ * n3) * plane + own);
            ql[j] = v.x;
            qh[j] = v.y;
        }
    }
#pragma unroll 1
    for (int j = 0; j < PH; ++j) {
        issue(j % RS);
        cp_async_commit();
    }
    int sz = 0, si = PH % RS;                   // stage of plane z, stage of the next issue
    const int rbase = (ty + NH) * SXV;
#pragma unroll 1
    for (int zb = z0; zb < z1; zb += Q) {
#pragma unroll
        for (int st = 0; st < Q; ++st) {
            const int z = zb + st;
            if (z >= z1) break;
            issue(si);
            cp_async_commit();
            cp_async_wait<PH>();
            __syncthreads();
            if (active) {
                const ulonglong2* ys = stY(sz);
                u64 r[10];
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    const ulonglong2 v = ys[rbase + tx + j];
                    r[2 * j] = v.x;
                    r[2 * j + 1] = v.y;
                }
                u64 u[8];
#pragma unroll
                for (int k = 1; k <= 7; ++k) u[k] = pk2(hi2(r[k]), lo2(r[k + 1]));
                const ulonglong2 vv = stI(sz, 1)[tid];
                const u64 cl = ql[(st + NH) % Q], ch = qh[(st + NH) % Q];
                u64 xl = 0ull, xh = 0ull, yl = 0ull, yh = 0ull, zl = 0ull, zh = 0ull;
#pragma unroll
                for (int p = 1; p <= NH; ++p) {
                    const u64 dzl = fma2(m2, cl, add2(ql[(st + NH + p) % Q], ql[(st + NH - p) % Q]));
                    const u64 dzh = fma2(m2, ch, add2(qh[(st + NH + p) % Q], qh[(st + NH - p) % Q]));
                    const u64 lp = (p & 1) ? u[(8 + p - 1) / 2] : r[(8 + p) / 2];
                    const u64 lm = (p & 1) ? u[(8 - p - 1) / 2] : r[(8 - p) / 2];
                    const u64 hp = (p & 1) ? u[(10 + p - 1) / 2] : r[(10 + p) / 2];
                    const u64 hm = (p & 1) ? u[(10 - p - 1) / 2] : r[(10 - p) / 2];
                    const u64 dxl = fma2(m2, cl, add2(lp, lm));
                    const u64 dxh = fma2(m2, ch, add2(hp, hm));
                    const ulonglong2 up = ys[rbase + p * SXV + tx + 2];
                    const ulonglong2 dn = ys[rbase - p * SXV + tx + 2];
                    const u64 dyl = fma2(m2, cl, add2(up.x, dn.x));
                    const u64 dyh = fma2(m2, ch, add2(up.y, dn.y));
                    if (p == 1) {
                        zl = mul2(wz[0], dzl); zh = mul2(wz[0], dzh);
                        xl = mul2(wx[0], dxl); xh = mul2(wx[0], dxh);
                        yl = mul2(wy[0], dyl); yh = mul2(wy[0], dyh);
                    } else {
                        zl = fma2(wz[p - 1], dzl, zl); zh = fma2(wz[p - 1], dzh, zh);
                        xl = fma2(wx[p - 1], dxl, xl); xh = fma2(wx[p - 1], dxh, xh);
                        yl = fma2(wy[p - 1], dyl, yl); yh = fma2(wy[p - 1], dyh, yh);
                    }
                }
                u64 al = mul2(fma2(alp2, vv.x, cen2), cl);
                u64 ah = mul2(fma2(alp2, vv.y, cen2), ch);
                al = add2(al, add2(add2(xl, yl), zl));
                ah = add2(ah, add2(add2(xh, yh), zh));
                if (Yp) {
                    const ulonglong2 pv = stI(sz, 2)[tid];
                    al = fma2(bet2, pv.x, al);
                    ah = fma2(bet2, pv.y, ah);
                }
                *reinterpret_cast<ulonglong2*>(Yo + (long)z * plane + own) = make_ulonglong2(al, ah);
                if (z + 1 < z1) {
                    const ulonglong2 f = stI(sz, 0)[tid];
                    ql[st] = f.x;                 // slot of plane z - NH takes plane z + NH + 1
                    qh[st] = f.y;
                }
            }
            if (++sz == RS) sz = 0;
            if (++si == RS) si = 0;
        }
    }
    cp_async_wait<0>();
}

// Two y-rows per thread (rows A = 2 ty and B = 2 ty + 1 of the tile, 4 x-points each): the
// y-neighbour rows of the pair are read once for both (row rb + 1 + p serves A's pair p + 1
// and B's pair p, row rb - p serves A's pair p and B's pair p + 1; the two centre rows come
// from the z-queues), halving the shared-memory bytes of the y-terms, and the copy and loop
// work of a plane is shared by 8 points.  Per point the arithmetic and its order are those of
// k_stencil_f32s (the results are the same bits).
template <int TXT, int TYT, int PH>
struct Split2Cfg {
    static constexpr int NH = 6, HX = 8;
    static constexpr int TXP = TXT * 4;
    static constexpr int TY = 2 * TYT;                 // rows of the tile
    static constexpr int SXV = (TXP + 2 * HX) / 4;     // float4 vectors per halo row
    static constexpr int SY = TY + 2 * NH;
    static constexpr int NT = TXT * TYT;               // threads
    static constexpr int RS = PH + 2;
    static constexpr int NVS = SXV * SY;
    static constexpr int PER = (NVS + NT - 1) / NT;
    static constexpr size_t YB = 16 * (size_t)NVS;     // halo plane
    static constexpr size_t IB = 32 * (size_t)NT;      // two float4 per thread (rows A, B)
    static constexpr size_t STAGE = YB + 3 * IB;       // halo | feed | V | Yprev
    static constexpr size_t SMEM = STAGE * RS;
};

template <int TXT, int TYT, int PH>
__global__ void __launch_bounds__(TXT * TYT, 1)
k_stencil_f32s2(StencilDev<float> a) {
    const Coef<float> cf = resolve_coef(a);
    using C = Split2Cfg<TXT, TYT, PH>;
    constexpr int NH = C::NH, HX = C::HX, SXV = C::SXV, RS = C::RS, NT = C::NT, PER = C::PER;
    constexpr int Q = 2 * NH + 1;
    static_assert(C::YB % 16 == 0 && C::STAGE % 16 == 0, "stage regions stay 16-byte aligned");
    extern __shared__ __align__(128) unsigned char smem[];

    const int tid = threadIdx.x;
    const int tx = tid % TXT, ty = tid / TXT;
    const int col = blockIdx.z / a.nzc;
    const int zc = blockIdx.z - col * a.nzc;
    const int z0 = zc * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.n3);
    const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
    const long plane = (long)n1 * n2;
    const int gx0 = blockIdx.x * C::TXP, gy0 = blockIdx.y * C::TY;

    const float* __restrict__ Y = reinterpret_cast<const float*>(a.Y) + (size_t)col * a.ld;
    const float* Yp = a.Yprev ? reinterpret_cast<const float*>(a.Yprev) + (size_t)col * a.ld : nullptr;
    float* Yo = reinterpret_cast<float*>(a.Yout) + (size_t)col * a.ld;

    int s_idx[PER];
    const float* s_src[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NT;
        s_idx[k] = -1;
        s_src[k] = Y;
        if (i < C::NVS) {
            const int cx = i % SXV, iy = i / SXV;
            const int gx = gx0 - HX + cx * 4, gy = gy0 - NH + iy;
            const int wx = floordiv(gx, n1), wy = floordiv(gy, n2);
            s_idx[k] = i;
            s_src[k] = Y + (long)(gy - wy * n2) * n1 + (gx - wx * n1);
        }
    }
    const int gxt = gx0 + tx * 4, gyA = gy0 + 2 * ty;
    const bool actA = (gxt < n1) && (gyA < n2);
    const bool actB = (gxt < n1) && (gyA + 1 < n2);
    const long ownA = (long)gyA * n1 + gxt, ownB = ownA + n1;

    auto stY = [&](int st) { return reinterpret_cast<ulonglong2*>(smem + C::STAGE * (size_t)st); };
    auto stI = [&](int st, int k) {            // k = 0 feed, 1 V, 2 Yprev; [2 tid + row]
        return reinterpret_cast<ulonglong2*>(smem + C::STAGE * (size_t)st + C::YB + C::IB * (size_t)k);
    };
    int ip = z0;
    long ioff = (long)z0 * plane;
    int fz = z0 + NH + 1;
    while (fz >= n3) fz -= n3;
    long foff = (long)fz * plane;
    auto issue = [&](int st) {
        if (ip < z1) {
            ulonglong2* ys = stY(st);
#pragma unroll
            for (int k = 0; k < PER; ++k)
                if (s_idx[k] >= 0) cp_async<16>(ys + s_idx[k], s_src[k] + ioff);
            if (actA) {
                cp_async<16>(stI(st, 1) + 2 * tid, a.V + ioff + ownA);
                if (Yp) cp_async<16>(stI(st, 2) + 2 * tid, Yp + ioff + ownA);
            }
            if (actB) {
                cp_async<16>(stI(st, 1) + 2 * tid + 1, a.V + ioff + ownB);
                if (Yp) cp_async<16>(stI(st, 2) + 2 * tid + 1, Yp + ioff + ownB);
            }
        }
        if (ip + 1 < z1) {
            if (actA) cp_async<16>(stI(st, 0) + 2 * tid, Y + foff + ownA);
            if (actB) cp_async<16>(stI(st, 0) + 2 * tid + 1, Y + foff + ownB);
        }
        ++ip;
        ioff += plane;
        if (++fz == n3) { fz = 0; foff = 0; } else foff += plane;
    };

    u64 wx[NH], wy[NH], wz[NH];
#pragma unroll
    for (int p = 0; p < NH; ++p) {
        wx[p] = pk2(cf.w[0][p], cf.w[0][p]);
        wy[p] = pk2(cf.w[1][p], cf.w[1][p]);
        wz[p] = pk2(cf.w[2][p], cf.w[2][p]);
    }
    const u64 cen2 = pk2(cf.center, cf.center), alp2 = pk2(cf.alpha, cf.alpha), bet2 = pk2(cf.beta, cf.beta);
    const u64 m2 = pk2(-2.0f, -2.0f);

    u64 qAl[Q], qAh[Q], qBl[Q], qBh[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        qAl[j] = qAh[j] = qBl[j] = qBh[j] = 0ull;
        const int p = z0 - NH + j;
        const int wz_ = floordiv(p, n3);
        const long zo = (long)(p - wz_ * n3) * plane;
        if (actA) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(Y + zo + ownA);
            qAl[j] = v.x;
            qAh[j] = v.y;
        }
        if (actB) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(Y + zo + ownB);
            qBl[j] = v.x;
            qBh[j] = v.y;
        }
    }
#pragma unroll 1
    for (int j = 0; j < PH; ++j) {
        issue(j % RS);
        cp_async_commit();
    }
    int sz = 0, si = PH % RS;
    const int rb = 2 * ty + NH;                 // halo row of row A
    // x-terms of one row: halo row hr, centre (cl, ch), into (xl, xh)
    auto xterms = [&](const ulonglong2* ys, int hr, u64 cl, u64 ch, u64& xl, u64& xh) {
        u64 r[10];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const ulonglong2 v = ys[hr * SXV + tx + j];
            r[2 * j] = v.x;
            r[2 * j + 1] = v.y;
        }
        u64 u[8];
#pragma unroll
        for (int k = 1; k <= 7; ++k) u[k] = pk2(hi2(r[k]), lo2(r[k + 1]));
#pragma unroll
        for (int p = 1; p <= NH; ++p) {
            const u64 lp = (p & 1) ? u[(8 + p - 1) / 2] : r[(8 + p) / 2];
            const u64 lm = (p & 1) ? u[(8 - p - 1) / 2] : r[(8 - p) / 2];
            const u64 hp = (p & 1) ? u[(10 + p - 1) / 2] : r[(10 + p) / 2];
            const u64 hm = (p & 1) ? u[(10 - p - 1) / 2] : r[(10 - p) / 2];
            const u64 dxl = fma2(m2, cl, add2(lp, lm));
            const u64 dxh = fma2(m2, ch, add2(hp, hm));
            if (p == 1) { xl = mul2(wx[0], dxl); xh = mul2(wx[0], dxh); }
            else { xl = fma2(wx[p - 1], dxl, xl); xh = fma2(wx[p - 1], dxh, xh); }
        }
    };
#pragma unroll 1
    for (int zb = z0; zb < z1; zb += Q) {
#pragma unroll
        for (int st = 0; st < Q; ++st) {
            const int z = zb + st;
            if (z >= z1) break;
            issue(si);
            cp_async_commit();
            cp_async_wait<PH>();
            __syncthreads();
            if (actA || actB) {
                const ulonglong2* ys = stY(sz);
                const u64 cAl = qAl[(st + NH) % Q], cAh = qAh[(st + NH) % Q];
                const u64 cBl = qBl[(st + NH) % Q], cBh = qBh[(st + NH) % Q];
                // y-terms of both rows; upl/uph = row rb + p, dnl/dnh = row rb + 1 - p (the
                // rows A's pair p and B's pair p - 1 share), advanced pairwise
                u64 yAl = 0ull, yAh = 0ull, yBl = 0ull, yBh = 0ull;
                u64 upl = cBl, uph = cBh, dnl = cAl, dnh = cAh;
                if (!actB) {                    // row B outside the cell: its periodic image
                    const ulonglong2 c1 = ys[(rb + 1) * SXV + tx + 2];
                    upl = c1.x;
                    uph = c1.y;
                }
#pragma unroll
                for (int p = 1; p <= NH; ++p) {
                    const ulonglong2 nu = ys[(rb + 1 + p) * SXV + tx + 2];      // row rb + 1 + p
                    const ulonglong2 nd = ys[(rb - p) * SXV + tx + 2];          // row rb - p
                    const u64 dAl = fma2(m2, cAl, add2(upl, nd.x));
                    const u64 dAh = fma2(m2, cAh, add2(uph, nd.y));
                    const u64 dBl = fma2(m2, cBl, add2(nu.x, dnl));
                    const u64 dBh = fma2(m2, cBh, add2(nu.y, dnh));
                    if (p == 1) {
                        yAl = mul2(wy[0], dAl); yAh = mul2(wy[0], dAh);
                        yBl = mul2(wy[0], dBl); yBh = mul2(wy[0], dBh);
                    } else {
                        yAl = fma2(wy[p - 1], dAl, yAl); yAh = fma2(wy[p - 1], dAh, yAh);
                        yBl = fma2(wy[p - 1], dBl, yBl); yBh = fma2(wy[p - 1], dBh, yBh);
                    }
                    upl = nu.x; uph = nu.y;
                    dnl = nd.x; dnh = nd.y;
                }
                // row A: z-terms, x-terms, combination (the order of k_stencil_f32s)
                {
                    u64 zl = 0ull, zh = 0ull, xl = 0ull, xh = 0ull;
#pragma unroll
                    for (int p = 1; p <= NH; ++p) {
                        const u64 dzl = fma2(m2, cAl, add2(qAl[(st + NH + p) % Q], qAl[(st + NH - p) % Q]));
                        const u64 dzh = fma2(m2, cAh, add2(qAh[(st + NH + p) % Q], qAh[(st + NH - p) % Q]));
                        if (p == 1) { zl = mul2(wz[0], dzl); zh = mul2(wz[0], dzh); }
                        else { zl = fma2(wz[p - 1], dzl, zl); zh = fma2(wz[p - 1], dzh, zh); }
                    }
                    xterms(ys, rb, cAl, cAh, xl, xh);
                    const ulonglong2 vv = stI(sz, 1)[2 * tid];
                    u64 al = mul2(fma2(alp2, vv.x, cen2), cAl);
                    u64 ah = mul2(fma2(alp2, vv.y, cen2), cAh);
                    al = add2(al, add2(add2(xl, yAl), zl));
                    ah = add2(ah, add2(add2(xh, yAh), zh));
                    if (Yp) {
                        const ulonglong2 pv = stI(sz, 2)[2 * tid];
                        al = fma2(bet2, pv.x, al);
                        ah = fma2(bet2, pv.y, ah);
                    }
                    if (actA) *reinterpret_cast<ulonglong2*>(Yo + (long)z * plane + ownA) = make_ulonglong2(al, ah);
                }
                {
                    u64 zl = 0ull, zh = 0ull, xl = 0ull, xh = 0ull;
#pragma unroll
                    for (int p = 1; p <= NH; ++p) {
                        const u64 dzl = fma2(m2, cBl, add2(qBl[(st + NH + p) % Q], qBl[(st + NH - p) % Q]));
                        const u64 dzh = fma2(m2, cBh, add2(qBh[(st + NH + p) % Q], qBh[(st + NH - p) % Q]));
                        if (p == 1) { zl = mul2(wz[0], dzl); zh = mul2(wz[0], dzh); }
                        else { zl = fma2(wz[p - 1], dzl, zl); zh = fma2(wz[p - 1], dzh, zh); }
                    }
                    xterms(ys, rb + 1, cBl, cBh, xl, xh);
                    const ulonglong2 vv = stI(sz, 1)[2 * tid + 1];
                    u64 bl = mul2(fma2(alp2, vv.x, cen2), cBl);
                    u64 bh = mul2(fma2(alp2, vv.y, cen2), cBh);
                    bl = add2(bl, add2(add2(xl, yBl), zl));
                    bh = add2(bh, add2(add2(xh, yBh), zh));
                    if (Yp) {
                        const ulonglong2 pv = stI(sz, 2)[2 * tid + 1];
                        bl = fma2(bet2, pv.x, bl);
                        bh = fma2(bet2, pv.y, bh);
                    }
                    if (actB) *reinterpret_cast<ulonglong2*>(Yo + (long)z * plane + ownB) = make_ulonglong2(bl, bh);
                }
                if (z + 1 < z1) {
                    const ulonglong2 fa = stI(sz, 0)[2 * tid], fb = stI(sz, 0)[2 * tid + 1];
                    qAl[st] = fa.x; qAh[st] = fa.y;         // slot of plane z - NH takes plane z + NH + 1
                    qBl[st] = fb.x; qBh[st] = fb.y;
                }
            }
            if (++sz == RS) sz = 0;
            if (++si == RS) si = 0;
        }
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------- complex float form
// Complex float (Bloch orbitals), two consecutive x-points per thread held as two packed
// (re, im) pairs: the Laplacian's real weights, V and the recurrence act on re and im alike,
// so every add and FMA is one f32x2 instruction on one complex value, and the x-neighbours of
// both points are whole pairs (no register moves to form them).  Same split ring as the real
// float form: a stage holds the halo'd plane z (x/y neighbours, NHC = 6 points = 3 vectors of
// halo on each side of a row), plus three per-thread interior slots: the queue feed plane
// z + NH + 1, V (two floats) and Yprev of plane z.  Bloch factors: a halo slot whose copy
// wrapped across an x or y face is multiplied by exp(i k_a L_a)^wraps by the thread that
// copied it, after its copy landed and before the plane's barrier (interior tiles have no
// such slots); a queue plane that wrapped in z takes exp(i k_3 L_3)^wraps when it enters
// the queue.
template <int TXT, int TY, int PH>
struct SplitCCfg {
    static constexpr int NH = 6, HXV = 3;               // halo: 6 complex = 3 vectors per side
    static constexpr int TXP = TXT * 2;                 // complex points per tile row
    static constexpr int SXV = TXT + 2 * HXV;           // 16-byte vectors per halo row
    static constexpr int SY = TY + 2 * NH;
    static constexpr int NT = TXT * TY;
    static constexpr int RS = PH + 2;
    static constexpr int NVS = SXV * SY;
    static constexpr int PER = (NVS + NT - 1) / NT;
    static constexpr size_t YB = 16 * (size_t)NVS;      // halo plane
    static constexpr size_t IB = 16 * (size_t)NT;       // one vector per thread (feed, Yprev)
    static constexpr size_t VB = 8 * (size_t)NT;        // two floats per thread (V)
    static constexpr size_t STAGE = YB + 2 * IB + VB;   // halo | feed | Yprev | V
    static constexpr size_t SMEM = STAGE * RS;
};

__device__ __forceinline__ u64 f2u(float2 v) { return pk2(v.x, v.y); }
__device__ __forceinline__ float2 u2f(u64 v) { return make_float2(lo2(v), hi2(v)); }

template <int TXT, int TY, int PH>
__global__ void __launch_bounds__(TXT * TY)
k_stencil_c32s(StencilDev<float> a) {
    const Coef<float> cf = resolve_coef(a);
    using C = SplitCCfg<TXT, TY, PH>;
    constexpr int NH = C::NH, HXV = C::HXV, SXV = C::SXV, RS = C::RS, NT = C::NT, PER = C::PER;
    constexpr int Q = 2 * NH + 1;
    static_assert(C::YB % 16 == 0 && C::STAGE % 16 == 0, "stage regions stay 16-byte aligned");
    extern __shared__ __align__(128) unsigned char smem[];

    const int tid = threadIdx.x;
    const int tx = tid % TXT, ty = tid / TXT;
    const int col = blockIdx.z / a.nzc;
    const int zc = blockIdx.z - col * a.nzc;
    const int z0 = zc * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.n3);
    const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
    const long plane = (long)n1 * n2;
    const int gx0 = blockIdx.x * C::TXP, gy0 = blockIdx.y * TY;

    // element = one complex float (8 bytes)
    const float2* __restrict__ Y = reinterpret_cast<const float2*>(a.Y) + (size_t)col * a.ld;
    const float2* Yp = a.Yprev ? reinterpret_cast<const float2*>(a.Yprev) + (size_t)col * a.ld : nullptr;
    float2* Yo = reinterpret_cast<float2*>(a.Yout) + (size_t)col * a.ld;

    int s_idx[PER];
    const float2* s_src[PER];
    float2 s_ph[PER];            // Bloch factor of a slot that wrapped in x or y
    bool s_wrap[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NT;
        s_idx[k] = -1;
        s_src[k] = Y;
        s_ph[k] = make_float2(1.f, 0.f);
        s_wrap[k] = false;
        if (i < C::NVS) {
            const int cx = i % SXV, iy = i / SXV;
            const int gx = gx0 + 2 * (cx - HXV), gy = gy0 - NH + iy;
            const int wx = floordiv(gx, n1), wy = floordiv(gy, n2);
            s_idx[k] = i;
            s_src[k] = Y + (long)(gy - wy * n2) * n1 + (gx - wx * n1);
            if (wx != 0 || wy != 0) {
                s_wrap[k] = true;
                s_ph[k] = cmul(phase_pow<float2>(a.ph[0][0], a.ph[0][1], wx), phase_pow<float2>(a.ph[1][0], a.ph[1][1], wy));
            }
        }
    }
    const bool active = (gx0 + tx * 2 < n1) && (gy0 + ty < n2);
    const long own = (long)(gy0 + ty) * n1 + (gx0 + tx * 2);

    auto stY = [&](int st) { return reinterpret_cast<ulonglong2*>(smem + C::STAGE * (size_t)st); };
    auto stI = [&](int st, int k) {            // k = 0 feed, 1 Yprev
        return reinterpret_cast<ulonglong2*>(smem + C::STAGE * (size_t)st + C::YB + C::IB * (size_t)k);
    };
    auto stV = [&](int st) { return reinterpret_cast<float2*>(smem + C::STAGE * (size_t)st + C::YB + 2 * C::IB); };
    int ip = z0;
    long ioff = (long)z0 * plane;
    int fz = z0 + NH + 1;
    while (fz >= n3) fz -= n3;
    long foff = (long)fz * plane;
    const float2* Yown = Y + own;
    const float* Vown = a.V + own;
    const float2* Pown = Yp ? Yp + own : nullptr;
    auto issue = [&](int st) {
        if (ip < z1) {
            ulonglong2* ys = stY(st);
#pragma unroll
            for (int k = 0; k < PER; ++k)
                if (s_idx[k] >= 0) cp_async<16>(ys + s_idx[k], s_src[k] + ioff);
            if (active) {
                cp_async<8>(stV(st) + tid, Vown + ioff);
                if (Pown) cp_async<16>(stI(st, 1) + tid, Pown + ioff);
            }
        }
        if (active && ip + 1 < z1) cp_async<16>(stI(st, 0) + tid, Yown + foff);
        ++ip;
        ioff += plane;
        if (++fz == n3) { fz = 0; foff = 0; } else foff += plane;
    };

    u64 wx[NH], wy[NH], wz[NH];
#pragma unroll
    for (int p = 0; p < NH; ++p) {
        wx[p] = pk2(cf.w[0][p], cf.w[0][p]);
        wy[p] = pk2(cf.w[1][p], cf.w[1][p]);
        wz[p] = pk2(cf.w[2][p], cf.w[2][p]);
    }
    const u64 cen2 = pk2(cf.center, cf.center), alp2 = pk2(cf.alpha, cf.alpha), bet2 = pk2(cf.beta, cf.beta);
    const u64 m2 = pk2(-2.0f, -2.0f);

    // z-queues of the two points (planes z0-NH .. z0+NH), Bloch factors of wrapped planes
    u64 ql[Q], qh[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        ql[j] = 0ull;
        qh[j] = 0ull;
        if (active) {
            const int p = z0 - NH + j;
            const int wz_ = floordiv(p, n3);
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(Y + (long)(p - wz_ * n3) * plane + own);
            ql[j] = v.x;
            qh[j] = v.y;
            if (wz_ != 0) {
                const float2 f = phase_pow<float2>(a.ph[2][0], a.ph[2][1], wz_);
                ql[j] = f2u(cmul(u2f(ql[j]), f));
                qh[j] = f2u(cmul(u2f(qh[j]), f));
            }
        }
    }
    // wrap count and Bloch factor of the feed plane consumed next (plane z + NH + 1)
    int fzc = z0 + NH + 1, fwc = 0;
    while (fzc >= n3) { fzc -= n3; ++fwc; }
    float2 fph = phase_pow<float2>(a.ph[2][0], a.ph[2][1], fwc);
#pragma unroll 1
    for (int j = 0; j < PH; ++j) {
        issue(j % RS);
        cp_async_commit();
    }
    int sz = 0, si = PH % RS;
    const int rbase = (ty + NH) * SXV;
#pragma unroll 1
    for (int zb = z0; zb < z1; zb += Q) {
#pragma unroll
        for (int st = 0; st < Q; ++st) {
            const int z = zb + st;
            if (z >= z1) break;
            issue(si);
            cp_async_commit();
            cp_async_wait<PH>();
            // this thread's wrapped halo slots of plane z take their Bloch factors
            {
                ulonglong2* ys = stY(sz);
#pragma unroll
                for (int k = 0; k < PER; ++k)
                    if (s_wrap[k]) {
                        ulonglong2 v = ys[s_idx[k]];
                        v.x = f2u(cmul(u2f(v.x), s_ph[k]));
                        v.y = f2u(cmul(u2f(v.y), s_ph[k]));
                        ys[s_idx[k]] = v;
                    }
            }
            __syncthreads();
            if (active) {
                const ulonglong2* ys = stY(sz);
                // the row around the thread's two points: complex x-offsets -6 .. +7
                u64 r[14];
#pragma unroll
                for (int j = 0; j < 7; ++j) {
                    const ulonglong2 v = ys[rbase + tx + j];
                    r[2 * j] = v.x;
                    r[2 * j + 1] = v.y;
                }
                const float2 vv = stV(sz)[tid];
                const u64 cl = ql[(st + NH) % Q], ch = qh[(st + NH) % Q];
                u64 xl = 0ull, xh = 0ull, yl = 0ull, yh = 0ull, zl = 0ull, zh = 0ull;
#pragma unroll
                for (int p = 1; p <= NH; ++p) {
                    const u64 dzl = fma2(m2, cl, add2(ql[(st + NH + p) % Q], ql[(st + NH - p) % Q]));
                    const u64 dzh = fma2(m2, ch, add2(qh[(st + NH + p) % Q], qh[(st + NH - p) % Q]));
                    const u64 dxl = fma2(m2, cl, add2(r[6 + p], r[6 - p]));
                    const u64 dxh = fma2(m2, ch, add2(r[7 + p], r[7 - p]));
                    const ulonglong2 up = ys[rbase + p * SXV + tx + HXV];
                    const ulonglong2 dn = ys[rbase - p * SXV + tx + HXV];
                    const u64 dyl = fma2(m2, cl, add2(up.x, dn.x));
                    const u64 dyh = fma2(m2, ch, add2(up.y, dn.y));
                    if (p == 1) {
                        zl = mul2(wz[0], dzl); zh = mul2(wz[0], dzh);
                        xl = mul2(wx[0], dxl); xh = mul2(wx[0], dxh);
                        yl = mul2(wy[0], dyl); yh = mul2(wy[0], dyh);
                    } else {
                        zl = fma2(wz[p - 1], dzl, zl); zh = fma2(wz[p - 1], dzh, zh);
                        xl = fma2(wx[p - 1], dxl, xl); xh = fma2(wx[p - 1], dxh, xh);
                        yl = fma2(wy[p - 1], dyl, yl); yh = fma2(wy[p - 1], dyh, yh);
                    }
                }
                u64 al = mul2(fma2(alp2, pk2(vv.x, vv.x), cen2), cl);
                u64 ah = mul2(fma2(alp2, pk2(vv.y, vv.y), cen2), ch);
                al = add2(al, add2(add2(xl, yl), zl));
                ah = add2(ah, add2(add2(xh, yh), zh));
                if (Yp) {
                    const ulonglong2 pv = stI(sz, 1)[tid];
                    al = fma2(bet2, pv.x, al);
                    ah = fma2(bet2, pv.y, ah);
                }
                *reinterpret_cast<ulonglong2*>(Yo + (long)z * plane + own) = make_ulonglong2(al, ah);
                if (z + 1 < z1) {
                    const ulonglong2 f = stI(sz, 0)[tid];
                    // slot of plane z - NH takes plane z + NH + 1 (with its Bloch factor)
                    if (fwc != 0) {
                        ql[st] = f2u(cmul(u2f(f.x), fph));
                        qh[st] = f2u(cmul(u2f(f.y), fph));
                    } else {
                        ql[st] = f.x;
                        qh[st] = f.y;
                    }
                }
            }
            if (++fzc == n3) {
                fzc = 0;
                ++fwc;
                fph = phase_pow<float2>(a.ph[2][0], a.ph[2][1], fwc);
            }
            if (++sz == RS) sz = 0;
            if (++si == RS) si = 0;
        }
    }
    cp_async_wait<0>();
}

template <int TXT, int TY, int PH>
static int run_c32s(hub_t h, const StencilArgs& s) {
    using Cfg = SplitCCfg<TXT, TY, PH>;
    StencilDev<float> d;
    d.Y = s.Y;
    d.Yprev = s.Yprev;
    d.Yout = s.Yout;
    d.V = reinterpret_cast<const float*>(s.V);
    d.n1 = s.n1; d.n2 = s.n2; d.n3 = s.n3; d.ld = s.ld;
    fill_coefficients<float>(s, d);
    for (int a = 0; a < 3; ++a) {
        d.ph[a][0] = s.phase[a][0];
        d.ph[a][1] = s.phase[a][1];
    }
    const int tiles = ((s.n1 + Cfg::TXP - 1) / Cfg::TXP) * ((s.n2 + TY - 1) / TY);
    const long want = 8L * h->num_sms;
    const long per = (long)tiles * s.ncol;
    int nzc = 1;
    if (per < want) nzc = (int)((want + per - 1) / per);
    int zchunk = (s.n3 + nzc - 1) / nzc;
    if (zchunk < 16) zchunk = s.n3 < 16 ? s.n3 : 16;
    nzc = (s.n3 + zchunk - 1) / zchunk;
    while ((long)s.ncol * nzc > 65535) { zchunk *= 2; nzc = (s.n3 + zchunk - 1) / zchunk; }
    d.zchunk = zchunk;
    d.nzc = nzc;
    HUB_CUDA_TRY(h, cudaFuncSetAttribute(k_stencil_c32s<TXT, TY, PH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
    dim3 grid((s.n1 + Cfg::TXP - 1) / Cfg::TXP, (s.n2 + TY - 1) / TY, s.ncol * nzc);
    ProfScope ps(h, HUB_K_STENCIL);
    k_stencil_c32s<TXT, TY, PH><<<grid, TXT * TY, Cfg::SMEM, h->stream>>>(d);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

template <int TXT, int TYT, int PH>
static int run_f32s2(hub_t h, const StencilArgs& s) {
    using Cfg = Split2Cfg<TXT, TYT, PH>;
    StencilDev<float> d;
    d.Y = s.Y;
    d.Yprev = s.Yprev;
    d.Yout = s.Yout;
    d.V = reinterpret_cast<const float*>(s.V);
    d.n1 = s.n1; d.n2 = s.n2; d.n3 = s.n3; d.ld = s.ld;
    fill_coefficients<float>(s, d);
    for (int a = 0; a < 3; ++a) {
        d.ph[a][0] = 1.0;
        d.ph[a][1] = 0.0;
    }
    const int tiles = ((s.n1 + Cfg::TXP - 1) / Cfg::TXP) * ((s.n2 + Cfg::TY - 1) / Cfg::TY);
    const long want = 4L * h->num_sms;
    const long per = (long)tiles * s.ncol;
    int nzc = 1;
    if (per < want) nzc = (int)((want + per - 1) / per);
    int zchunk = (s.n3 + nzc - 1) / nzc;
    if (zchunk < 16) zchunk = s.n3 < 16 ? s.n3 : 16;
    nzc = (s.n3 + zchunk - 1) / zchunk;
    while ((long)s.ncol * nzc > 65535) { zchunk *= 2; nzc = (s.n3 + zchunk - 1) / zchunk; }
    d.zchunk = zchunk;
    d.nzc = nzc;
    HUB_CUDA_TRY(h, cudaFuncSetAttribute(k_stencil_f32s2<TXT, TYT, PH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
    dim3 grid((s.n1 + Cfg::TXP - 1) / Cfg::TXP, (s.n2 + Cfg::TY - 1) / Cfg::TY, s.ncol * nzc);
    ProfScope ps(h, HUB_K_STENCIL);
    k_stencil_f32s2<TXT, TYT, PH><<<grid, TXT * TYT, Cfg::SMEM, h->stream>>>(d);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

template <int TXT, int TY, int PH>
static int run_f32s(hub_t h, const StencilArgs& s) {
    using Cfg = SplitCfg<TXT, TY, PH>;
    StencilDev<float> d;
    d.Y = s.Y;
    d.Yprev = s.Yprev;
    d.Yout = s.Yout;
    d.V = reinterpret_cast<const float*>(s.V);
    d.n1 = s.n1; d.n2 = s.n2; d.n3 = s.n3; d.ld = s.ld;
    fill_coefficients<float>(s, d);
    for (int a = 0; a < 3; ++a) {
        d.ph[a][0] = 1.0;
        d.ph[a][1] = 0.0;
    }
    const int tiles = ((s.n1 + Cfg::TXP - 1) / Cfg::TXP) * ((s.n2 + TY - 1) / TY);
    const long want = 8L * h->num_sms;
    const long per = (long)tiles * s.ncol;
    int nzc = 1;
    if (per < want) nzc = (int)((want + per - 1) / per);
    int zchunk = (s.n3 + nzc - 1) / nzc;
    if (zchunk < 16) zchunk = s.n3 < 16 ? s.n3 : 16;
    nzc = (s.n3 + zchunk - 1) / zchunk;
    while ((long)s.ncol * nzc > 65535) { zchunk *= 2; nzc = (s.n3 + zchunk - 1) / zchunk; }
    d.zchunk = zchunk;
    d.nzc = nzc;
    HUB_CUDA_TRY(h, cudaFuncSetAttribute(k_stencil_f32s<TXT, TY, PH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
    dim3 grid((s.n1 + Cfg::TXP - 1) / Cfg::TXP, (s.n2 + TY - 1) / TY, s.ncol * nzc);
    ProfScope ps(h, HUB_K_STENCIL);
    k_stencil_f32s<TXT, TY, PH><<<grid, TXT * TY, Cfg::SMEM, h->stream>>>(d);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

template <typename R, bool CPLX, int VEC, int TXT, int TY, int P>
static int run_vec(hub_t h, const StencilArgs& s) {
    using Cfg = VecCfg<R, CPLX, VEC, TXT, TY, P>;
    StencilDev<R> d;
    d.Y = s.Y;
    d.Yprev = s.Yprev;
    d.Yout = s.Yout;
    d.V = reinterpret_cast<const R*>(s.V);
    d.n1 = s.n1; d.n2 = s.n2; d.n3 = s.n3; d.ld = s.ld;
    fill_coefficients<R>(s, d);
    for (int a = 0; a < 3; ++a) {
        d.ph[a][0] = s.phase[a][0];
        d.ph[a][1] = s.phase[a][1];
    }
    const int tiles = ((s.n1 + Cfg::TXP - 1) / Cfg::TXP) * ((s.n2 + TY - 1) / TY);
    const long want = 4L * h->num_sms;
    const long per = (long)tiles * s.ncol;
    int nzc = 1;
    if (per < want) nzc = (int)((want + per - 1) / per);
    int zchunk = (s.n3 + nzc - 1) / nzc;
    if (zchunk < 16) zchunk = s.n3 < 16 ? s.n3 : 16;
    nzc = (s.n3 + zchunk - 1) / zchunk;
    while ((long)s.ncol * nzc > 65535) { zchunk *= 2; nzc = (s.n3 + zchunk - 1) / zchunk; }
    d.zchunk = zchunk;
    d.nzc = nzc;
    HUB_CUDA_TRY(h, cudaFuncSetAttribute(k_stencil_vec<R, CPLX, VEC, TXT, TY, P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
    dim3 grid((s.n1 + Cfg::TXP - 1) / Cfg::TXP, (s.n2 + TY - 1) / TY, s.ncol * nzc);
    ProfScope ps(h, HUB_K_STENCIL);
    k_stencil_vec<R, CPLX, VEC, TXT, TY, P><<<grid, TXT * TY, Cfg::SMEM, h->stream>>>(d);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

template <typename R, bool CPLX, int TX, int TY, int P>
static int run_cfg(hub_t h, const StencilArgs& s) {
    using Cfg = StencilCfg<R, CPLX, TX, TY, P>;
    StencilDev<R> d;
    d.Y = s.Y;
    d.Yprev = s.Yprev;
    d.Yout = s.Yout;
    d.V = reinterpret_cast<const R*>(s.V);
    d.n1 = s.n1; d.n2 = s.n2; d.n3 = s.n3; d.ld = s.ld;
    fill_coefficients<R>(s, d);
    for (int a = 0; a < 3; ++a) {
        d.ph[a][0] = s.phase[a][0];
        d.ph[a][1] = s.phase[a][1];
    }
    const int tiles = ((s.n1 + TX - 1) / TX) * ((s.n2 + TY - 1) / TY);
    // enough CTAs to fill every SM several times, chunks long enough that the prologue of
    // 2*NH+P planes stays a modest overhead
    const long want = 6L * h->num_sms;
    const long per = (long)tiles * s.ncol;
    int nzc = 1;
    if (per < want) nzc = (int)((want + per - 1) / per);
    int zchunk = (s.n3 + nzc - 1) / nzc;
    if (zchunk < 16) zchunk = s.n3 < 16 ? s.n3 : 16;
    nzc = (s.n3 + zchunk - 1) / zchunk;
    while ((long)s.ncol * nzc > 65535) { zchunk *= 2; nzc = (s.n3 + zchunk - 1) / zchunk; }
    d.zchunk = zchunk;
    d.nzc = nzc;
    HUB_CUDA_TRY(h, cudaFuncSetAttribute(k_stencil<R, CPLX, TX, TY, P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
    dim3 grid((s.n1 + TX - 1) / TX, (s.n2 + TY - 1) / TY, s.ncol * nzc);
    ProfScope ps(h, HUB_K_STENCIL);
    k_stencil<R, CPLX, TX, TY, P><<<grid, TX * TY, Cfg::SMEM, h->stream>>>(d);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

// ---------------------------------------------------------------------------- gradient
// G = d_axis X by the 2*n0-th order centred first derivative of Sec. II.B:
//   G_i = sum_p w_p (X_{i+p} - X_{i-p}),  w_p = (-1)^{p+1} (n0!)^2 / (h p (n0-p)! (n0+p)!)
// An index past a cell face maps back with exp(i k_a L_a) per crossing (complex only).
// One warp per grid row (fixed y, z) of one column, lanes along x: no per-element index
// division, coalesced loads; the neighbours along y and z are rows of the same column that
// neighbouring warps also read, so they come from L1/L2.  Sums in the working type (float
// blocks stay on the float pipe; FP64 is bound by the FP64 pipe: 12 operations per element).
struct GradArgs {
    double w[kMaxHalf];
    double ph_re, ph_im;
    int n0, axis;
};

constexpr int kGradRows = 8;   // warps (rows) per CTA

template <typename T>
__device__ __forceinline__ T sub(T a, T b);
template <> __device__ __forceinline__ double sub(double a, double b) { return a - b; }
template <> __device__ __forceinline__ float sub(float a, float b) { return a - b; }
template <> __device__ __forceinline__ double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
template <> __device__ __forceinline__ float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <typename R, bool CPLX>
__global__ void __launch_bounds__(32 * kGradRows)
k_fd_gradient(const typename VT<R, CPLX>::T* __restrict__ X, int ld, int n1, int n2, int n3, GradArgs a,
              typename VT<R, CPLX>::T* __restrict__ G) {
    using T = typename VT<R, CPLX>::T;
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * kGradRows + (threadIdx.x >> 5);   // row = y + n2 * z
    if (row >= n2 * n3) return;
    const int y = row % n2, z = row / n2;
    const T* xc = X + (long)blockIdx.y * ld;
    T* gc = G + (long)blockIdx.y * ld;
    const long own = (long)row * n1;
    R w[kMaxHalf];
    for (int p = 0; p < kMaxHalf; ++p) w[p] = (R)a.w[p];
    for (int x = lane; x < n1; x += 32) {
        T acc = zero_of(T{});
        for (int p = 1; p <= a.n0; ++p) {
            long of, ob;       // offsets of the +p and -p neighbours in the column
            int wf = 0, wb = 0;
            if (a.axis == 0) {
                int xf = x + p, xb = x - p;
                while (xf >= n1) { xf -= n1; ++wf; }
                while (xb < 0) { xb += n1; --wb; }
                of = own + xf;
                ob = own + xb;
            } else if (a.axis == 1) {
                int yf = y + p, yb = y - p;
                while (yf >= n2) { yf -= n2; ++wf; }
                while (yb < 0) { yb += n2; --wb; }
                of = ((long)z * n2 + yf) * n1 + x;
                ob = ((long)z * n2 + yb) * n1 + x;
            } else {
                int zf = z + p, zb = z - p;
                while (zf >= n3) { zf -= n3; ++wf; }
                while (zb < 0) { zb += n3; --wb; }
                of = ((long)zf * n2 + y) * n1 + x;
                ob = ((long)zb * n2 + y) * n1 + x;
            }
            T vf = xc[of], vb = xc[ob];
            if constexpr (CPLX) {
                if (wf) vf = cmul(phase_pow<T>(a.ph_re, a.ph_im, wf), vf);
                if (wb) vb = cmul(phase_pow<T>(a.ph_re, a.ph_im, wb), vb);
            }
            acc = fmar(w[p - 1], sub(vf, vb), acc);
        }
        gc[own + x] = acc;
    }
}

int launch_fd_gradient(hub_t h, const void* X, int ld, int ncol, int axis, const double* w, void* G) {
    if (ncol == 0) return HUB_OK;
    GradArgs a{};
    for (int p = 0; p < h->n0; ++p) a.w[p] = w[p];
    a.n0 = h->n0;
    a.axis = axis;
    const double th = h->kpt[axis] * h->L[axis];
    a.ph_re = std::cos(th);
    a.ph_im = std::sin(th);
    if (ncol > 65535) return fail(h, HUB_EINVAL, "at most 65535 columns per gradient launch");
    const dim3 grid((unsigned)((h->n2 * h->n3 + kGradRows - 1) / kGradRows), (unsigned)ncol);
    const int threads = 32 * kGradRows;
    ProfScope ps(h, HUB_K_FORCE);
    if (h->esize == 8) {
        if (h->cplx) k_fd_gradient<double, true><<<grid, threads, 0, h->stream>>>((const double2*)X, ld, h->n1, h->n2, h->n3, a, (double2*)G);
        else k_fd_gradient<double, false><<<grid, threads, 0, h->stream>>>((const double*)X, ld, h->n1, h->n2, h->n3, a, (double*)G);
    } else {
        if (h->cplx) k_fd_gradient<float, true><<<grid, threads, 0, h->stream>>>((const float2*)X, ld, h->n1, h->n2, h->n3, a, (float2*)G);
        else k_fd_gradient<float, false><<<grid, threads, 0, h->stream>>>((const float*)X, ld, h->n1, h->n2, h->n3, a, (float*)G);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

// Tile shapes the autotuner chooses from, per kernel family (index 0 is the default).
int stencil_variants(hub_t h) {
    const int es = h->esize * (h->cplx ? 2 : 1);
    if (h->esize == 4) return h->cplx ? 6 : 9;   // float real (packed) / float complex (packed, vector)
    return es == 16 ? 2 : 3;              // double complex / double real (scalar pipeline)
}

int launch_stencil(hub_t h, const StencilArgs& a) {
    if (a.ncol == 0) return HUB_OK;
    const int es = h->esize * (h->cplx ? 2 : 1);
    const int vec = 16 / es;
    const bool aligned = (a.n1 % vec == 0) && (a.ld % vec == 0) &&
                         ((uintptr_t)a.Y % 16 == 0) && ((uintptr_t)a.Yout % 16 == 0) &&
                         (!a.Yprev || (uintptr_t)a.Yprev % 16 == 0) && ((uintptr_t)a.V % 16 == 0);
    const int v = h->stencil_variant;
    if (aligned && h->esize == 4) {
        // float streams from HBM: vector copies, packed pair arithmetic for real data
        if (!h->cplx) {
            switch (v) {
                case 1: return run_f32s<8, 8, 3>(h, a);
                case 2: return run_f32s<8, 32, 2>(h, a);
                case 3: return run_f32s<8, 16, 3>(h, a);
                case 4: return run_f32s<16, 8, 2>(h, a);
                case 5: return run_f32s<8, 8, 2>(h, a);
                case 6: return run_f32s2<8, 8, 2>(h, a);
                case 7: return run_f32s2<8, 16, 2>(h, a);
                case 8: return run_f32s2<16, 8, 2>(h, a);
                default: return run_f32s<8, 16, 2>(h, a);
            }
        }
        // complex: packed-pair split ring, or the vector form
        switch (v) {
            case 1: return run_c32s<8, 8, 2>(h, a);
            case 2: return run_c32s<16, 8, 2>(h, a);
            case 3: return run_vec<float, true, 2, 16, 16, 2>(h, a);
            case 4: return run_vec<float, true, 2, 16, 8, 2>(h, a);
            case 5: return run_vec<float, true, 2, 8, 16, 2>(h, a);
            default: return run_c32s<8, 16, 2>(h, a);
        }
    }
    // FP64 is bound by the FP64 pipe: a short ring keeps two CTAs per SM
    if (h->esize == 8) {
        if (h->cplx) return v == 1 ? run_cfg<double, true, 32, 4, 2>(h, a) : run_cfg<double, true, 32, 8, 2>(h, a);
        switch (v) {
            case 1: return run_cfg<double, false, 32, 4, 4>(h, a);
            case 2: return run_cfg<double, false, 64, 4, 2>(h, a);
            default: return run_cfg<double, false, 32, 8, 2>(h, a);
        }
    }
    return h->cplx ? run_cfg<float, true, 32, 8, 2>(h, a) : run_cfg<float, false, 32, 8, 4>(h, a);
}

}  // namespace hub
