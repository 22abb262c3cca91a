// Atom-centred localized functions on the grid: KB-type nonlocal projectors and Hubbard
// orbitals share one machinery (Sec. II.B: the DFT+U implementation mirrors the nonlocal
// pseudopotential; all integrals of one atom are computed simultaneously).
//
// A "site" is one (atom, kind) pair with nproj functions  radial(|x - R - T|) Y_lm  summed
// over lattice images T within the cutoff, times exp(i k.T) (Sec. II.A.1, Bloch-mapped
// orbitals).  Every site keeps the sorted list of grid points any of its images touches
// and the values there (point-major).  Three kernels use the tables:
//   gather:    C[row, n] = dV * sum_l conj(vals[l, p]) X[idx[l], n]      (<phi_p|x_n>)
//   transform: W = gamma .* C (KB) or W = M C with M = (U/2)(I - 2 D) (Hubbard, Eq. DerED)
//   scatter:   Y[g, n] += alpha * sum_{entries e at g} vals_e . W[rows_e, n]
// The scatter walks a per-grid-point CSR so that no two threads write the same element.
// Real float handles also keep a brick form of the tables (dense values per 8x8x4 brick,
// see "brick form" below) for a dense scatter and an alternative gather.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <type_traits>
#include <unordered_map>

#include "hub_internal.cuh"
#include "cplx.cuh"

namespace hub {

namespace {

constexpr int GITEM = 1024;    // points per gather work item

__device__ __forceinline__ void solid_harmonics(int l, double x, double y, double z, double* out) {
    // r^l Y_lm for the real orthonormal harmonics, m = -l..l (no Condon-Shortley sign)
    const double PI = 3.14159265358979323846;
    if (l == 0) {
        out[0] = 0.5 / sqrt(PI);
    } else if (l == 1) {
        const double k = sqrt(3.0 / (4.0 * PI));
        out[0] = k * y; out[1] = k * z; out[2] = k * x;
    } else {
        const double k1 = 0.5 * sqrt(15.0 / PI), k0 = 0.25 * sqrt(5.0 / PI), k2 = 0.25 * sqrt(15.0 / PI);
        out[0] = k1 * x * y;
        out[1] = k1 * y * z;
        out[2] = k0 * (2.0 * z * z - x * x - y * y);
        out[3] = k1 * x * z;
        out[4] = k2 * (x * x - y * y);
    }
}

template <typename R, bool CPLX>
__global__ void k_table_values(const SiteDev* __restrict__ sites, const int* __restrict__ items,
                               const int* __restrict__ idx, R* __restrict__ vals, int n1, int n2,
                               double h1, double h2, double h3, double L1, double L2, double L3,
                               double k1, double k2, double k3) {
    const int it = blockIdx.x;
    const int s = items[3 * it], first = items[3 * it + 1], cnt = items[3 * it + 2];
    const SiteDev S = sites[s];
    for (int l = threadIdx.x; l < cnt; l += blockDim.x) {
        const int row = first + l;               // absolute table row
        const int g = idx[row];
        const int i1 = g % n1, i2 = (g / n1) % n2, i3 = g / (n1 * n2);
        const double x = i1 * h1, y = i2 * h2, z = i3 * h3;
        double re[kMaxProj], im[kMaxProj];
        for (int p = 0; p < kMaxProj; ++p) { re[p] = 0.0; im[p] = 0.0; }
        for (int t1 = S.tlo[0]; t1 <= S.thi[0]; ++t1)
            for (int t2 = S.tlo[1]; t2 <= S.thi[1]; ++t2)
                for (int t3 = S.tlo[2]; t3 <= S.thi[2]; ++t3) {
                    const double T1 = t1 * L1, T2 = t2 * L2, T3 = t3 * L3;
                    const double dx = x - S.R[0] - T1, dy = y - S.R[1] - T2, dz = z - S.R[2] - T3;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 >= S.rc * S.rc) continue;
                    double c = 1.0, sn = 0.0;
                    if (CPLX) sincos(k1 * T1 + k2 * T2 + k3 * T3, &sn, &c);
                    int p = 0;
                    for (int ch = 0; ch < S.nch; ++ch) {
                        double ylm[5];
                        solid_harmonics(S.l[ch], dx, dy, dz, ylm);
                        const double rad = S.N[ch] * exp(-r2 / (2.0 * S.rs[ch] * S.rs[ch]));
                        for (int m = 0; m < 2 * S.l[ch] + 1; ++m, ++p) {
                            re[p] += c * rad * ylm[m];
                            im[p] += sn * rad * ylm[m];
                        }
                    }
                }
        R* out = vals + (size_t)(CPLX ? 2 : 1) * (S.val_off + (size_t)(row - S.pt_off) * S.nproj);
        for (int p = 0; p < S.nproj; ++p) {
            if (CPLX) { out[2 * p] = (R)re[p]; out[2 * p + 1] = (R)im[p]; }
            else out[p] = (R)re[p];
        }
    }
}

// ---------------------------------------------------------------------------- gather
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if constexpr (sizeof(T) == 2 * sizeof(float) && !std::is_same<T, double>::value) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        } else if constexpr (std::is_same<T, double2>::value) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        } else {
            v += __shfl_xor_sync(0xffffffffu, v, o);
        }
    }
    return v;
}

// One warp per (work item, NC columns), GW warps per CTA on neighbouring column groups:
// lanes stride over the item's points, each lane keeps the NP x NC partial inner products in
// registers, and one warp-shuffle reduction per item produces the partial sums (no shared
// memory, no block barriers).  NP (the site's number of projectors) is a template argument so no lane
// multiplies padding.
template <typename T, typename D, int NP, int NC, int PTS>
__device__ __forceinline__ void gather_body(const T* __restrict__ X, int ld, int nc, int c0,
                                            const int* __restrict__ idx, const T* __restrict__ vp0,
                                            int first, int cnt, int lane, D* __restrict__ part,
                                            size_t pbase, int ncol) {
    T acc[NP][NC];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[p][j] = zero_of(T());
    // PTS points per lane and iteration (PTS times the independent loads in flight); the
    // grid indices of the next iteration are fetched one iteration ahead
    int l = lane;
    if (l + 32 * (PTS - 1) < cnt) {
        long gn[PTS];
#pragma unroll
        for (int q = 0; q < PTS; ++q) gn[q] = idx[first + l + 32 * q];
        for (; l + 32 * (PTS - 1) < cnt; l += 32 * PTS) {
            long gq[PTS];
#pragma unroll
            for (int q = 0; q < PTS; ++q) gq[q] = gn[q];
            if (l + 32 * PTS + 32 * (PTS - 1) < cnt) {
#pragma unroll
                for (int q = 0; q < PTS; ++q) gn[q] = idx[first + l + 32 * PTS + 32 * q];
            }
            T xq[PTS][NC];
#pragma unroll
            for (int q = 0; q < PTS; ++q)
#pragma unroll
                for (int j = 0; j < NC; ++j)
                    xq[q][j] = j < nc ? X[gq[q] + (size_t)(c0 + j) * ld] : zero_of(T());
#pragma unroll
            for (int q = 0; q < PTS; ++q) {
                const T* vq = vp0 + (size_t)(l + 32 * q) * NP;
                T pq[NP];
#pragma unroll
                for (int p = 0; p < NP; ++p) pq[p] = vq[p];
#pragma unroll
                for (int j = 0; j < NC; ++j)
#pragma unroll
                    for (int p = 0; p < NP; ++p) acc[p][j] = cfma_conj(pq[p], xq[q][j], acc[p][j]);
            }
        }
    }
    for (; l < cnt; l += 32) {
        const long g = idx[first + l];
        const T* vp = vp0 + (size_t)l * NP;
        T phi[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) phi[p] = vp[p];
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            if (j < nc) {
                const T x = X[g + (size_t)(c0 + j) * ld];
#pragma unroll
                for (int p = 0; p < NP; ++p) acc[p][j] = cfma_conj(phi[p], x, acc[p][j]);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const T v = warp_sum(acc[p][j]);
            if (lane == 0 && j < nc) {
                D d;
                if constexpr (sizeof(T) == sizeof(D) && std::is_same<T, D>::value) d = v;
                else if constexpr (std::is_same<D, double2>::value) d = make_double2((double)v.x, (double)v.y);
                else d = (double)v;
                part[pbase + (size_t)p * ncol + c0 + j] = d;
            }
        }
}

template <typename R, bool CPLX, int GW, int PTS, int NC>
__global__ void __launch_bounds__(GW * 32)
k_gather(const typename VT<R, CPLX>::T* __restrict__ X, int ld, int ncol,
         const SiteDev* __restrict__ sites, const int* __restrict__ items,
         const int* __restrict__ idx, const typename VT<R, CPLX>::T* __restrict__ vals,
         typename VT<double, CPLX>::T* __restrict__ part) {
    using T = typename VT<R, CPLX>::T;
    using D = typename VT<double, CPLX>::T;
    const int it = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = items[3 * it], first = items[3 * it + 1], cnt = items[3 * it + 2];
    const int np = sites[s].nproj;
    const int c0 = (blockIdx.y * GW + warp) * NC;
    if (c0 >= ncol) return;
    const int nc = min(NC, ncol - c0);
    const T* vp0 = vals + (size_t)sites[s].val_off + (size_t)(first - sites[s].pt_off) * np;
    const size_t pbase = (size_t)it * kMaxProj * ncol;
    switch (np) {
        case 1: gather_body<T, D, 1, NC, PTS>(X, ld, nc, c0, idx, vp0, first, cnt, lane, part, pbase, ncol); break;
        case 2: gather_body<T, D, 2, NC, PTS>(X, ld, nc, c0, idx, vp0, first, cnt, lane, part, pbase, ncol); break;
        case 3: gather_body<T, D, 3, NC, PTS>(X, ld, nc, c0, idx, vp0, first, cnt, lane, part, pbase, ncol); break;
        case 4: gather_body<T, D, 4, NC, PTS>(X, ld, nc, c0, idx, vp0, first, cnt, lane, part, pbase, ncol); break;
        case 5: gather_body<T, D, 5, NC, PTS>(X, ld, nc, c0, idx, vp0, first, cnt, lane, part, pbase, ncol); break;
        case 6: gather_body<T, D, 6, NC, PTS>(X, ld, nc, c0, idx, vp0, first, cnt, lane, part, pbase, ncol); break;
        case 7: gather_body<T, D, 7, NC, PTS>(X, ld, nc, c0, idx, vp0, first, cnt, lane, part, pbase, ncol); break;
        case 8: gather_body<T, D, 8, NC, PTS>(X, ld, nc, c0, idx, vp0, first, cnt, lane, part, pbase, ncol); break;
        case 9: gather_body<T, D, 9, NC, PTS>(X, ld, nc, c0, idx, vp0, first, cnt, lane, part, pbase, ncol); break;
        default: break;   // build_tables rejects sites with more than kMaxProj functions
    }
}

// W row of a site from its inner products c (KB: gamma C; Hubbard: M C, Eq. DerED)
template <typename R, bool CPLX>
__device__ __forceinline__ void site_transform(const SiteDev& S, const typename VT<double, CPLX>::T* c,
                                               const double* __restrict__ gamma, const double* __restrict__ M,
                                               typename VT<R, CPLX>::T* __restrict__ W, int n, int ncol) {
    using D = typename VT<double, CPLX>::T;
    using T = typename VT<R, CPLX>::T;
    for (int p = 0; p < S.nproj; ++p) {
        D w = zero_of(D());
        if (S.kind == 0) {
            w = mulr(gamma[S.proj_off + p], c[p]);
        } else {
            // coefficient of phi_p: sum_m M[p][m] C_m  (M = (U/2)(I - 2D))
            for (int m = 0; m < S.nproj; ++m) {
                D mm;
                if constexpr (CPLX) {
                    const double* Mi = M + (size_t)S.hub_index * 50;
                    mm = make_double2(Mi[2 * (p * 5 + m)], Mi[2 * (p * 5 + m) + 1]);
                } else {
                    mm = M[(size_t)S.hub_index * 25 + p * 5 + m];
                }
                w = cfma(mm, c[m], w);
            }
        }
        T wv;
        if constexpr (CPLX) wv = T{(R)w.x, (R)w.y};
        else wv = (R)w;
        W[(size_t)(S.proj_off + p) * ncol + n] = wv;
    }
}

// brick form: C of each projector row from its float partials over bricks.  One CTA per
// (row, 128 orbitals): warp w sums the row's partial rows w, w + 8, ..., each lane 4 orbitals
// 32 apart, in compensated float sums (Kahan: the rounding error of every addition is carried
// in a second float, so the sum keeps close to double accuracy on the FP32 pipe, which GB300
// runs far faster than its FP64 pipe); the eight warp sums are added in double in a fixed
// order.
constexpr int RR_COLS = 128;
__global__ void __launch_bounds__(256)
k_reduce_rows_dense(int ncol, double dV, const int* __restrict__ roff, const int* __restrict__ rent,
                    const float* __restrict__ part, double* __restrict__ C) {
    __shared__ double red[8][RR_COLS];
    const int r = blockIdx.x;
    const int n0 = blockIdx.y * RR_COLS;
    const int e0 = roff[r], e1 = roff[r + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int e = e0 + w; e < e1; e += 8) {
        const float* src = part + (size_t)rent[e] * ncol + n0 + lane;
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (n0 + lane + 32 * k < ncol) ? src[32 * k] : 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float y = v[k] - c[k];
            const float t = s[k] + y;
            c[k] = (t - s[k]) - y;
            s[k] = t;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) red[w][lane + 32 * k] = (double)s[k] - (double)c[k];
    __syncthreads();
    if (threadIdx.x < RR_COLS && n0 + (int)threadIdx.x < ncol) {
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += red[k][threadIdx.x];
        C[(size_t)r * ncol + n0 + threadIdx.x] = dV * sum;
    }
}

__global__ void k_transform_sites(int nsites, int ncol, const SiteDev* __restrict__ sites,
                                  const double* __restrict__ C, const double* __restrict__ gamma,
                                  const double* __restrict__ M, float* __restrict__ W) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nsites * ncol) return;
    const int s = (int)(t / ncol), n = (int)(t - (long)s * ncol);
    const SiteDev S = sites[s];
    double c[kMaxProj];
    for (int p = 0; p < S.nproj; ++p) c[p] = C[(size_t)(S.proj_off + p) * ncol + n];
    site_transform<float, false>(S, c, gamma, M, W, n, ncol);
}

// reduce partials of each site and apply the coefficient transform
template <typename R, bool CPLX>
__global__ void k_reduce_transform(int nsites, int ncol, double dV, const SiteDev* __restrict__ sites,
                                   const int* __restrict__ item_first,
                                   const typename VT<double, CPLX>::T* __restrict__ part,
                                   const double* __restrict__ gamma, const double* __restrict__ M,
                                   typename VT<double, CPLX>::T* __restrict__ C,
                                   typename VT<R, CPLX>::T* __restrict__ W, int want_W) {
    using D = typename VT<double, CPLX>::T;
    using T = typename VT<R, CPLX>::T;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nsites * ncol) return;
    const int s = (int)(t / ncol), n = (int)(t - (long)s * ncol);
    const SiteDev S = sites[s];
    D c[kMaxProj];
    for (int p = 0; p < S.nproj; ++p) {
        D acc = zero_of(D());
        for (int it = item_first[s]; it < item_first[s + 1]; ++it)
            acc = add(acc, part[((size_t)it * kMaxProj + p) * ncol + n]);
        c[p] = mulr(dV, acc);
        C[(size_t)(S.proj_off + p) * ncol + n] = c[p];
    }
    if (want_W) site_transform<R, CPLX>(S, c, gamma, M, W, n, ncol);
}

// ---------------------------------------------------------------------------- scatter
// One thread per grid point that carries entries, taken in the scatter order (points grouped
// by the list of sites touching them, so that a warp's lanes run the same loops and read the
// same W rows), looping over all columns NC at a time: the point's CSR entries and values are
// fetched from HBM once and re-read from L1 for the later column groups.  Per entry, the
// site's values multiply W rows (16-byte vector loads when the rows are aligned); Y is
// updated once per column.
template <typename R, bool CPLX>
__global__ void __launch_bounds__(128)
k_scatter(typename VT<R, CPLX>::T* __restrict__ Y, int ld, int ncol, int norder,
          const int* __restrict__ order, const int* __restrict__ csr_off, const int2* __restrict__ csr_ent,
          const typename VT<R, CPLX>::T* __restrict__ vals,
          const typename VT<R, CPLX>::T* __restrict__ W, R alpha, int vec_ok,
          const double* __restrict__ alpha_dev) {
    using T = typename VT<R, CPLX>::T;
    if (alpha_dev) alpha = (R)alpha_dev[0];
    // columns per group: 64 bytes of a W row; complex float takes 16 columns (128 bytes):
    // rutile complex block 3.11 -> 2.83 ms
    constexpr int NC = (CPLX && sizeof(R) == 4) ? 16 : 64 / (int)sizeof(T);
    constexpr int PER16 = 16 / sizeof(T);
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= norder) return;
    const long g = order[i];
    const int e0 = csr_off[g], e1 = csr_off[g + 1];
    for (int c0 = 0; c0 < ncol; c0 += NC) {
        const int nc = min(NC, ncol - c0);
        T acc[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = zero_of(T());
        int2 m = csr_ent[e0];
        for (int e = e0; e < e1; ++e) {
            const int2 mn = (e + 1 < e1) ? csr_ent[e + 1] : m;      // next entry, in flight early
            const int np = m.y & 15;
            const T* wrow = W + (size_t)(m.y >> 4) * ncol + c0;
            const T* vrow = vals + m.x;
            for (int p = 0; p < np; ++p, wrow += ncol) {
                const T v = vrow[p];
                if (vec_ok && nc == NC) {
                    float4 q4[NC / PER16];
#pragma unroll
                    for (int k = 0; k < NC / PER16; ++k) q4[k] = reinterpret_cast<const float4*>(wrow)[k];
#pragma unroll
                    for (int k = 0; k < NC / PER16; ++k) {
                        const T* w = reinterpret_cast<const T*>(&q4[k]);
#pragma unroll
                        for (int i = 0; i < PER16; ++i) acc[k * PER16 + i] = cfma(v, w[i], acc[k * PER16 + i]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < NC; ++j)
                        if (j < nc) acc[j] = cfma(v, wrow[j], acc[j]);
                }
            }
            m = mn;
        }
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            if (j < nc) {
                T* y = Y + (size_t)(c0 + j) * ld + g;
                *y = fmar(alpha, acc[j], *y);
            }
        }
    }
}

// ---------------------------------------------------------------------------- brick form
// Real float only.  The grid is cut into bricks of 8 x 8 x 4 points (32 rows of 8 along x;
// point p = x + 8 row, row = y + 8 z inside the brick).  Every brick lists the functions of
// the sites that touch it, in entries of at most 64 (a site's functions stay together, fp =
// their count rounded up to 4), and keeps their values as a dense block [fp][256]
// (function-major, points in brick_slot order), zero where a function vanishes.
// Both directions then become small dense products per brick:
//   gather:  part[prow + f, n] = sum_p phi[p, f] X[g(p), n]    (partial inner products,
//            summed per function over its bricks by k_reduce_transform_dense)
//   scatter: Y[g(p), n] += alpha sum_f phi[p, f] W[frow[f], n]
// with every X and Y element read once per brick and pass, in 16-byte rows.
constexpr int GD_COLS = 32, GD_XS = GD_COLS + 4;     // gather: columns per pass, smem row stride
constexpr int SD_COLS = 32;                          // scatter: columns per pass


__global__ void k_brick_fill(int npts, const int2* __restrict__ rowinfo, const SiteDev* __restrict__ sites,
                             const float* __restrict__ vals, float* __restrict__ phi) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= npts) return;
    const int2 ri = rowinfo[r];
    const int np = sites[ri.y].nproj;
    const size_t v0 = (size_t)sites[ri.y].val_off + (size_t)(r - sites[ri.y].pt_off) * np;
    for (int p = 0; p < np; ++p) phi[ri.x + (size_t)p * BRP] = vals[v0 + p];
}

__device__ __forceinline__ long brick_point(int b, int nbx, int nby, int p, int n1, int n2, int n3, bool* ok) {
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int row = p >> 3;
    const int x = bx * BRX + (p & 7), y = by * BRY + (row & 7), z = bz * BRZ + (row >> 3);
    *ok = x < n1 && y < n2 && z < n3;
    return x + (long)n1 * (y + (long)n2 * z);
}

// one CTA per (entry, 32 columns): 128 threads = 16 function groups of 4 x 8 column groups
// of 4.  The X tile is staged point-major in shared memory; values are read as float4 rows
// from L1 (the entry's block is shared by the CTA's warps).
__global__ void __launch_bounds__(128)
k_gather_dense(const float* __restrict__ X, int ld, int ncol, int n1, int n2, int n3, int nbx, int nby,
               const int4* __restrict__ bent, const float* __restrict__ phi, float* __restrict__ part) {
    __shared__ __align__(16) float xs[BRP * GD_XS];
    const int4 E = bent[blockIdx.x];
    const int fp = E.y;
    const int c0 = blockIdx.y * GD_COLS;
    // X tile: 32 columns x 32 rows of 8 points (two 16-byte loads, one whole sector, per
    // thread; consecutive threads take consecutive columns, so the transposing stores into
    // the point-major tile hit distinct banks)
    for (int i = threadIdx.x; i < GD_COLS * 32; i += blockDim.x) {
        const int c = i & (GD_COLS - 1), row = i / GD_COLS;
        const int p = row * 8;
        bool ok0, ok1;
        const long g = brick_point(E.x, nbx, nby, p, n1, n2, n3, &ok0);
        brick_point(E.x, nbx, nby, p + 4, n1, n2, n3, &ok1);
        float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
        if (c0 + c < ncol) {
            const float* src = X + (size_t)(c0 + c) * ld + g;
            if (ok0) va = *reinterpret_cast<const float4*>(src);
            if (ok1) vb = *reinterpret_cast<const float4*>(src + 4);
        }
        const float v[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) xs[(p + k) * GD_XS + c] = v[k];
    }
    __syncthreads();
    const int fg = threadIdx.x >> 3, cg = threadIdx.x & 7;
    if (fg * 4 >= fp) return;
    const float* ph = phi + E.z + (size_t)fg * 4 * BRP;
    float acc[4][4] = {};
#pragma unroll 4
    for (int p = 0; p < BRP; ++p) {
        const float4 x = *reinterpret_cast<const float4*>(xs + p * GD_XS + cg * 4);
        const int q = brick_slot(p);
        const float fv[4] = {ph[q], ph[BRP + q], ph[2 * BRP + q], ph[3 * BRP + q]}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[k][j] = fmaf(fv[k], xv[j], acc[k][j]);
    }
    const int cb = c0 + cg * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float* out = part + (size_t)(E.w + fg * 4 + k) * ncol;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (cb + j < ncol) out[cb + j] = acc[k][j];
    }
}

// one CTA per brick, looping over the columns SD_COLS at a time: 256 threads = 8 column
// groups (of 4) x 32 rows (of 8 points).  Values are read from global memory function-major
// (each half row is 16 bytes, and a warp's 32 rows of one half are 512 contiguous bytes; the
// entry's block stays in L1/L2 over the passes), W rows of the pass are staged in shared
// memory and read as one broadcast per warp.
// (Measured on the rutile workload, this beat packed f32x2 FMAs, a 4-row x 8-group warp
// mapping, and staging the values in shared memory.)
__global__ void __launch_bounds__(256, 3)
k_scatter_dense(float* __restrict__ Y, int ld, int ncol, int n1, int n2, int n3, int nbx, int nby,
                const int4* __restrict__ bent, const int* __restrict__ bfirst, const float* __restrict__ phi,
                const int* __restrict__ frow, const float* __restrict__ W, float alpha,
                const double* __restrict__ alpha_dev) {
    __shared__ __align__(16) float ws[BRF * SD_COLS];
    if (alpha_dev) alpha = (float)alpha_dev[0];
    const int e0 = bfirst[blockIdx.x], e1 = bfirst[blockIdx.x + 1];
    const int b = bent[e0].x;
    const int cg = threadIdx.x >> 5, row = threadIdx.x & 31;
    bool ok0, ok1;
    const long g0 = brick_point(b, nbx, nby, row * 8, n1, n2, n3, &ok0);
    brick_point(b, nbx, nby, row * 8 + 4, n1, n2, n3, &ok1);
    for (int c0 = 0; c0 < ncol; c0 += SD_COLS) {
        float acc[8][4] = {};
        for (int e = e0; e < e1; ++e) {
            const int4 E = bent[e];
            const int fp = E.y;
            __syncthreads();                       // previous pass / entry fully read
            for (int i = threadIdx.x; i < fp * SD_COLS; i += blockDim.x) {
                const int f = i / SD_COLS, c = i - f * SD_COLS;
                const int r = frow[E.w + f];
                ws[i] = (r >= 0 && c0 + c < ncol) ? W[(size_t)r * ncol + c0 + c] : 0.f;
            }
            __syncthreads();
            const float* ph = phi + E.z + row * 4;
            // the eight column groups start at staggered functions (each sums its functions
            // in a fixed rotated order), so that the warps do not request the same value
            // lines at the same time: L1 then serves most of them (rutile: 0.98 -> 0.87 ms)
            const int fs = (cg * fp) >> 3;
#pragma unroll 4
            for (int i = 0; i < fp; ++i) {
                const int f = i + fs < fp ? i + fs : i + fs - fp;
                const float4 pa = __ldg(reinterpret_cast<const float4*>(ph + (size_t)f * BRP));
                const float4 pb = __ldg(reinterpret_cast<const float4*>(ph + (size_t)f * BRP + 128));
                const float4 w4 = *reinterpret_cast<const float4*>(ws + f * SD_COLS + cg * 4);
                const float pv[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
                const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(pv[i], wv[j], acc[i][j]);
            }
        }
        float4 ya[4], yb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + cg * 4 + j;
            const float* y = Y + (size_t)c * ld + g0;
            ya[j] = (ok0 && c < ncol) ? *reinterpret_cast<const float4*>(y) : make_float4(0.f, 0.f, 0.f, 0.f);
            yb[j] = (ok1 && c < ncol) ? *reinterpret_cast<const float4*>(y + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + cg * 4 + j;
            float* y = Y + (size_t)c * ld + g0;
            if (ok0 && c < ncol) {
                float4 v = ya[j];
                v.x = fmaf(alpha, acc[0][j], v.x); v.y = fmaf(alpha, acc[1][j], v.y);
                v.z = fmaf(alpha, acc[2][j], v.z); v.w = fmaf(alpha, acc[3][j], v.w);
                *reinterpret_cast<float4*>(y) = v;
            }
            if (ok1 && c < ncol) {
                float4 v = yb[j];
                v.x = fmaf(alpha, acc[4][j], v.x); v.y = fmaf(alpha, acc[5][j], v.y);
                v.z = fmaf(alpha, acc[6][j], v.z); v.w = fmaf(alpha, acc[7][j], v.w);
                *reinterpret_cast<float4*>(y + 4) = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------- occupation
template <bool CPLX>
__global__ void k_occupation(int ncol, const SiteDev* __restrict__ sites, const int* __restrict__ hub_sites,
                             const typename VT<double, CPLX>::T* __restrict__ C,
                             const double* __restrict__ f, double kweight,
                             double* __restrict__ D, double* __restrict__ eu, const double* __restrict__ U) {
    using Dt = typename VT<double, CPLX>::T;
    const int hsite = blockIdx.x;
    const SiteDev S = sites[hub_sites[hsite]];
    __shared__ double red[25][2][33];
    double are[25], aim[25];
    for (int q = 0; q < 25; ++q) { are[q] = 0.0; aim[q] = 0.0; }
    for (int n = threadIdx.x; n < ncol; n += blockDim.x) {
        Dt c[5];
        for (int m = 0; m < 5; ++m) c[m] = C[(size_t)(S.proj_off + m) * ncol + n];
        const double fn = f[n];
        for (int m = 0; m < 5; ++m)
            for (int mp = 0; mp < 5; ++mp) {
                // D_mm' += f_n C_m conj(C_m')
                if constexpr (CPLX) {
                    are[m * 5 + mp] += fn * (c[m].x * c[mp].x + c[m].y * c[mp].y);
                    aim[m * 5 + mp] += fn * (c[m].y * c[mp].x - c[m].x * c[mp].y);
                } else {
                    are[m * 5 + mp] += fn * c[m] * c[mp];
                }
            }
    }
    // deterministic block reduction: warp shuffles, then warp 0 over the warps
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = 0; q < 25; ++q) {
        double vr = are[q], vi = aim[q];
        for (int o = 16; o > 0; o >>= 1) {
            vr += __shfl_down_sync(0xffffffffu, vr, o);
            vi += __shfl_down_sync(0xffffffffu, vi, o);
        }
        if (lane == 0) { red[q][0][wid] = vr; red[q][1][wid] = vi; }
    }
    __syncthreads();
    __shared__ double Dm[25][2];
    if (threadIdx.x < 25) {
        double vr = 0.0, vi = 0.0;
        for (int w = 0; w < nw; ++w) { vr += red[threadIdx.x][0][w]; vi += red[threadIdx.x][1][w]; }
        Dm[threadIdx.x][0] = kweight * vr;
        Dm[threadIdx.x][1] = kweight * vi;
        D[(size_t)hsite * 50 + 2 * threadIdx.x] = kweight * vr;
        D[(size_t)hsite * 50 + 2 * threadIdx.x + 1] = kweight * vi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // E_U contribution (U/2) Tr(D - D^2); Tr(D^2) = sum_mm' D_mm' D_m'm
        double tr = 0.0, tr2 = 0.0;
        for (int m = 0; m < 5; ++m) {
            tr += Dm[m * 5 + m][0];
            for (int mp = 0; mp < 5; ++mp)
                tr2 += Dm[m * 5 + mp][0] * Dm[mp * 5 + m][0] - Dm[m * 5 + mp][1] * Dm[mp * 5 + m][1];
        }
        eu[hsite] = 0.5 * U[hsite] * (tr - tr2);
    }
}

// ---------------------------------------------------------------------------- forces
// Hubbard force component `axis` of each Hubbard atom (Sec. II.A.3, final force equation):
//   F = Re sum_mm' U (2 D_m'm - delta_mm') kweight sum_n f_n conj(G_m'n) C_mn
//     = -2 kweight Re sum_n f_n sum_m' conj(G_m'n) W_m'n,   W = M C,  M = (U/2)(I - 2D)
// with C_mn = <phi_m|x_n> and G_m'n = <phi_m'|d_axis x_n>.  One CTA per Hubbard atom, a
// deterministic reduction over the columns.
template <bool CPLX>
__global__ void k_hub_force(int ncol, const SiteDev* __restrict__ sites, const int* __restrict__ hub_sites,
                            const typename VT<double, CPLX>::T* __restrict__ C,
                            const typename VT<double, CPLX>::T* __restrict__ G,
                            const double* __restrict__ f, double kweight, const double* __restrict__ M,
                            int axis, double* __restrict__ F) {
    using Dt = typename VT<double, CPLX>::T;
    const int hsite = blockIdx.x;
    const SiteDev S = sites[hub_sites[hsite]];
    __shared__ double Ms[25][2];
    __shared__ double red[32];
    if (threadIdx.x < 25) {
        if constexpr (CPLX) {
            Ms[threadIdx.x][0] = M[((size_t)hsite * 25 + threadIdx.x) * 2];
            Ms[threadIdx.x][1] = M[((size_t)hsite * 25 + threadIdx.x) * 2 + 1];
        } else {
            Ms[threadIdx.x][0] = M[(size_t)hsite * 25 + threadIdx.x];
            Ms[threadIdx.x][1] = 0.0;
        }
    }
    __syncthreads();
    double acc = 0.0;
    for (int n = threadIdx.x; n < ncol; n += blockDim.x) {
        Dt c[5];
        for (int m = 0; m < 5; ++m) c[m] = C[(size_t)(S.proj_off + m) * ncol + n];
        double s = 0.0;
        for (int p = 0; p < 5; ++p) {
            const Dt g = G[(size_t)(S.proj_off + p) * ncol + n];
            if constexpr (CPLX) {
                double wr = 0.0, wi = 0.0;       // W_p = sum_m M_pm C_m
                for (int m = 0; m < 5; ++m) {
                    wr += Ms[p * 5 + m][0] * c[m].x - Ms[p * 5 + m][1] * c[m].y;
                    wi += Ms[p * 5 + m][0] * c[m].y + Ms[p * 5 + m][1] * c[m].x;
                }
                s += g.x * wr + g.y * wi;        // Re(conj(g) W)
            } else {
                double w = 0.0;
                for (int m = 0; m < 5; ++m) w += Ms[p * 5 + m][0] * c[m];
                s += g * w;
            }
        }
        acc += f[n] * s;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red[w];
        F[(size_t)hsite * 3 + axis] = -2.0 * kweight * t;
    }
}

// ---------------------------------------------------------------------------- stress moments
// Moment integrals of the Hubbard stress (Sec. II.A.4) for one gradient block G = d_a X:
//   Gm_b[(proj_off + m) * ncol + n] = dV sum_points conj(mom_bm(g)) G[g, n],   b = x, y, z,
//   mom_bm(g) = sum_T phi_m(x_g - R - T) (x_g - R - T)_b exp(i k.T),
// the moment about each periodic image's own centre.  The image sum is evaluated again here
// (the tables hold only its total).  One CTA per (Hubbard atom, column); threads stride over
// the atom's table points; a block reduction of the 15 (complex) sums.
template <typename T, bool CPLX>
__global__ void __launch_bounds__(256)
k_moment_gather(const T* __restrict__ G, int ld, int ncol, const SiteDev* __restrict__ sites,
                const int* __restrict__ hub_sites, const int* __restrict__ idx, int n1, int n2,
                double h1, double h2, double h3, double L1, double L2, double L3, double k1, double k2,
                double k3, double dV, double* __restrict__ Gm0, double* __restrict__ Gm1,
                double* __restrict__ Gm2) {
    constexpr int CW = CPLX ? 2 : 1;
    const SiteDev S = sites[hub_sites[blockIdx.x]];
    const int n = blockIdx.y;
    double acc[3][5][CW];
    for (int b = 0; b < 3; ++b)
        for (int m = 0; m < 5; ++m)
            for (int c = 0; c < CW; ++c) acc[b][m][c] = 0.0;
    for (int row = S.pt_off + threadIdx.x; row < S.pt_off + S.npts; row += blockDim.x) {
        const int g = idx[row];
        const int i1 = g % n1, i2 = (g / n1) % n2, i3 = g / (n1 * n2);
        const double x = i1 * h1, y = i2 * h2, z = i3 * h3;
        const T gv = G[(long)n * ld + g];
        double gr, gi = 0.0;
        if constexpr (CPLX) { gr = gv.x; gi = gv.y; } else { gr = (double)gv; }
        for (int t1 = S.tlo[0]; t1 <= S.thi[0]; ++t1)
            for (int t2 = S.tlo[1]; t2 <= S.thi[1]; ++t2)
                for (int t3 = S.tlo[2]; t3 <= S.thi[2]; ++t3) {
                    const double T1 = t1 * L1, T2 = t2 * L2, T3 = t3 * L3;
                    const double d[3] = {x - S.R[0] - T1, y - S.R[1] - T2, z - S.R[2] - T3};
                    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 >= S.rc * S.rc) continue;
                    double c = 1.0, sn = 0.0;
                    if (CPLX) sincos(k1 * T1 + k2 * T2 + k3 * T3, &sn, &c);
                    double ylm[5];
                    solid_harmonics(2, d[0], d[1], d[2], ylm);
                    const double rad = S.N[0] * exp(-r2 / (2.0 * S.rs[0] * S.rs[0]));
                    // conj(phi_m d_b e^{i k.T}) * g, accumulated per (b, m)
                    const double pr = c * gr + sn * gi, pi = c * gi - sn * gr;
#pragma unroll
                    for (int m = 0; m < 5; ++m) {
                        const double v = rad * ylm[m];
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            acc[b][m][0] += v * d[b] * pr;
                            if constexpr (CPLX) acc[b][m][CW - 1] += v * d[b] * pi;
                        }
                    }
                }
    }
    __shared__ double red[8][3 * 5 * CW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b = 0; b < 3; ++b)
        for (int m = 0; m < 5; ++m)
            for (int c = 0; c < CW; ++c) {
                double v = acc[b][m][c];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) red[wid][(b * 5 + m) * CW + c] = v;
            }
    __syncthreads();
    if (threadIdx.x < 3 * 5 * CW) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
        const int b = threadIdx.x / (5 * CW), m = (threadIdx.x / CW) % 5, c = threadIdx.x % CW;
        double* out = b == 0 ? Gm0 : (b == 1 ? Gm1 : Gm2);
        out[((size_t)(S.proj_off + m) * ncol + n) * CW + c] = dV * v;
    }
}

__global__ void k_sum_serial(const double* __restrict__ x, int n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += x[i];
        *out = s;
    }
}

double radial_norm(int l, double rs) {
    return std::sqrt(2.0 / (std::tgamma(l + 1.5) * std::pow(rs, 2 * l + 3)));
}

template <typename Tp>
int upload(hub_t h, Tp** dptr, const std::vector<Tp>& v) {
    if (*dptr) { cudaFree(*dptr); *dptr = nullptr; }
    if (v.empty()) return HUB_OK;
    HUB_CUDA_TRY(h, cudaMalloc((void**)dptr, v.size() * sizeof(Tp)));
    HUB_CUDA_TRY(h, cudaMemcpy(*dptr, v.data(), v.size() * sizeof(Tp), cudaMemcpyHostToDevice));
    return HUB_OK;
}

}  // namespace

// ---------------------------------------------------------------------------- host side

void free_table(Table& t) {
    void* ptrs[] = {t.d_sites, t.d_items, t.d_item_first, t.d_idx, t.d_vals, t.d_csr_off,
                    t.d_csr_ent, t.d_order, t.d_gamma, t.d_hub_sites, t.d_U,
                    t.d_M[0], t.d_M[1], t.d_bent, t.d_bfirst, t.d_phi, t.d_frow, t.d_roff,
                    t.d_rent, t.d_tcg, t.d_tcg_row, t.d_tchi, t.d_tclo, t.d_tcs_brick, t.d_tcs_frow, t.d_tcs_hi,
                    t.d_tcs_lo};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    t = Table();
}

static int floordiv_host(double a) { return (int)std::floor(a); }

// Brick form of the tables (real float working type, n1 a multiple of 4): entries, dense
// values copied from the point-major table, and the reduction lists of the gather.
static int build_bricks(hub_t h, Table& t, const std::vector<std::vector<int>>& site_pts) {
    const int n1 = h->n1, n2 = h->n2;
    t.nbx = (h->n1 + BRX - 1) / BRX;
    t.nby = (h->n2 + BRY - 1) / BRY;
    t.nbz = (h->n3 + BRZ - 1) / BRZ;
    const long nb = (long)t.nbx * t.nby * t.nbz;
    auto brick_of = [&](int g) -> long {
        const int x = g % n1, y = (g / n1) % n2, z = g / (n1 * n2);
        return x / BRX + t.nbx * (y / BRY + (long)t.nby * (z / BRZ));
    };
    auto point_in = [&](int g) -> int {
        const int x = g % n1, y = (g / n1) % n2, z = g / (n1 * n2);
        return (x % BRX) + BRX * ((y % BRY) + BRY * (z % BRZ));
    };
    std::vector<std::vector<int>> bs(nb);           // sites touching each brick, ascending
    for (int s = 0; s < t.nsites; ++s) {
        std::vector<long> bl;
        bl.reserve(site_pts[s].size());
        for (int g : site_pts[s]) bl.push_back(brick_of(g));
        std::sort(bl.begin(), bl.end());
        bl.erase(std::unique(bl.begin(), bl.end()), bl.end());
        for (long b : bl) bs[b].push_back(s);
    }
    std::vector<int4> bent;
    std::vector<int> bfirst, frow;
    std::unordered_map<long long, std::pair<int, int>> where;   // (site, brick) -> entry, offset
    long phi_off = 0, prow = 0;
    for (long b = 0; b < nb; ++b) {
        const std::vector<int>& L = bs[b];
        if (L.empty()) continue;
        bfirst.push_back((int)bent.size());
        size_t i = 0;
        while (i < L.size()) {
            int f = 0;
            size_t j = i;
            const int e = (int)bent.size();
            while (j < L.size() && f + t.h_sites[L[j]].nproj <= BRF) {
                where[(long long)L[j] * nb + b] = {e, f};
                f += t.h_sites[L[j]].nproj;
                ++j;
            }
            const int fp = (f + 3) & ~3;
            bent.push_back(make_int4((int)b, fp, (int)phi_off, (int)prow));
            for (size_t k = i; k < j; ++k)
                for (int q = 0; q < t.h_sites[L[k]].nproj; ++q) frow.push_back(t.h_sites[L[k]].proj_off + q);
            for (int q = f; q < fp; ++q) frow.push_back(-1);
            phi_off += (long)fp * BRP;
            prow += fp;
            if (phi_off >= (1L << 31) || prow >= (1L << 31)) return HUB_OK;    // stay point-major
            i = j;
        }
    }
    bfirst.push_back((int)bent.size());
    std::vector<int2> rowinfo(t.npts);
    for (int s = 0; s < t.nsites; ++s) {
        const SiteDev& S = t.h_sites[s];
        for (int l = 0; l < S.npts; ++l) {
            const int g = site_pts[s][l];
            const auto& w = where.at((long long)s * nb + brick_of(g));
            const int4& E = bent[w.first];
            rowinfo[S.pt_off + l] = make_int2(E.z + w.second * BRP + brick_slot(point_in(g)), s);
        }
    }
    std::vector<int> roff(t.nproj + 1, 0), rent(prow);
    for (long r = 0; r < prow; ++r)
        if (frow[r] >= 0) roff[frow[r] + 1]++;
    for (int r = 0; r < t.nproj; ++r) roff[r + 1] += roff[r];
    {
        std::vector<int> fill(roff.begin(), roff.end() - 1);
        for (long r = 0; r < prow; ++r)
            if (frow[r] >= 0) rent[fill[frow[r]]++] = (int)r;
    }
    int rc;
    int2* d_rowinfo = nullptr;
    if ((rc = upload(h, &t.d_bent, bent))) return rc;
    if ((rc = upload(h, &t.d_bfirst, bfirst))) return rc;
    if ((rc = upload(h, &t.d_frow, frow))) return rc;
    if ((rc = upload(h, &t.d_roff, roff))) return rc;
    if ((rc = upload(h, &t.d_rent, rent))) return rc;
    if ((rc = upload(h, &d_rowinfo, rowinfo))) return rc;
    HUB_CUDA_TRY(h, cudaMalloc((void**)&t.d_phi, (size_t)phi_off * sizeof(float)));
    HUB_CUDA_TRY(h, cudaMemsetAsync(t.d_phi, 0, (size_t)phi_off * sizeof(float), h->stream));
    {
        ProfScope ps(h, HUB_K_TABLE);
        k_brick_fill<<<(t.npts + 255) / 256, 256, 0, h->stream>>>(t.npts, d_rowinfo, t.d_sites,
                                                                (const float*)t.d_vals, t.d_phi);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    cudaFree(d_rowinfo);
    t.nbent = (int)bent.size();
    t.nbused = (int)bfirst.size() - 1;
    t.npart_rows = prow;
    t.dense = 1;
    return build_tc_tables(h, t);
}

int build_tables(hub_t h, int natoms, const double* pos, const int* kb_nchan, const int* kb_l,
                 const double* kb_rs, const double* kb_gamma, const double* kb_rc,
                 const int* hub_l, const double* hub_rs, const double* hub_rc,
                 const double* hub_U) {
    Table t;
    const int n[3] = {h->n1, h->n2, h->n3};
    std::vector<std::vector<int>> site_pts;
    std::vector<double> gamma_rows;
    int ch_base = 0;
    for (int a = 0; a < natoms; ++a) {
        const double* R = pos + 3 * a;
        const int nch = kb_nchan ? kb_nchan[a] : 0;
        for (int kind = 0; kind < 2; ++kind) {
            SiteDev S{};
            S.R[0] = R[0]; S.R[1] = R[1]; S.R[2] = R[2];
            S.hub_index = -1;
            S.kind = kind;
            if (kind == 0) {
                if (nch <= 0) continue;
                if (nch > 3) return fail(h, HUB_EINVAL, "at most 3 KB channels per atom");
                S.rc = kb_rc[a];
                S.nch = nch;
                for (int c = 0; c < nch; ++c) {
                    S.l[c] = kb_l[ch_base + c];
                    S.rs[c] = kb_rs[ch_base + c];
                    if (S.l[c] < 0 || S.l[c] > 2 || S.rs[c] <= 0)
                        return fail(h, HUB_EINVAL, "KB channel needs 0 <= l <= 2 and rs > 0");
                    S.N[c] = radial_norm(S.l[c], S.rs[c]);
                }
            } else {
                if (!hub_l || hub_l[a] < 0) continue;
                if (hub_l[a] != 2) return fail(h, HUB_EINVAL, "only d (l = 2) Hubbard shells");
                S.rc = hub_rc[a];
                S.nch = 1;
                S.l[0] = 2;
                S.rs[0] = hub_rs[a];
                if (S.rs[0] <= 0) return fail(h, HUB_EINVAL, "Hubbard rs must be > 0");
                S.N[0] = radial_norm(2, hub_rs[a]);
                S.hub_index = (int)t.h_U.size();
                t.h_U.push_back(hub_U[a]);
                t.h_hub_sites.push_back((int)t.h_sites.size());
                t.h_hub_atom.push_back(a);
            }
            if (!(S.rc > 0)) return fail(h, HUB_EINVAL, "cutoff radius must be > 0");
            int np = 0;
            for (int c = 0; c < S.nch; ++c) np += 2 * S.l[c] + 1;
            if (np > kMaxProj) return fail(h, HUB_EINVAL, "at most 9 functions per atom and kind");
            S.nproj = np;
            // grid points within rc of any lattice image R + T
            std::vector<int> pts;
            int tlo[3], thi[3], tmin[3] = {1 << 30, 1 << 30, 1 << 30}, tmax[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
            for (int ax = 0; ax < 3; ++ax) {
                tlo[ax] = floordiv_host((-R[ax] - S.rc) / h->L[ax]) - 1;
                thi[ax] = floordiv_host((h->L[ax] - R[ax] + S.rc) / h->L[ax]) + 1;
            }
            for (int t1 = tlo[0]; t1 <= thi[0]; ++t1)
                for (int t2 = tlo[1]; t2 <= thi[1]; ++t2)
                    for (int t3 = tlo[2]; t3 <= thi[2]; ++t3) {
                        const int tt[3] = {t1, t2, t3};
                        double c[3];
                        int lo[3], hi[3];
                        bool empty = false;
                        for (int ax = 0; ax < 3; ++ax) {
                            c[ax] = R[ax] + tt[ax] * h->L[ax];
                            lo[ax] = std::max((int)std::ceil((c[ax] - S.rc) / h->h[ax]), 0);
                            hi[ax] = std::min((int)std::floor((c[ax] + S.rc) / h->h[ax]), n[ax] - 1);
                            if (hi[ax] < lo[ax]) empty = true;
                        }
                        if (empty) continue;
                        bool any = false;
                        for (int k3 = lo[2]; k3 <= hi[2]; ++k3) {
                            const double dz = k3 * h->h[2] - c[2];
                            for (int k2 = lo[1]; k2 <= hi[1]; ++k2) {
                                const double dy = k2 * h->h[1] - c[1];
                                for (int k1 = lo[0]; k1 <= hi[0]; ++k1) {
                                    const double dx = k1 * h->h[0] - c[0];
                                    if (dx * dx + dy * dy + dz * dz < S.rc * S.rc) {
                                        pts.push_back(k1 + n[0] * (k2 + n[1] * k3));
                                        any = true;
                                    }
                                }
                            }
                        }
                        if (any)
                            for (int ax = 0; ax < 3; ++ax) {
                                tmin[ax] = std::min(tmin[ax], tt[ax]);
                                tmax[ax] = std::max(tmax[ax], tt[ax]);
                            }
                    }
            std::sort(pts.begin(), pts.end());
            pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
            if (pts.empty()) continue;   // cannot happen for rc > 0 and a grid inside the cell
            for (int ax = 0; ax < 3; ++ax) { S.tlo[ax] = tmin[ax]; S.thi[ax] = tmax[ax]; }
            S.npts = (int)pts.size();
            S.pt_off = t.npts;
            S.val_off = t.nvals;
            S.proj_off = t.nproj;
            if ((long)t.nvals + (long)S.npts * np > 2000000000L)
                return fail(h, HUB_EINVAL, "projector tables exceed 2^31 values");
            t.npts += S.npts;
            t.nvals += S.npts * np;
            t.nproj += np;
            for (int c = 0; c < S.nch; ++c)
                for (int m = 0; m < 2 * S.l[c] + 1; ++m)
                    gamma_rows.push_back(kind == 0 ? kb_gamma[ch_base + c] : 0.0);
            t.h_sites.push_back(S);
            site_pts.push_back(std::move(pts));
        }
        ch_base += nch;
    }
    t.nsites = (int)t.h_sites.size();
    t.nhub = (int)t.h_U.size();
    t.natoms = natoms;

    // flat row -> grid index, gather items, CSR of entries per grid point
    std::vector<int> idx(t.npts);
    std::vector<int> items;
    t.h_item_first.assign(t.nsites + 1, 0);
    for (int s = 0; s < t.nsites; ++s) {
        const SiteDev& S = t.h_sites[s];
        std::copy(site_pts[s].begin(), site_pts[s].end(), idx.begin() + S.pt_off);
        t.h_item_first[s] = (int)items.size() / 3;
        for (int f = 0; f < S.npts; f += GITEM) {
            items.push_back(s);
            items.push_back(S.pt_off + f);
            items.push_back(std::min(GITEM, S.npts - f));
        }
    }
    t.nitems = (int)items.size() / 3;
    t.h_item_first[t.nsites] = t.nitems;
    std::vector<int> csr_off(h->Nd + 1, 0);
    for (int r = 0; r < t.npts; ++r) csr_off[idx[r] + 1]++;
    for (long g = 0; g < h->Nd; ++g) csr_off[g + 1] += csr_off[g];
    std::vector<int> fill(csr_off.begin(), csr_off.end() - 1);
    std::vector<int2> csr_ent(t.npts);
    if (t.nproj >= (1 << 26)) return fail(h, HUB_EINVAL, "too many projector rows");
    for (int s = 0; s < t.nsites; ++s) {
        const SiteDev& S = t.h_sites[s];
        for (int l = 0; l < S.npts; ++l) {
            const int e = fill[idx[S.pt_off + l]]++;
            csr_ent[e] = make_int2(S.val_off + l * S.nproj, (S.proj_off << 4) | S.nproj);
        }
    }
    // scatter order: the points that carry entries.  Double working types group them by the
    // list of sites touching them (then by grid index), so that the lanes of a warp walk the
    // same entry list (same trip counts, one W row per site for the whole warp): a masked
    // lane still costs FP64 pipe time.  Float types keep grid order, where neighbouring
    // lanes update neighbouring elements of Y (measured faster for complex float).
    std::vector<int> order;
    for (long g = 0; g < h->Nd; ++g)
        if (csr_off[g + 1] > csr_off[g]) order.push_back((int)g);
    if (h->esize == 8) std::sort(order.begin(), order.end(), [&](int a, int b) {
        const int na = csr_off[a + 1] - csr_off[a], nb = csr_off[b + 1] - csr_off[b];
        if (na != nb) return na < nb;
        for (int k = 0; k < na; ++k) {
            const int sa = csr_ent[csr_off[a] + k].y, sb = csr_ent[csr_off[b] + k].y;
            if (sa != sb) return sa < sb;
        }
        return a < b;
    });
    t.norder = (int)order.size();

    int rc;
    if ((rc = upload(h, &t.d_sites, t.h_sites))) return rc;
    if ((rc = upload(h, &t.d_items, items))) return rc;
    if ((rc = upload(h, &t.d_item_first, t.h_item_first))) return rc;
    if ((rc = upload(h, &t.d_idx, idx))) return rc;
    if ((rc = upload(h, &t.d_order, order))) return rc;
    if ((rc = upload(h, &t.d_csr_off, csr_off))) return rc;
    if ((rc = upload(h, &t.d_csr_ent, csr_ent))) return rc;
    if ((rc = upload(h, &t.d_gamma, gamma_rows))) return rc;
    if ((rc = upload(h, &t.d_hub_sites, t.h_hub_sites))) return rc;
    if ((rc = upload(h, &t.d_U, t.h_U))) return rc;
    const size_t vbytes = (size_t)t.nvals * h->esize * (h->cplx ? 2 : 1);
    if (vbytes) {
        HUB_CUDA_TRY(h, cudaMalloc(&t.d_vals, vbytes));
        dim3 grid(t.nitems);
        const double* kp = h->kpt;
        ProfScope ps(h, HUB_K_TABLE);
        if (h->esize == 8) {
            if (h->cplx)
                k_table_values<double, true><<<grid, 256, 0, h->stream>>>(t.d_sites, t.d_items, t.d_idx, (double*)t.d_vals, h->n1, h->n2, h->h[0], h->h[1], h->h[2], h->L[0], h->L[1], h->L[2], kp[0], kp[1], kp[2]);
            else
                k_table_values<double, false><<<grid, 256, 0, h->stream>>>(t.d_sites, t.d_items, t.d_idx, (double*)t.d_vals, h->n1, h->n2, h->h[0], h->h[1], h->h[2], h->L[0], h->L[1], h->L[2], kp[0], kp[1], kp[2]);
        } else {
            if (h->cplx)
                k_table_values<float, true><<<grid, 256, 0, h->stream>>>(t.d_sites, t.d_items, t.d_idx, (float*)t.d_vals, h->n1, h->n2, h->h[0], h->h[1], h->h[2], h->L[0], h->L[1], h->L[2], kp[0], kp[1], kp[2]);
            else
                k_table_values<float, false><<<grid, 256, 0, h->stream>>>(t.d_sites, t.d_items, t.d_idx, (float*)t.d_vals, h->n1, h->n2, h->h[0], h->h[1], h->h[2], h->L[0], h->L[1], h->L[2], kp[0], kp[1], kp[2]);
        }
        HUB_CUDA_TRY(h, cudaGetLastError());
    }
    if (h->esize == 4 && !h->cplx && h->n1 % 4 == 0 && t.nsites > 0) {
        HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));     // values are ready
        if ((rc = build_bricks(h, t, site_pts))) return rc;
    }
    const size_t mbytes = (size_t)std::max(t.nhub, 1) * 25 * sizeof(double) * (h->cplx ? 2 : 1);
    for (int s = 0; s < 2; ++s) {
        HUB_CUDA_TRY(h, cudaMalloc((void**)&t.d_M[s], mbytes));
        HUB_CUDA_TRY(h, cudaMemsetAsync(t.d_M[s], 0, mbytes, h->stream));
    }
    // the D = 0 coefficients M = (U/2) I
    for (int s = 0; s < 2; ++s) {
        std::vector<double> M((size_t)std::max(t.nhub, 1) * 25 * (h->cplx ? 2 : 1), 0.0);
        for (int i = 0; i < t.nhub; ++i)
            for (int m = 0; m < 5; ++m) M[(size_t)(i * 25 + m * 5 + m) * (h->cplx ? 2 : 1)] = 0.5 * t.h_U[i];
        HUB_CUDA_TRY(h, cudaMemcpyAsync(t.d_M[s], M.data(), M.size() * sizeof(double),
                                        cudaMemcpyHostToDevice, h->stream));
        HUB_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        t.h_M[s] = M;                  // host copy of the coefficients in use
    }
    free_table(h->proj);
    h->proj = std::move(t);
    h->mem_gen++;
    return HUB_OK;
}

static int gather_dense(hub_t h, const void* X, int ncol, int ld, int spin, bool want_W) {
    Table& t = h->proj;
    int rc;
    if ((rc = ensure(h, &h->d_part, &h->part_bytes, (size_t)t.npart_rows * ncol * sizeof(float)))) return rc;
    if ((rc = ensure(h, &h->d_C, &h->C_bytes, (size_t)t.nproj * ncol * sizeof(double)))) return rc;
    if ((rc = ensure(h, &h->d_W, &h->W_bytes, (size_t)t.nproj * ncol * sizeof(float)))) return rc;
    if (h->gather_dense >= 2 && t.tc) {
        if ((rc = launch_gather_tc(h, X, ncol, ld))) return rc;
    } else {
        ProfScope ps(h, HUB_K_GATHER);
        dim3 g(t.nbent, (ncol + GD_COLS - 1) / GD_COLS);
        k_gather_dense<<<g, 128, 0, h->stream>>>((const float*)X, ld, ncol, h->n1, h->n2, h->n3, t.nbx, t.nby,
                                                 t.d_bent, t.d_phi, (float*)h->d_part);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    {
        ProfScope ps(h, HUB_K_TRANSFORM);
        dim3 g(t.nproj, (ncol + RR_COLS - 1) / RR_COLS);
        k_reduce_rows_dense<<<g, 256, 0, h->stream>>>(ncol, h->dV, t.d_roff, t.d_rent, (const float*)h->d_part,
                                                      (double*)h->d_C);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    if (want_W) {
        const long nthr = (long)t.nsites * ncol;
        ProfScope ps(h, HUB_K_TRANSFORM);
        k_transform_sites<<<(unsigned)((nthr + 127) / 128), 128, 0, h->stream>>>(
            t.nsites, ncol, t.d_sites, (const double*)h->d_C, t.d_gamma, t.d_M[spin], (float*)h->d_W);
        HUB_CUDA_TRY(h, cudaGetLastError());
    }
    return HUB_OK;
}

static int scatter_dense(hub_t h, void* Y, int ncol, int ld, double alpha, const double* alpha_dev) {
    Table& t = h->proj;
    ProfScope ps(h, HUB_K_SCATTER);
    k_scatter_dense<<<t.nbused, 256, 0, h->stream>>>((float*)Y, ld, ncol, h->n1, h->n2, h->n3, t.nbx, t.nby,
                                                        t.d_bent, t.d_bfirst, t.d_phi, t.d_frow,
                                                        (const float*)h->d_W, (float)alpha, alpha_dev);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

// the brick form applies to real float blocks whose columns start on 16-byte boundaries
static bool use_dense(hub_t h, const void* A, int ld) {
    return h->proj.dense && h->esize == 4 && !h->cplx && ld % 4 == 0 && (uintptr_t)A % 16 == 0;
}

template <typename R, bool CPLX>
static int gather_t(hub_t h, const void* X, int ncol, int ld, int spin, bool want_W) {
    using T = typename VT<R, CPLX>::T;
    using D = typename VT<double, CPLX>::T;
    Table& t = h->proj;
    int rc;
    if ((rc = ensure(h, &h->d_part, &h->part_bytes, (size_t)t.nitems * kMaxProj * ncol * sizeof(D)))) return rc;
    if ((rc = ensure(h, &h->d_C, &h->C_bytes, (size_t)t.nproj * ncol * sizeof(D)))) return rc;
    if ((rc = ensure(h, &h->d_W, &h->W_bytes, (size_t)t.nproj * ncol * sizeof(T)))) return rc;
    // columns per warp (the value table is re-read once per column group): 16 bytes of each
    // point's row, except complex float, which takes four columns (32 bytes) with two points
    // per lane and iteration (rutile, 348 columns: 4.28 -> 2.66 ms; eight columns 2.58 ms at
    // 255 registers)
    constexpr bool C64 = CPLX && sizeof(R) == 4;
    constexpr int NC = C64 ? 4 : 16 / (int)sizeof(T);
    { ProfScope ps(h, HUB_K_GATHER);
    // one warp per CTA and four points per lane and iteration: the fastest of the shapes
    // measured on the rutile workload (1, 2, 4, 8 warps x 2, 4 points)
    constexpr int GW = 1, PTS = C64 ? 2 : 4;
    dim3 g1(t.nitems, (ncol + GW * NC - 1) / (GW * NC));
    k_gather<R, CPLX, GW, PTS, NC><<<g1, GW * 32, 0, h->stream>>>((const T*)X, ld, ncol, t.d_sites, t.d_items,
                                                                t.d_idx, (const T*)t.d_vals, (D*)h->d_part);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    const long nthr = (long)t.nsites * ncol;
    { ProfScope ps(h, HUB_K_TRANSFORM);
    k_reduce_transform<R, CPLX><<<(unsigned)((nthr + 127) / 128), 128, 0, h->stream>>>(
        t.nsites, ncol, h->dV, t.d_sites, t.d_item_first, (const D*)h->d_part, t.d_gamma,
        t.d_M[spin], (D*)h->d_C, (T*)h->d_W, want_W ? 1 : 0); }
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int launch_gather(hub_t h, const void* X, int ncol, int ld, int spin, bool want_W) {
    if (ncol == 0 || h->proj.nsites == 0) return HUB_OK;
    if (h->gather_dense && use_dense(h, X, ld)) return gather_dense(h, X, ncol, ld, spin, want_W);
    if (h->esize == 8) return h->cplx ? gather_t<double, true>(h, X, ncol, ld, spin, want_W)
                                      : gather_t<double, false>(h, X, ncol, ld, spin, want_W);
    return h->cplx ? gather_t<float, true>(h, X, ncol, ld, spin, want_W)
                   : gather_t<float, false>(h, X, ncol, ld, spin, want_W);
}

template <typename R, bool CPLX>
static int scatter_t(hub_t h, void* Y, int ncol, int ld, double alpha, const double* alpha_dev) {
    using T = typename VT<R, CPLX>::T;
    Table& t = h->proj;
    const int vec_ok = ((ncol * sizeof(T)) % 16 == 0) && ((uintptr_t)h->d_W % 16 == 0);
    if (t.norder == 0) return HUB_OK;
    dim3 grid((unsigned)((t.norder + 127) / 128));
    ProfScope ps(h, HUB_K_SCATTER);
    k_scatter<R, CPLX><<<grid, 128, 0, h->stream>>>((T*)Y, ld, ncol, t.norder, t.d_order, t.d_csr_off, t.d_csr_ent,
                                                    (const T*)t.d_vals, (const T*)h->d_W, (R)alpha, vec_ok,
                                                    alpha_dev);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int launch_scatter(hub_t h, void* Y, int ncol, int ld, double alpha, const double* alpha_dev) {
    if (ncol == 0 || h->proj.nsites == 0) return HUB_OK;
    if (use_dense(h, Y, ld)) {
        if (h->gather_dense == 3 && h->proj.tc) return launch_scatter_tc(h, Y, ncol, ld, alpha, alpha_dev);
        return scatter_dense(h, Y, ncol, ld, alpha, alpha_dev);
    }
    if (h->esize == 8) return h->cplx ? scatter_t<double, true>(h, Y, ncol, ld, alpha, alpha_dev)
                                      : scatter_t<double, false>(h, Y, ncol, ld, alpha, alpha_dev);
    return h->cplx ? scatter_t<float, true>(h, Y, ncol, ld, alpha, alpha_dev)
                   : scatter_t<float, false>(h, Y, ncol, ld, alpha, alpha_dev);
}

int launch_occupation(hub_t h, int ncol, const double* f_dev, double kweight, double* D_dev) {
    Table& t = h->proj;
    if (t.nhub == 0) {
        HUB_CUDA_TRY(h, cudaMemsetAsync(h->d_scal, 0, sizeof(double), h->stream));
        return HUB_OK;
    }
    double* eu = h->d_scal + 256;   // per-atom E_U contributions (slots 256..375)
    if (t.nhub > 120) return fail(h, HUB_EINVAL, "more than 120 Hubbard atoms not supported");
    {
    ProfScope ps(h, HUB_K_OCCUPATION);
    if (h->cplx)
        k_occupation<true><<<t.nhub, 256, 0, h->stream>>>(ncol, t.d_sites, t.d_hub_sites, (const double2*)h->d_C,
                                                         f_dev, kweight, D_dev, eu, t.d_U);
    else
        k_occupation<false><<<t.nhub, 256, 0, h->stream>>>(ncol, t.d_sites, t.d_hub_sites, (const double*)h->d_C,
                                                          f_dev, kweight, D_dev, eu, t.d_U);
    }
    HUB_CUDA_TRY(h, cudaGetLastError());
    ProfScope ps2(h, HUB_K_OCCUPATION);
    k_sum_serial<<<1, 32, 0, h->stream>>>(eu, t.nhub, h->d_scal);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int launch_moment_gather(hub_t h, const void* G, int ld, int ncol, double* Gm0, double* Gm1, double* Gm2) {
    Table& t = h->proj;
    if (t.nhub == 0 || ncol == 0) return HUB_OK;
    if (ncol > 65535) return fail(h, HUB_EINVAL, "at most 65535 columns per moment gather");
    const double kp[3] = {h->cplx ? h->kpt[0] : 0.0, h->cplx ? h->kpt[1] : 0.0, h->cplx ? h->kpt[2] : 0.0};
    const dim3 grid((unsigned)t.nhub, (unsigned)ncol);
    ProfScope ps(h, HUB_K_FORCE);
#define HUB_MOMENT_ARGS ld, ncol, t.d_sites, t.d_hub_sites, t.d_idx, h->n1, h->n2, h->h[0], h->h[1], h->h[2], \
        h->L[0], h->L[1], h->L[2], kp[0], kp[1], kp[2], h->dV, Gm0, Gm1, Gm2
    if (h->esize == 8) {
        if (h->cplx) k_moment_gather<double2, true><<<grid, 256, 0, h->stream>>>((const double2*)G, HUB_MOMENT_ARGS);
        else k_moment_gather<double, false><<<grid, 256, 0, h->stream>>>((const double*)G, HUB_MOMENT_ARGS);
    } else {
        if (h->cplx) k_moment_gather<float2, true><<<grid, 256, 0, h->stream>>>((const float2*)G, HUB_MOMENT_ARGS);
        else k_moment_gather<float, false><<<grid, 256, 0, h->stream>>>((const float*)G, HUB_MOMENT_ARGS);
    }
#undef HUB_MOMENT_ARGS
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

int launch_hub_force(hub_t h, int spin, int ncol, const double* f_dev, double kweight,
                     const void* C0, int axis, double* F_dev) {
    Table& t = h->proj;
    if (t.nhub == 0 || ncol == 0) return HUB_OK;
    ProfScope ps(h, HUB_K_OCCUPATION);
    if (h->cplx)
        k_hub_force<true><<<t.nhub, 256, 0, h->stream>>>(ncol, t.d_sites, t.d_hub_sites, (const double2*)C0,
                                                        (const double2*)h->d_C, f_dev, kweight, t.d_M[spin],
                                                        axis, F_dev);
    else
        k_hub_force<false><<<t.nhub, 256, 0, h->stream>>>(ncol, t.d_sites, t.d_hub_sites, (const double*)C0,
                                                         (const double*)h->d_C, f_dev, kweight, t.d_M[spin],
                                                         axis, F_dev);
    HUB_CUDA_TRY(h, cudaGetLastError());
    return HUB_OK;
}

}  // namespace hub
