/*
 * bte_resident.cu -- batched solver with the state resident on chip.
 *
 * One thread-block cluster (C CTAs, C in 1..16) owns one parameter point at
 * a time and keeps its four grid arrays (a, b of the whole and fractional
 * grids, Sec. 3) in the CTAs' shared memory for every step of the run: CTA
 * r holds harmonic rows [r R, (r+1) R) over all phi_y columns, plus one halo
 * row above and below.  A time step is the two half-steps of the leap-frog
 * scheme (Eqs. leap_frog_1, leap_frog_2), each applied in place -- the whole
 * grid's update reads only the fractional grid and each cell's own value,
 * and vice versa -- with a cluster barrier after each half-step.  A CTA
 * writes its first and last rows also into the halo rows of the
 * neighbouring CTAs (distributed shared memory) as it makes them, so that
 * after the barrier every row a CTA reads is in its own shared memory.
 * Per-cell
 * operations are those of the streaming kernel, in the same order (the
 * compiler may still contract multiply-adds differently); the per-step sums
 * of rows 0 and 1 (Eqs. v_dr_generic, norm_in_phi) are added in another
 * order.
 *
 * Clusters take points from a queue (an atomic counter over a list sorted
 * by cost); there are no spin-waits: the only waits are cluster barriers,
 * which every CTA of a cluster passes the same number of times (all CTAs
 * run the same point for the same number of steps).
 *
 * The single-instance solver's on-chip mode launches the same kernel with
 * one point: the run continues from step k0 of that instance (drive phase
 * (k0 + k) mod P) and the per-step drift velocity and norm go to its trace.
 */
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "bte_device.cuh"
#include "bte_internal.h"

namespace cg = cooperative_groups;

namespace bte {
namespace {

using dev::cluster_arrive;
using dev::cluster_wait;
using dev::cn_cell;
using dev::F2;
using dev::Half;
using dev::half_drive;
using dev::two_sum;
using dev::warp_sum;
using dev::warp_sum_f2;
using dev::CnK;
using dev::Rn;
using dev::rot_factor;
using dev::stencil_a;
using dev::stencil_b;

template <typename T>
struct RV {
    static constexpr int V = 16 / (int)sizeof(T); /* columns per work unit (16 bytes) */
};

template <typename T>
__device__ __forceinline__ void ld_vec(const T* p, T (&x)[RV<T>::V]) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
    } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        x[0] = v.x;
        x[1] = v.y;
    }
}

template <typename T>
__device__ __forceinline__ void st_vec(T* p, const T (&x)[RV<T>::V]) {
    if constexpr (sizeof(T) == 4)
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    else
        *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
}

/* central differences x[m+1] - x[m-1] of a group, the outer neighbours
 * taken from the adjacent lanes' groups where those are the adjacent
 * columns (l_adj / r_adj), else loaded.  Every lane of the warp must call
 * it (the shuffles need the full warp). */
template <typename T>
__device__ __forceinline__ void diff_sh(const T* p, bool l_adj, bool r_adj, T (&d)[RV<T>::V]) {
    constexpr int V = RV<T>::V;
    T own[V];
    ld_vec<T>(p, own);
    const T from_l = __shfl_up_sync(0xffffffffu, own[V - 1], 1);
    const T from_r = __shfl_down_sync(0xffffffffu, own[0], 1);
    const T left = l_adj ? from_l : p[-1];
    const T right = r_adj ? from_r : p[V];
    d[0] = own[1] - left;
#pragma unroll
    for (int e = 1; e < V - 1; ++e) d[e] = own[e + 1] - own[e - 1];
    d[V - 1] = right - own[V - 2];
}

/* central differences of a group with the outer neighbours loaded (the
 * group's own values as one 16-byte load) */
template <typename T>
__device__ __forceinline__ void diff_ld(const T* p, T (&d)[RV<T>::V]) {
    constexpr int V = RV<T>::V;
    T own[V];
    ld_vec<T>(p, own);
    const T left = p[-1], right = p[V];
    d[0] = own[1] - left;
#pragma unroll
    for (int e = 1; e < V - 1; ++e) d[e] = own[e + 1] - own[e - 1];
    d[V - 1] = right - own[V - 2];
}

/* One half-step (Sec. 3, Eqs. a_t_plus_1, b_t_plus_1, in increment form) on
 * the V cells of a group at harmonic n, in place: oA, oB the own grid's a, b;
 * da_u, da_d, db_u, db_d the phi_y differences of the other grid's a and b
 * in rows n-1 (u) and n+1 (d); t0, t1 the rotation factors
 * (E + B phi_m) dt/2 at the start and end of the half-step.  The same
 * operations in the same order as the streaming kernel (cn_row), so the
 * two give the same bits per cell. */
template <typename T>
__device__ __forceinline__ void cell_group(T* oA, T* oB, const T (&da_u)[RV<T>::V],
                                           const T (&da_d)[RV<T>::V], const T (&db_u)[RV<T>::V],
                                           const T (&db_d)[RV<T>::V], int n, int m0, int M, T hr,
                                           const T (&gc)[RV<T>::V], const T (&t0)[RV<T>::V],
                                           const T (&t1)[RV<T>::V], const CnK<T>& K, T cc,
                                           bool on, T* remU = nullptr, T* remD = nullptr,
                                           size_t rem_db = 0) {
    constexpr int V = RV<T>::V;
    T oa[V], ob[V], an[V], bn[V], na[V], nb[V];
    ld_vec<T>(oA, oa);
    ld_vec<T>(oB, ob);
    const T chi = (n == 1) ? (T)2 : (T)1;
    dev::cn_row<T, V>(oa, ob, db_d, db_u, da_u, da_d, cc, chi, hr, gc, (T)n, t0, t1, K, an, bn);
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const bool ok = m0 + e <= M;
        na[e] = ok ? an[e] : (T)0;
        nb[e] = (ok && n > 0) ? bn[e] : (T)0;
    }
    if (!on) return;
    st_vec<T>(oA, na);
    st_vec<T>(oB, nb);
    /* a boundary row also goes to the halo rows of the neighbouring CTAs
     * that read it in the next half-step (distributed shared memory;
     * rem_db: element offset of the b array from the a array) */
    if (remU) {
        st_vec<T>(remU, na);
        st_vec<T>(remU + rem_db, nb);
    }
    if (remD) {
        st_vec<T>(remD, na);
        st_vec<T>(remD + rem_db, nb);
    }
}

/* global array a of a point: 0 a_w, 1 b_w, 2 a_f, 3 b_f */
template <typename T>
__device__ __forceinline__ T* gsel(const BatchInst<T>& I, int a) {
    return a == 0 ? I.a_w[0] : a == 1 ? I.b_w[0] : a == 2 ? I.a_f[0] : I.b_f[0];
}

template <typename T>
__global__ void __launch_bounds__(512, 1) resident_kernel(ResArgs<T> A) {
    constexpr int V = RV<T>::V;
    constexpr int LG = V;              /* local ghost columns before m = 0 */
    constexpr int GG = Cols<T>::G;     /* global ghost columns before m = 0 */
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int C = A.C;
    double* red = reinterpret_cast<double*>(smem + A.red_off); /* [2][32] warp partials */
    int* s_next = reinterpret_cast<int*>(red + 64);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = (nthr + 31) >> 5;

    for (;;) {
        if (rank == 0 && tid == 0) *s_next = (int)atomicAdd(A.queue, 1u);
        cl.sync();
        const int qi = *cl.map_shared_rank(s_next, 0);
        cl.sync(); /* every CTA has read the index before rank 0 may replace it */
        if (qi >= A.count) break;
        const BatchInst<T>& I = A.inst[A.order[qi]];
        const int N = I.N, M = I.M, N1 = N + 1, gp = I.pitch, PP = I.P;
        const int rows_per = (N1 + C - 1) / C;
        const int r0 = min(N1, rank * rows_per), r1 = min(N1, r0 + rows_per), R = r1 - r0;
        const int ncg = (M + 1 + V - 1) / V;
        const long long K = I.K, Kw = I.Kw;
        const T h = I.h, hh = I.hh;
        const CnK<T> cn = dev::cn_constants<T>(h, I.nu, I.xi);
        /* shared-memory layout of this point: 4 arrays of rows_per + 2 rows
         * (halo, own rows, halo) with row stride P = ghost + columns + ghost */
        const int P = LG + ncg * V + V;
        const size_t arr = (size_t)(rows_per + 2) * P;
        T* sAw = reinterpret_cast<T*>(smem);
        T* sBw = sAw + arr;
        T* sAf = sBw + arr;
        T* sBf = sAf + arr;
        T* sG = sBf + arr; /* [P] column factor of a0 */
        T* sPh = sG + P;   /* [P] phi_m */
        T* sR = sPh + P;   /* [rows_per + 2] row factor of a0, rows r0-1 .. r0+rows_per */

        /* ---- load: zero everything, then rows r0-1 .. r1 that exist ---- */
        for (size_t q = tid; q < 4 * arr + 2 * (size_t)P + rows_per + 2; q += nthr) sAw[q] = (T)0;
        __syncthreads();
        {
            const int rows = R + 2;
            for (int q = tid; q < 4 * rows * ncg; q += nthr) {
                const int a = q / (rows * ncg);
                const int rem = q - a * rows * ncg;
                const int li = rem / ncg, g = rem - li * ncg;
                const int n = r0 - 1 + li;
                if (n < 0 || n > N) continue;
                T v[V];
                ld_vec<T>(gsel(I, a) + (size_t)n * gp + GG + g * V, v);
                st_vec<T>(sAw + a * arr + (size_t)li * P + LG + g * V, v);
            }
            for (int q = tid; q < ncg * V; q += nthr) {
                sG[LG + q] = I.col_g[GG + q];
                sPh[LG + q] = I.col_phi[GG + q];
            }
            for (int q = tid; q < R + 2; q += nthr) {
                const int n = r0 - 1 + q;
                sR[q] = (n >= 0 && n <= N) ? I.row_a0[n] : (T)0;
            }
        }
        __syncthreads();

        /* window accumulators (thread 0 of rank 0) */
        /* window accumulators in shared memory (thread 0 of rank 0 only
         * touches them; keeping them out of every thread's registers) */
        double* acc = red + 64 + 2; /* [6], after the warp partials and s_next */
        double* rot = acc + 6;      /* [4]: window cos, sin and the per-step rotation */
        if (tid == 0)
            for (int q = 0; q < 6; ++q) acc[q] = 0.0;
        /* halo rows: shared row 0 holds row r0-1 (the last row of rank-1),
         * shared row R+1 row r1 (the first row of rank+1), both as loaded
         * and then as the neighbours push them each half-step (the four
         * arrays of a CTA are contiguous, arr elements apart).  Rows outside
         * 0..N are halo rows that stay zero (no neighbour writes them). */
        const bool have_up = r0 >= 1 && R > 0, have_dn = r1 <= N && R > 0;
        /* a CTA's first own row is the halo row below the last own row of
         * rank-1 (its shared row rows_per + 1), its last own row the halo
         * row above rank+1's first (its shared row 0) */
        T* halo_up = have_up ? cl.map_shared_rank(sAw, rank - 1) + (size_t)(rows_per + 1) * P : nullptr;
        T* halo_dn = have_dn ? cl.map_shared_rank(sAw, rank + 1) : nullptr;

        /* interior rows 1..R-2 read only this CTA's rows: thread -> (column
         * group gl, row block rp), fixed for the point.  A block of nrow
         * consecutive rows [lo, lo + nrow) is walked as two chains of stride
         * 2 (lo, lo+2, ... then lo+1, lo+3, ...): the other grid's
         * differences of row i+1 serve rows i and i+2, so each chain loads
         * one other-grid row per row it updates, plus one at its start.  Every
         * thread runs the same number of iterations (the differences use
         * warp shuffles); iterations past row R-2 read clamped rows and store
         * nothing. */
        const int cpp = min(ncg, nthr);
        const int rsplit = nthr / cpp;
        const int gl = tid % cpp, rp = tid / cpp;
        const bool t_on = rp < rsplit;
        const int npass = (ncg + cpp - 1) / cpp;
        const int nint = R > 2 ? R - 2 : 0;
        const int nrow = (nint + rsplit - 1) / rsplit;
        const int lo = 1 + rp * nrow;
        /* boundary rows 0 and R-1 (one row when R == 1) */
        const int nbnd = R >= 2 ? 2 : R;

        /* one half-step on the rows of this CTA: own grid (o) updated in place
         * from the other grid (x) */
        auto half_interior = [&](int o, int x, const Half<T>& D) {
            for (int pass = 0; pass < npass; ++pass) {
                const int g = pass * cpp + gl;
                const bool g_on = t_on && g < ncg;
                const int m0 = (g_on ? g : 0) * V;
                const bool l_adj = lane > 0 && gl > 0;
                const bool r_adj = lane < 31 && gl + 1 < cpp && g + 1 < ncg;
                T gc[V], t0[V], t1[V];
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const T ph = sPh[LG + m0 + e];
                    gc[e] = sG[LG + m0 + e];
                    t0[e] = rot_factor<T>(D.E0, D.B0, ph, hh);
                    t1[e] = rot_factor<T>(D.E1, D.B1, ph, hh);
                }
                const T* xa = sAw + x * arr + LG + m0; /* other grid, shared row 0 */
                for (int ch = 0; ch < 2; ++ch) {
                    const int len = (nrow + 1 - ch) / 2; /* same for every thread */
                    if (len == 0) continue;             /* also when R < 3 */
                    const int i0 = lo + ch;
                    /* differences of the other grid's row i0-1 (shared row i0) */
                    T da_u[V], db_u[V];
                    {
                        const int il = min(i0, R - 2);
                        diff_sh<T>(xa + (size_t)il * P, l_adj, r_adj, da_u);
                        diff_sh<T>(xa + arr + (size_t)il * P, l_adj, r_adj, db_u);
                    }
#pragma unroll 1
                    for (int ii = 0; ii < len; ++ii) {
                        const int i = i0 + 2 * ii;
                        const bool on = g_on && i < R - 1;
                        const int il = min(i, R - 2);
                        T da_d[V], db_d[V];
                        diff_sh<T>(xa + (size_t)(il + 2) * P, l_adj, r_adj, da_d);
                        diff_sh<T>(xa + arr + (size_t)(il + 2) * P, l_adj, r_adj, db_d);
                        const size_t c = (size_t)(il + 1) * P + LG + m0;
                        cell_group<T>(sAw + o * arr + c, sAw + (o + 1) * arr + c, da_u, da_d, db_u,
                                      db_d, r0 + il, m0, M, Rn<T>::mul(h, sR[il + 1]), gc, t0, t1,
                                      cn, D.cc, on);
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            da_u[e] = da_d[e];
                            db_u[e] = db_d[e];
                        }
                    }
                }
            }
        };
        auto half_boundary = [&](int o, int x, const Half<T>& D) {
            for (int u = tid; u < nbnd * ncg; u += nthr) {
                const int b = u / ncg, g = u - b * ncg;
                const int il = b == 0 ? 0 : R - 1;
                const int m0 = g * V;
                const size_t c = (size_t)(il + 1) * P + LG + m0;
                /* rows il-1 and il+1 of the other grid, halo rows included:
                 * all in this CTA's shared memory */
                const T* up = sAw + x * arr + c - P;
                const T* dn = sAw + x * arr + c + P;
                T da_u[V], da_d[V], db_u[V], db_d[V];
                diff_ld<T>(up, da_u);
                diff_ld<T>(dn, da_d);
                diff_ld<T>(up + arr, db_u);
                diff_ld<T>(dn + arr, db_d);
                T gc[V], t0[V], t1[V];
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const T ph = sPh[LG + m0 + e];
                    gc[e] = sG[LG + m0 + e];
                    t0[e] = rot_factor<T>(D.E0, D.B0, ph, hh);
                    t1[e] = rot_factor<T>(D.E1, D.B1, ph, hh);
                }
                T* remU = (il == 0 && halo_up) ? halo_up + o * arr + LG + m0 : nullptr;
                T* remD = (il == R - 1 && halo_dn) ? halo_dn + o * arr + LG + m0 : nullptr;
                cell_group<T>(sAw + o * arr + c, sAw + (o + 1) * arr + c, da_u, da_d, db_u, db_d,
                              r0 + il, m0, M, Rn<T>::mul(h, sR[il + 1]), gc, t0, t1, cn, D.cc,
                              true, remU, remD, arr);
            }
        };

        /* split cluster barriers: a CTA signals when its rows of one grid are
         * complete, updates its interior rows of the other grid meanwhile,
         * and waits only before the rows that read a neighbour.  Rank 0 adds
         * the new whole grid's rows 0 (a) and 1 (b) while the fractional
         * half-step runs (that half-step leaves the whole grid unchanged);
         * thread 0 folds the warp partials into the window sums after the
         * step's last block barrier. */
        /* drive phase (k0 + k) mod P of step k, kept as a counter */
        int kk = PP > 0 ? (int)(I.k0 % PP) : 0;
        /* thread 0 of rank 0: cos of the window phase 2 pi ((k + 1) mod P) / P,
         * advanced by one rotation per step and reset to its exact value at
         * the start of every period (rounding grows over at most P steps) */
        int kc = PP > 0 ? 1 % PP : 0;
        if (rank == 0 && tid == 0) {
            const double two_pi = 6.283185307179586476925286766559;
            rot[0] = PP > 0 ? cos(two_pi * (double)kc / (double)PP) : 1.0;
            rot[1] = PP > 0 ? sin(two_pi * (double)kc / (double)PP) : 0.0;
            rot[2] = PP > 0 ? cos(two_pi / (double)PP) : 1.0;
            rot[3] = PP > 0 ? sin(two_pi / (double)PP) : 0.0;
        }
        cluster_arrive(); /* initial state loaded */
        for (long long k = 0; k < K; ++k) {
            const Half<T> Dw = half_drive<T>(I.e_whole, I.dstride, kk);
            const Half<T> Df = half_drive<T>(I.e_frac, I.dstride, kk);
            /* ---- whole grid: z_w^{k+1} = T(z_w^k; S(z_f^{k+1/2})) ---- */
            half_interior(0, 2, Dw);
            cluster_wait();
            half_boundary(0, 2, Dw);
            __syncthreads();
            cluster_arrive();
            if (rank == 0) {
                /* local rows 0 and 1 are shared rows 1 and 2; without a row 1
                 * (N = 0) shared row 2 is a zero halo row.  FP64 states add in
                 * FP64; FP32 states in hi + lo pairs of FP32 (FP64-grade) */
                double pn, pv;
                if constexpr (sizeof(T) == 8) {
                    pn = 0.0;
                    pv = 0.0;
                    for (int g = tid; g < ncg; g += nthr) {
                        T va[V], vb[V];
                        ld_vec<T>(sAw + P + LG + g * V, va);
                        ld_vec<T>(sBw + 2 * P + LG + g * V, vb);
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            pn += (double)va[e];
                            pv += (double)vb[e];
                        }
                    }
                    pn = warp_sum(pn);
                    pv = warp_sum(pv);
                } else {
                    F2 fn{0.0f, 0.0f}, fv{0.0f, 0.0f};
                    for (int g = tid; g < ncg; g += nthr) {
                        T va[V], vb[V];
                        ld_vec<T>(sAw + P + LG + g * V, va);
                        ld_vec<T>(sBw + 2 * P + LG + g * V, vb);
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            const F2 tn = two_sum(fn.hi, (float)va[e]);
                            fn = F2{tn.hi, __fadd_rn(fn.lo, tn.lo)};
                            const F2 tv = two_sum(fv.hi, (float)vb[e]);
                            fv = F2{tv.hi, __fadd_rn(fv.lo, tv.lo)};
                        }
                    }
                    pn = warp_sum_f2(fn);
                    pv = warp_sum_f2(fv);
                }
                if (lane == 0) {
                    red[warp] = pn;
                    red[32 + warp] = pv;
                }
            }
            /* ---- fractional grid: z_f^{k+3/2} = T(z_f^{k+1/2}; S(z_w^{k+1})) ---- */
            half_interior(2, 0, Df);
            cluster_wait();
            half_boundary(2, 0, Df);
            __syncthreads();
            cluster_arrive();
            if (rank == 0 && tid == 0) {
                double sn = 0, sv = 0;
                for (int w = 0; w < nwarp; ++w) {
                    sn += red[w];
                    sv += red[32 + w];
                }
                const double vv = I.vscale * sv, nn = I.nscale * sn;
                const long long k1 = k + 1;
                if (k1 > K - Kw) {
                    /* omega = 0 (P = 0): the angle omega t is 0 */
                    acc[0] += vv * rot[0];
                    acc[1] += vv;
                }
                if (PP > 0) {
                    if (++kc == PP) {
                        kc = 0;
                        rot[0] = 1.0;
                        rot[1] = 0.0;
                    } else {
                        const double c = rot[0], sn = rot[1];
                        rot[0] = c * rot[2] - sn * rot[3];
                        rot[1] = sn * rot[2] + c * rot[3];
                    }
                }
                acc[2] = fmax(acc[2], fabs(nn - 1.0));
                if (!isfinite(vv) || !isfinite(nn)) acc[3] = 1.0;
                acc[4] = vv;
                acc[5] = nn;
                if (I.trace_v) {
                    I.trace_v[I.k0 + k1] = vv;
                    I.trace_n[I.k0 + k1] = nn;
                }
            }
            if (PP > 0 && ++kk == PP) kk = 0; /* P = 0 (omega = 0): row 0 every step */
        }
        cluster_wait(); /* pairs the last arrive */

        /* ---- results: window sums, final state ---- */
        if (rank == 0 && tid == 0) {
            for (int q = 0; q < 6; ++q) I.acc[q] = acc[q];
        }
        for (int q = tid; q < 4 * R * ncg; q += nthr) {
            const int a = q / (R * ncg);
            const int rem = q - a * R * ncg;
            const int i = rem / ncg, g = rem - i * ncg;
            T v[V];
            ld_vec<T>(sAw + a * arr + (size_t)(i + 1) * P + LG + g * V, v);
            st_vec<T>(gsel(I, a) + (size_t)(r0 + i) * gp + GG + g * V, v);
        }
        /* the next point's load overwrites shared memory that neighbours
         * may still read in their last boundary rows: wait for the cluster */
        cl.sync();
    }
}

}  // namespace

template <typename T>
size_t resident_smem_bytes(int N, int M, int C, size_t* arrays_bytes) {
    constexpr int V = RV<T>::V;
    const int rows_per = (N + 1 + C - 1) / C;
    const int ncg = (M + 1 + V - 1) / V;
    const size_t P = (size_t)(V + ncg * V + V);
    const size_t arr = (size_t)(rows_per + 2) * P;
    size_t b = (4 * arr + 2 * P + rows_per + 2) * sizeof(T);
    b = (b + 15) / 16 * 16;
    if (arrays_bytes) *arrays_bytes = b;
    return b + 64 * sizeof(double) + 16 + 10 * sizeof(double);
}

template <typename T>
int resident_max_clusters(int C, size_t smem, int threads, int* clusters) {
    cudaError_t e = cudaFuncSetAttribute(resident_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(resident_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaOccupancyMaxActiveClusters(clusters, resident_kernel<T>, &cfg);
    return (int)e;
}

template <typename T>
int launch_resident(const ResArgs<T>& a, int clusters, int threads, size_t smem, void* stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * a.C, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = a.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, resident_kernel<T>, a);
    return e == cudaSuccess ? 0 : (int)e;
}

template size_t resident_smem_bytes<float>(int, int, int, size_t*);
template size_t resident_smem_bytes<double>(int, int, int, size_t*);
template int resident_max_clusters<float>(int, size_t, int, int*);
template int resident_max_clusters<double>(int, size_t, int, int*);
template int launch_resident<float>(const ResArgs<float>&, int, int, size_t, void*);
template int launch_resident<double>(const ResArgs<double>&, int, int, size_t, void*);

}  // namespace bte
