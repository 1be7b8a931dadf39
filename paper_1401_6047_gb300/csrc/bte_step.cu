/*
 * bte_step.cu -- the fused leap-frog step kernel (sm_103a).
 *
 * One launch performs one full step of Sec. 3 (Eqs. leap_frog_1, leap_frog_2):
 *     whole grid       z^{t+1}   = T(z^t;       S(z^{t+1/2}))
 *     fractional grid  z^{t+3/2} = T(z^{t+1/2}; S(z^{t+1}))
 * T is the Crank-Nicolson operator of Eqs. a_t_plus_1 / b_t_plus_1 and S the
 * 4-point diagonal stencil of the paper's A^t / B^t terms, which only needs
 * the central differences  D x_r(m) = x_r(m+1) - x_r(m-1)  of rows r = n+-1:
 *     B^t_{n,m} = c (D b_{n+1} - D b_{n-1}),  A^t_{n,m} = c (chi(n) D a_{n-1} - D a_{n+1}),
 *     c = B dt / (4 dphi).
 *
 * Work items.  The grid is cut into items of tile_m phi_y columns x chunk_n
 * harmonic rows.  Persistent CTAs take items q = blockIdx.x, +gridDim.x, ...
 * An item is walked upward in n with a one-row lag: at row j the CTA builds
 * the new whole-grid row j (its columns plus one halo column per side) and
 * then the new fractional row j-1, which needs the new whole rows j-2 and j.
 *
 * Threads.  Compute thread t owns the column pair (2t, 2t+1) of the tile.
 * One extra warp (the producer) issues the TMA bulk copies that stream the
 * old fractional and whole rows into a ring of RS shared-memory stages
 * (cp.async.bulk + mbarrier, RS-2 rows ahead of use, continuing across
 * items), and computes the two halo cells of each new whole row.
 *
 * Data reuse.  Every old fractional row is read from shared memory once per
 * thread when it arrives; its own values and central differences stay in
 * registers for the two rows that use them.  A new whole row goes to
 * shared memory once (for the neighbours' differences) and straight from
 * registers to global memory; the new fractional row goes from registers to
 * global memory.  One __syncthreads per row.
 *
 * Observables (Sec. 2, Eqs. v_dr_generic and norm_in_phi): items that own
 * rows 0 and 1 reduce sum_m a_{0,m} and sum_m b_{1,m} in FP64; the last of
 * them to arrive adds the per-tile partials in tile order, so the trace is
 * bitwise reproducible.
 *
 * Every mbarrier wait is bounded (~2 s of %globaltimer); on expiry the kernel
 * records an error word that the host reports as BTE_ETIMEOUT.
 */
#include <cuda_runtime.h>

#include <cstdint>

#include "bte_device.cuh"
#include "bte_internal.h"

namespace bte {

namespace {

using namespace dev;

/* largest block: 512 compute threads + producer warp in FP32; FP64 tiles
 * stop at 512 columns (256 + 32 threads) to leave room for its registers */
template <typename T>
struct MaxBlock {
    static constexpr int value = sizeof(T) == 4 ? 544 : 288;
};

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <typename T>
struct StepCfg {
    static constexpr int H = 16 / (int)sizeof(T); /* zero ghost / halo columns = 16 bytes */
    static constexpr int RS = sizeof(T) == 4 ? 8 : 6; /* TMA ring stages */
};

template <typename T>
__host__ __device__ inline int compute_threads(int tile_m) {
    return tile_m / 2;
}
__host__ __device__ inline int round_warp(int n) { return (n + 31) / 32 * 32; }

template <typename T>
__host__ __device__ inline size_t smem_layout(int tile_m, int chunk_n, size_t* offN, size_t* offR,
                                              size_t* offBar, size_t* offRed) {
    constexpr int H = StepCfg<T>::H, RS = StepCfg<T>::RS;
    const size_t LW = (size_t)tile_m + 2 * H;
    const size_t WN = (size_t)tile_m + 4;
    size_t o = 2 * (size_t)RS * 2 * LW * sizeof(T); /* old fractional + old whole rows */
    *offN = o;
    o += 2 * 2 * WN * sizeof(T); /* new whole rows, 2 slots x (a, b) */
    o = (o + 15) / 16 * 16;
    *offR = o;
    o += ((size_t)chunk_n + 4) * sizeof(T); /* row factors of the item */
    o = (o + 15) / 16 * 16;
    *offBar = o;
    o += RS * sizeof(uint64_t);
    *offRed = o;
    o += 33 * sizeof(double);
    return o;
}

template <typename T>
__global__ void __launch_bounds__(MaxBlock<T>::value) fused_step_kernel(StepArgs<T> A, int launch_i) {
    using V2 = typename Vec2<T>::type;
    constexpr int H = StepCfg<T>::H;
    constexpr int RS = StepCfg<T>::RS;
    extern __shared__ __align__(128) unsigned char smem_raw[];

    const int Wt = A.tile_m;
    const int NT = compute_threads<T>(Wt);
    const int NTr = round_warp(NT);
    const int LW = Wt + 2 * H;
    const int WN = Wt + 4;
    size_t offN, offR, offBar, offRed;
    smem_layout<T>(Wt, A.chunk_n, &offN, &offR, &offBar, &offRed);
    T* sF = reinterpret_cast<T*>(smem_raw);             /* [RS][2][LW] */
    T* sW = sF + (size_t)RS * 2 * LW;                   /* [RS][2][LW] */
    T* sN = reinterpret_cast<T*>(smem_raw + offN);      /* [2][2][WN]  */
    T* sR = reinterpret_cast<T*>(smem_raw + offR);      /* [chunk_n+4] */
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + offBar);
    double* red = reinterpret_cast<double*>(smem_raw + offRed);

    const int tid = threadIdx.x;
    const bool is_comp = tid < NT;
    const bool is_prod = tid >= NTr;
    const int lane = tid & 31;
    const int N = A.N, M = A.M, pitch = A.pitch;

    const long long k = *A.base + launch_i;
    const int cur = (int)(k & 1), nxt = cur ^ 1;
    const int kk = A.P > 0 ? (int)(k % A.P) : 0;
    const T Ews = (T)A.e_whole[kk], Ewe = (T)A.e_whole[kk + 1];
    const T Efs = (T)A.e_frac[kk], Efe = (T)A.e_frac[kk + 1];
    const T h = A.h, hh = A.hh, nu = A.nu, xi = A.xi, cc = A.c;
    const T* gFa = A.a_f[cur];
    const T* gFb = A.b_f[cur];
    const T* gWa = A.a_w[cur];
    const T* gWb = A.b_w[cur];
    T* oWa = A.a_w[nxt];
    T* oWb = A.b_w[nxt];
    T* oFa = A.a_f[nxt];
    T* oFb = A.b_f[nxt];
    const int ntx = A.ntx;
    const int items = A.ntx * A.nty;
    const uint32_t rowbytes = (uint32_t)(LW * sizeof(T));

    if (tid == NTr) {
        for (int s = 0; s < RS; ++s) mbar_init(smem_u32(&bar[s]), 1);
        fence_proxy_async_smem();
    }
    /* new-row buffers: index 0 and WN-1 are never written and stay zero */
    for (int q = tid; q < 4 * WN; q += blockDim.x) sN[q] = (T)0;
    __syncthreads();

    /* ---- producer state: global stage sequence across this CTA's items ---- */
    int p_item = blockIdx.x; /* item whose stages are being issued */
    int p_s = 0;             /* next stage of p_item                 */
    long long issued = 0;    /* stages issued so far                 */
    long long freed = 0;     /* stages whose slots may be reused     */
    auto item_rows = [&](int q, int& n0, int& n1) {
        const int ty = q / ntx;
        n0 = ty * A.chunk_n;
        n1 = min(n0 + A.chunk_n, N + 1);
    };
    /* issue as many stages as the ring allows (producer lane 0 only) */
    auto pump = [&]() {
        while (p_item < items && issued < freed + RS) {
            int n0, n1;
            item_rows(p_item, n0, n1);
            const int S = n1 - n0 + 4; /* rows n0-2 .. n1+1 */
            const int row = n0 - 2 + p_s;
            const int slot = (int)(issued % RS);
            const uint32_t mb = smem_u32(&bar[slot]);
            if (row < 0 || row > N) {
                mbar_arrive(mb);
            } else {
                const int tx = p_item % ntx;
                const int col0 = tx * Wt; /* = first owned physical column - H */
                const bool wneed = row >= n0 - 1 && row <= n1;
                mbar_arrive_tx(mb, rowbytes * (wneed ? 4u : 2u));
                const size_t off = (size_t)row * pitch + col0;
                T* dF = sF + (size_t)slot * 2 * LW;
                bulk_g2s(smem_u32(dF), gFa + off, rowbytes, mb);
                bulk_g2s(smem_u32(dF + LW), gFb + off, rowbytes, mb);
                if (wneed) {
                    T* dW = sW + (size_t)slot * 2 * LW;
                    bulk_g2s(smem_u32(dW), gWa + off, rowbytes, mb);
                    bulk_g2s(smem_u32(dW + LW), gWb + off, rowbytes, mb);
                }
            }
            ++issued;
            if (++p_s == S) {
                p_s = 0;
                p_item += gridDim.x;
            }
        }
    };
    if (tid == NTr) pump();

    bool timed_out = false;
    long long cbase = 0; /* global stage index of the current item's stage 0 */

    for (int q = blockIdx.x; q < items; q += gridDim.x) {
        const int tx = q % ntx;
        int n0, n1;
        item_rows(q, n0, n1);
        const int S = n1 - n0 + 4;
        const int p0 = H + tx * Wt; /* physical column of the tile's first column */

        __syncthreads(); /* the previous item's last row is done with sR and sN */
        /* row factors sigma_n I_n/I_0/pi of rows n0-1 .. n1 */
        for (int r = tid; r < n1 - n0 + 2; r += blockDim.x) {
            const int n = n0 - 1 + r;
            sR[r] = (n >= 0 && n <= N) ? A.row_a0[n] : (T)0;
        }

        /* per-column constants of the thread's pair */
        const int c = p0 + 2 * tid;         /* physical column of the pair   */
        const int lc = H + 2 * tid;         /* its index in a streamed row   */
        const bool ok0 = is_comp && (c - H) <= M;
        const bool ok1 = is_comp && (c + 1 - H) <= M;
        T g0 = 0, g1 = 0, bp0 = 0, bp1 = 0;
        if (ok0) {
            g0 = A.col_g[c];
            bp0 = A.col_bphi[c];
        }
        if (ok1) {
            g1 = A.col_g[c + 1];
            bp1 = A.col_bphi[c + 1];
        }
        const T ws0 = (Ews + bp0) * hh, ws1 = (Ews + bp1) * hh;
        const T we0 = (Ewe + bp0) * hh, we1 = (Ewe + bp1) * hh;
        const T fs0 = (Efs + bp0) * hh, fs1 = (Efs + bp1) * hh;
        const T fe0 = (Efe + bp0) * hh, fe1 = (Efe + bp1) * hh;

        /* producer lanes 0/1: the halo columns p0-1 and p0+Wt of new whole rows */
        const int hcol = (lane == 0) ? p0 - 1 : p0 + Wt;
        const bool hok = is_prod && lane < 2 && (hcol - H) >= 0 && (hcol - H) <= M;
        const int hlc = hcol - (p0 - H);
        T hg = 0, hbs = 0, hbe = 0;
        if (hok) {
            hg = A.col_g[hcol];
            const T bp = A.col_bphi[hcol];
            hbs = (Ews + bp) * hh;
            hbe = (Ewe + bp) * hh;
        }
        __syncthreads(); /* sR ready */

        /* rolling windows (registers): old fractional rows j-1, j (own pair
         * and central differences), central differences of new whole rows
         * j-2, j-1 */
        V2 fa_m1 = {0, 0}, fb_m1 = {0, 0}, fa_0 = {0, 0}, fb_0 = {0, 0};
        V2 dfa_m1 = {0, 0}, dfb_m1 = {0, 0}, dfa_0 = {0, 0}, dfb_0 = {0, 0};
        V2 dwa_m2 = {0, 0}, dwb_m2 = {0, 0}, dwa_m1 = {0, 0}, dwb_m1 = {0, 0};
        double part_n = 0.0, part_v = 0.0;

        /* stages 0 and 1 (old rows n0-2, n0-1) are consumed like row j+1 of
         * iterations n0-3 and n0-2, which only load */
        for (int j = n0 - 3; j <= n1; ++j) {
            const int si = j - n0 + 3; /* stage holding old row j+1 */
            const long long g = cbase + si;
            const int slot = (int)(g % RS);
            if (!mbar_wait(smem_u32(&bar[slot]), (uint32_t)((g / RS) & 1))) timed_out = true;

            /* old fractional row j+1: own pair and central differences */
            V2 fa_p1 = {0, 0}, fb_p1 = {0, 0}, dfa_p1 = {0, 0}, dfb_p1 = {0, 0};
            if (j + 1 >= 0 && j + 1 <= N && is_comp) {
                const T* ra = sF + (size_t)slot * 2 * LW;
                const T* rb = ra + LW;
                const V2 la = *reinterpret_cast<const V2*>(ra + lc - 2);
                const V2 oa = *reinterpret_cast<const V2*>(ra + lc);
                const V2 pa = *reinterpret_cast<const V2*>(ra + lc + 2);
                const V2 lb = *reinterpret_cast<const V2*>(rb + lc - 2);
                const V2 ob = *reinterpret_cast<const V2*>(rb + lc);
                const V2 pb = *reinterpret_cast<const V2*>(rb + lc + 2);
                fa_p1 = oa;
                fb_p1 = ob;
                dfa_p1.x = oa.y - la.y;
                dfa_p1.y = pa.x - oa.x;
                dfb_p1.x = ob.y - lb.y;
                dfb_p1.y = pb.x - ob.x;
            }

            if (j >= n0 - 1) {
                /* ---- new whole-grid row j ---- */
                const bool wrow = j >= 0 && j <= N;
                V2 wa_n = {0, 0}, wb_n = {0, 0};
                if (wrow) {
                    const int sw = (int)((cbase + si - 1) % RS); /* stage of old row j */
                    const T nf = (T)j;
                    const T chi = (j == 1) ? (T)2 : (T)1;
                    const T ha0 = h * sR[j - n0 + 1];
                    if (is_comp) {
                        const T* wa = sW + (size_t)sw * 2 * LW;
                        const V2 oa = *reinterpret_cast<const V2*>(wa + lc);
                        const V2 ob = *reinterpret_cast<const V2*>(wa + LW + lc);
                        T an, bn;
                        cn_cell<T>(oa.x, ob.x, cc * (dfb_p1.x - dfb_m1.x),
                                   cc * (chi * dfa_m1.x - dfa_p1.x), ha0 * g0, nf * ws0,
                                   nf * we0, nu, xi, h, an, bn);
                        wa_n.x = ok0 ? an : (T)0;
                        wb_n.x = (ok0 && j > 0) ? bn : (T)0;
                        cn_cell<T>(oa.y, ob.y, cc * (dfb_p1.y - dfb_m1.y),
                                   cc * (chi * dfa_m1.y - dfa_p1.y), ha0 * g1, nf * ws1,
                                   nf * we1, nu, xi, h, an, bn);
                        wa_n.y = ok1 ? an : (T)0;
                        wb_n.y = (ok1 && j > 0) ? bn : (T)0;
                        T* na = sN + (size_t)(j & 1) * 2 * WN;
                        *reinterpret_cast<V2*>(na + 2 + 2 * tid) = wa_n;
                        *reinterpret_cast<V2*>(na + WN + 2 + 2 * tid) = wb_n;
                        if (j >= n0 && j < n1) {
                            const size_t go = (size_t)j * pitch + c;
                            if (ok1) {
                                *reinterpret_cast<V2*>(oWa + go) = wa_n;
                                *reinterpret_cast<V2*>(oWb + go) = wb_n;
                            } else if (ok0) {
                                oWa[go] = wa_n.x;
                                oWb[go] = wb_n.x;
                            }
                        }
                        if (n0 == 0) {
                            if (j == 0) part_n += (double)wa_n.x + (double)wa_n.y;
                            if (j == 1) part_v += (double)wb_n.x + (double)wb_n.y;
                        }
                    } else if (is_prod && lane < 2) {
                        T an = 0, bn = 0;
                        if (hok) {
                            const T* fd_a = sF + (size_t)((cbase + si - 2) % RS) * 2 * LW;
                            const T* fu_a = sF + (size_t)slot * 2 * LW;
                            const bool dn = j - 1 >= 0, up = j + 1 <= N;
                            const T Dad = dn ? fd_a[hlc + 1] - fd_a[hlc - 1] : (T)0;
                            const T Dbd = dn ? fd_a[LW + hlc + 1] - fd_a[LW + hlc - 1] : (T)0;
                            const T Dau = up ? fu_a[hlc + 1] - fu_a[hlc - 1] : (T)0;
                            const T Dbu = up ? fu_a[LW + hlc + 1] - fu_a[LW + hlc - 1] : (T)0;
                            const T* wa = sW + (size_t)sw * 2 * LW;
                            cn_cell<T>(wa[hlc], wa[LW + hlc], cc * (Dbu - Dbd), cc * (chi * Dad - Dau),
                                       ha0 * hg, nf * hbs, nf * hbe, nu, xi, h, an, bn);
                            if (j == 0) bn = (T)0;
                        }
                        T* na = sN + (size_t)(j & 1) * 2 * WN;
                        const int idx = (lane == 0) ? 1 : Wt + 2;
                        na[idx] = an;
                        na[WN + idx] = bn;
                    }
                }
                __syncthreads();
                if (tid == NTr) {
                    /* every stage up to old row j-1 has been read for the last time */
                    const long long f = (j == n1) ? cbase + S : cbase + si - 1;
                    if (f > freed) freed = f;
                    fence_proxy_async_smem();
                    pump();
                }

                /* ---- new fractional row j-1 ---- */
                V2 dwa_0 = {0, 0}, dwb_0 = {0, 0};
                if (wrow && is_comp) {
                    const T* na = sN + (size_t)(j & 1) * 2 * WN;
                    const V2 la = *reinterpret_cast<const V2*>(na + 2 * tid);
                    const V2 pa = *reinterpret_cast<const V2*>(na + 2 * tid + 4);
                    const V2 lb = *reinterpret_cast<const V2*>(na + WN + 2 * tid);
                    const V2 pb = *reinterpret_cast<const V2*>(na + WN + 2 * tid + 4);
                    dwa_0.x = wa_n.y - la.y;
                    dwa_0.y = pa.x - wa_n.x;
                    dwb_0.x = wb_n.y - lb.y;
                    dwb_0.y = pb.x - wb_n.x;
                }
                const int r = j - 1;
                if (r >= n0 && r < n1 && is_comp && ok0) {
                    const T nf = (T)r;
                    const T chi = (r == 1) ? (T)2 : (T)1;
                    const T ha0 = h * sR[r - n0 + 1];
                    V2 fa_n, fb_n;
                    cn_cell<T>(fa_m1.x, fb_m1.x, cc * (dwb_0.x - dwb_m2.x),
                               cc * (chi * dwa_m2.x - dwa_0.x), ha0 * g0, nf * fs0, nf * fe0, nu,
                               xi, h, fa_n.x, fb_n.x);
                    cn_cell<T>(fa_m1.y, fb_m1.y, cc * (dwb_0.y - dwb_m2.y),
                               cc * (chi * dwa_m2.y - dwa_0.y), ha0 * g1, nf * fs1, nf * fe1, nu,
                               xi, h, fa_n.y, fb_n.y);
                    if (r == 0) {
                        fb_n.x = (T)0;
                        fb_n.y = (T)0;
                    }
                    const size_t go = (size_t)r * pitch + c;
                    if (ok1) {
                        *reinterpret_cast<V2*>(oFa + go) = fa_n;
                        *reinterpret_cast<V2*>(oFb + go) = fb_n;
                    } else {
                        oFa[go] = fa_n.x;
                        oFb[go] = fb_n.x;
                    }
                }

                /* ---- observables of rows 0 and 1 ---- */
                if (n0 == 0 && j == 1) {
                    const double sn = block_sum(part_n, red);
                    const double sv = block_sum(part_v, red);
                    if (tid == 0) {
                        A.part[tx] = sn;
                        A.part[ntx + tx] = sv;
                        __threadfence();
                        const unsigned t = atomicAdd(A.ticket, 1u);
                        if (t == (unsigned)(ntx - 1)) {
                            __threadfence();
                            double s_n = 0, s_v = 0;
                            const volatile double* pv = A.part;
                            for (int u = 0; u < ntx; ++u) {
                                s_n += pv[u];
                                s_v += pv[ntx + u];
                            }
                            A.trace_n[k + 1] = A.nscale * s_n;
                            A.trace_v[k + 1] = A.vscale * s_v;
                            *A.ticket = 0u;
                        }
                    }
                }
                dwa_m2 = dwa_m1;
                dwb_m2 = dwb_m1;
                dwa_m1 = dwa_0;
                dwb_m1 = dwb_0;
            }
            fa_m1 = fa_0;
            fb_m1 = fb_0;
            fa_0 = fa_p1;
            fb_0 = fb_p1;
            dfa_m1 = dfa_0;
            dfb_m1 = dfb_0;
            dfa_0 = dfa_p1;
            dfb_0 = dfb_p1;
        }
        cbase += S;
    }
    if (timed_out) atomicExch(A.err, kErrTimeout);
}

}  // namespace

static int ok_or(cudaError_t e) { return e == cudaSuccess ? 0 : (int)e; }

template <typename T>
size_t step_smem_bytes(int tile_m, int chunk_n) {
    size_t a, b, c, d;
    return smem_layout<T>(tile_m, chunk_n, &a, &b, &c, &d);
}

template <typename T>
int step_block_threads(int tile_m) {
    return round_warp(compute_threads<T>(tile_m)) + 32;
}

template <typename T>
int step_max_tile() {
    return 2 * (MaxBlock<T>::value - 32);
}

template <typename T>
int step_kernel_configure(int tile_m, int chunk_n, int* blocks_per_sm) {
    const size_t bytes = step_smem_bytes<T>(tile_m, chunk_n);
    cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fused_step_kernel<T>,
                                                      step_block_threads<T>(tile_m), bytes);
    if (e != cudaSuccess) return (int)e;
    *blocks_per_sm = nb;
    return 0;
}

template <typename T>
int launch_step(const StepArgs<T>& a, int i, void* stream) {
    fused_step_kernel<T><<<a.grid, step_block_threads<T>(a.tile_m),
                           step_smem_bytes<T>(a.tile_m, a.chunk_n), (cudaStream_t)stream>>>(a, i);
    return ok_or(cudaGetLastError());
}

#define BTE_STEP_INSTANTIATE(T)                                 \
    template size_t step_smem_bytes<T>(int, int);               \
    template int step_block_threads<T>(int);                    \
    template int step_max_tile<T>();                            \
    template int step_kernel_configure<T>(int, int, int*);      \
    template int launch_step<T>(const StepArgs<T>&, int, void*);
BTE_STEP_INSTANTIATE(float)
BTE_STEP_INSTANTIATE(double)

}  // namespace bte
