/*
 * bte_step.cu -- the fused leap-frog step kernel (sm_103a).
 *
 * One launch performs TS = 1 or 2 full steps of Sec. 3 (Eqs. leap_frog_1,
 * leap_frog_2), i.e. NST = 2 TS half-step stages:
 *     stage 0   whole grid       z^{k+1}   = T(z^k;       S(z^{k+1/2}))
 *     stage 1   fractional grid  z^{k+3/2} = T(z^{k+1/2}; S(z^{k+1}))
 *     stage 2   whole grid       z^{k+2}   = T(z^{k+1};   S(z^{k+3/2}))
 *     stage 3   fractional grid  z^{k+5/2} = T(z^{k+3/2}; S(z^{k+2}))
 * T is the Crank-Nicolson operator of Eqs. a_t_plus_1 / b_t_plus_1 and S the
 * 4-point diagonal stencil of the paper's A^t / B^t terms, which only needs
 * the central differences  D x_r(m) = x_r(m+1) - x_r(m-1)  of rows r = n+-1:
 *     B^t_{n,m} = c (D b_{n+1} - D b_{n-1}),  A^t_{n,m} = c (chi(n) D a_{n-1} - D a_{n+1}),
 *     c = B dt / (4 dphi).
 * Only the old state is read from memory and only the final whole and
 * fractional grids are written: with TS = 2 the memory traffic per step is
 * halved (temporal blocking).
 *
 * Work items.  The grid is cut into items of tile_m phi_y columns x chunk_n
 * harmonic rows; persistent CTAs take items q = blockIdx.x, +gridDim.x, ...
 * Stage s of an item covers its rows widened by e_s = NST-1-s on each side
 * (and its columns by a V-column halo group per side for s < NST-1), so
 * every stage has the neighbours it needs.  At row-iteration j stage s
 * computes row j - 2s: stage s reads rows j-2s+-1 of stage s-1, produced at
 * iterations j-1 and j-3, so the stages of one iteration are independent
 * and one __syncthreads per iteration suffices.  Stage outputs go to
 * 5-row shared-memory rings (slot = producing iteration mod 5).
 *
 * Threads.  Compute thread t owns V consecutive columns (V = 2 or 4) of the
 * tile.  One extra warp (the producer) issues the TMA bulk copies that
 * stream the old fractional and whole rows into a ring of RS shared-memory
 * stages (cp.async.bulk + mbarrier, continuing across items); its lanes 0
 * and 1 compute the halo column groups of the inner stages.
 *
 * Launch.  Programmatic dependent launch: the prologue runs while the
 * previous launch drains; griddepcontrol.wait precedes the first read of
 * the state.
 *
 * Observables (Sec. 2, Eqs. v_dr_generic and norm_in_phi): items that own
 * rows 0 and 1 reduce sum_m a_{0,m} and sum_m b_{1,m} of every new whole grid
 * in FP64; the last item to arrive adds the per-tile partials in tile order,
 * so the trace is bitwise reproducible.
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

template <typename T>
struct StepCfg {
    static constexpr int H = Cols<T>::H; /* streamed halo columns per side */
    static constexpr int G = Cols<T>::G;
    static constexpr int RS = 8; /* TMA ring stages (power of two) */
    static constexpr int NR = 5; /* rows per stage-output ring */
};

/* largest block: 512 compute threads + producer warp for FP32 with V = 2,
 * 256 + 32 otherwise */
template <typename T, int V>
struct MaxBlock {
    static constexpr int value = (sizeof(T) == 4 && V == 2) ? 544 : 288;
};

__host__ __device__ inline int round_warp(int n) { return (n + 31) / 32 * 32; }

struct SmemLayout {
    size_t offW, offRing, offZ, offR, offBar, offRed, total;
};

template <typename T>
__host__ __device__ inline SmemLayout smem_layout(int tile_m, int chunk_n, int V, int ts) {
    constexpr int H = StepCfg<T>::H, RS = StepCfg<T>::RS, NR = StepCfg<T>::NR;
    const size_t LW = (size_t)tile_m + 2 * H;
    const size_t RW = (size_t)tile_m + 4 * V;
    const size_t ZW = LW > RW ? LW : RW;
    SmemLayout L;
    size_t o = (size_t)RS * 2 * LW * sizeof(T); /* old fractional rows */
    L.offW = o;
    o += (size_t)RS * 2 * LW * sizeof(T); /* old whole rows */
    L.offRing = o;
    o += (size_t)(2 * ts - 1) * NR * 2 * RW * sizeof(T); /* stage-output rings */
    L.offZ = o;
    o += ZW * sizeof(T); /* a row of zeros */
    o = (o + 15) / 16 * 16;
    L.offR = o;
    o += ((size_t)chunk_n + 4 * ts + 4) * sizeof(T); /* row factors of the item */
    o = (o + 15) / 16 * 16;
    L.offBar = o;
    o += RS * sizeof(uint64_t);
    L.offRed = o;
    o += 33 * sizeof(double);
    L.total = o;
    return L;
}

/* V consecutive values at p (vector loads; p 16-byte aligned, 8 for V = 2 FP32). */
template <typename T, int V>
__device__ __forceinline__ void ld_own(const T* p, T (&x)[V]) {
    if constexpr (sizeof(T) * V == 8) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        x[0] = v.x;
        x[1] = v.y;
    } else if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
    } else {
#pragma unroll
        for (int e = 0; e < V; e += 2) {
            const double2 v = *reinterpret_cast<const double2*>(p + e);
            x[e] = v.x;
            x[e + 1] = v.y;
        }
    }
}

template <typename T, int V>
__device__ __forceinline__ void st_own(T* p, const T (&x)[V]) {
    if constexpr (sizeof(T) * V == 8) {
        *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
    } else if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    } else {
#pragma unroll
        for (int e = 0; e < V; e += 2)
            *reinterpret_cast<double2*>(p + e) = make_double2(x[e], x[e + 1]);
    }
}

/* Central differences of the V columns at p from p[-1] .. p[V]. */
template <typename T, int V>
__device__ __forceinline__ void row_diff(const T* p, T (&d)[V]) {
    T x[V];
    ld_own<T, V>(p, x);
    T left, right;
    if constexpr (sizeof(T) == 4) {
        left = reinterpret_cast<const float2*>(p - 2)->y;
        right = reinterpret_cast<const float2*>(p + V)->x;
    } else {
        left = p[-1];
        right = p[V];
    }
    d[0] = x[1] - left;
#pragma unroll
    for (int e = 1; e < V - 1; ++e) d[e] = x[e + 1] - x[e - 1];
    d[V - 1] = right - x[V - 2];
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename T, int V, int TS>
__global__ void __launch_bounds__(MaxBlock<T, V>::value)
    fused_step_kernel(StepArgs<T> A, int launch_i, int parity) {
    constexpr int H = StepCfg<T>::H;
    constexpr int G = StepCfg<T>::G;
    constexpr int RS = StepCfg<T>::RS;
    constexpr int NR = StepCfg<T>::NR;
    constexpr int NST = 2 * TS;
    extern __shared__ __align__(128) unsigned char smem_raw[];

    const int Wt = A.tile_m;
    const int NT = Wt / V;
    const int NTr = round_warp(NT);
    const int LW = Wt + 2 * H;
    const int RW = Wt + 4 * V;
    const SmemLayout SL = smem_layout<T>(Wt, A.chunk_n, V, TS);
    T* sF = reinterpret_cast<T*>(smem_raw);                /* [RS][2][LW] */
    T* sW = reinterpret_cast<T*>(smem_raw + SL.offW);      /* [RS][2][LW] */
    T* sRing = reinterpret_cast<T*>(smem_raw + SL.offRing); /* [NST-1][NR][2][RW] */
    const T* zrow = reinterpret_cast<const T*>(smem_raw + SL.offZ);
    T* sR = reinterpret_cast<T*>(smem_raw + SL.offR);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + SL.offBar);
    double* red = reinterpret_cast<double*>(smem_raw + SL.offRed);

    const int tid = threadIdx.x;
    const bool is_comp = tid < NT;
    const bool is_prod = tid >= NTr;
    const int lane = tid & 31;
    const bool is_halo = is_prod && lane < 2;
    const int N = A.N, M = A.M, pitch = A.pitch;
    const int ntx = A.ntx;
    const int items = A.ntx * A.nty;
    const int cur = (parity + launch_i) & 1, nxt = cur ^ 1;
    const uint32_t rowbytes = (uint32_t)(LW * sizeof(T));

    pdl_trigger();
    if (tid == NTr) {
        for (int s = 0; s < RS; ++s) mbar_init(smem_u32(&bar[s]), 1);
        fence_proxy_async_smem();
    }
    {
        /* stage rings and the zero row: entries never written stay zero */
        T* z = sRing;
        const int nz = (int)((SL.offR - SL.offRing) / sizeof(T));
        for (int q = tid; q < nz; q += blockDim.x) z[q] = (T)0;
    }

    const long long k = *A.base + launch_i * TS; /* only the counter kernel moves base */
    const int kk = A.P > 0 ? (int)(k % A.P) : 0;
    /* drive at the start and end of every stage (Sec. 2; reading R5) */
    T Es[NST], Ee[NST];
#pragma unroll
    for (int s = 0; s < NST; ++s) {
        const double* tab = (s & 1) ? A.e_frac : A.e_whole;
        Es[s] = (T)tab[kk + s / 2];
        Ee[s] = (T)tab[kk + s / 2 + 1];
    }
    const T h = A.h, hh = A.hh, nu = A.nu, xi = A.xi, cc = A.c;
    const T* gFa = A.a_f[cur];
    const T* gFb = A.b_f[cur];
    const T* gWa = A.a_w[cur];
    const T* gWb = A.b_w[cur];
    T* oWa = A.a_w[nxt];
    T* oFa = A.a_f[nxt];
    const size_t dWb = (size_t)(A.b_w[nxt] - oWa), dFb = (size_t)(A.b_f[nxt] - oFa);
    __syncthreads();

    /* everything below reads the previous launch's state */
    pdl_wait();

    /* rows an item touches: stage s covers [n0 - e_s, n1 + e_s) within [0, N],
     * e_s = NST-1-s; the old rows streamed are R0 = lo_0 - 1 .. R1 = hi_0 */
    auto item_geom = [&](int q, int& n0, int& n1, int& lo0, int& hi0) {
        const int ty = q / ntx;
        n0 = ty * A.chunk_n;
        n1 = min(n0 + A.chunk_n, N + 1);
        lo0 = max(n0 - (NST - 1), 0);
        hi0 = min(n1 + (NST - 1), N + 1);
    };

    /* ---- producer: issues the global stage sequence of this CTA's items ---- */
    int p_item = blockIdx.x, p_s = 0, p_S = 0, p_R0 = 0, p_lo0 = 0, p_hi0 = 0;
    size_t p_col0 = 0;
    long long p_issued = 0, p_freed = 0;
    auto p_load_item = [&]() {
        int n0, n1;
        item_geom(p_item, n0, n1, p_lo0, p_hi0);
        p_R0 = p_lo0 - 1;
        p_S = p_hi0 - p_R0 + 1;
        p_col0 = (size_t)(p_item % ntx) * Wt + (G - H);
    };
    auto pump = [&]() {
        while (p_item < items && p_issued < p_freed + RS) {
            const int row = p_R0 + p_s;
            const int slot = (int)(p_issued & (RS - 1));
            const uint32_t mb = smem_u32(&bar[slot]);
            if (row < 0 || row > N) {
                mbar_arrive(mb);
            } else {
                const bool wneed = row >= p_lo0 && row < p_hi0;
                mbar_arrive_tx(mb, rowbytes * (wneed ? 4u : 2u));
                const size_t off = (size_t)row * pitch + p_col0;
                T* dF = sF + (size_t)slot * 2 * LW;
                bulk_g2s(smem_u32(dF), gFa + off, rowbytes, mb);
                bulk_g2s(smem_u32(dF + LW), gFb + off, rowbytes, mb);
                if (wneed) {
                    T* dW = sW + (size_t)slot * 2 * LW;
                    bulk_g2s(smem_u32(dW), gWa + off, rowbytes, mb);
                    bulk_g2s(smem_u32(dW + LW), gWb + off, rowbytes, mb);
                }
            }
            ++p_issued;
            if (++p_s == p_S) {
                p_s = 0;
                p_item += gridDim.x;
                if (p_item < items) p_load_item();
            }
        }
    };
    if (tid == NTr && p_item < items) {
        p_load_item();
        pump();
    }

    bool timed_out = false;
    long long cbase = 0;   /* global TMA-stage index of the item's first old row */
    long long waited = -1; /* last global TMA stage waited for */

    for (int q = blockIdx.x; q < items; q += gridDim.x) {
        int n0, n1, lo0, hi0;
        item_geom(q, n0, n1, lo0, hi0);
        const int tx = q % ntx;
        const int R0 = lo0 - 1, R1 = hi0;
        const int S = R1 - R0 + 1;
        const int p0 = G + tx * Wt; /* physical column of the tile's first column */

        __syncthreads(); /* the previous item is done with sR and the rings */
        for (int r = tid; r < hi0 - lo0; r += blockDim.x) sR[r] = A.row_a0[lo0 + r];

        /* the thread's V columns: compute threads own tile columns; producer
         * lanes 0/1 take the halo groups left and right of the tile */
        int col;   /* physical column of the group */
        int lcol;  /* index in a streamed row      */
        int rcol;  /* index in a stage ring row    */
        if (is_halo) {
            col = (lane == 0) ? p0 - V : p0 + Wt;
            lcol = (lane == 0) ? H - V : H + Wt;
            rcol = (lane == 0) ? V : 2 * V + Wt;
        } else {
            col = p0 + V * tid;
            lcol = H + V * tid;
            rcol = 2 * V + V * tid;
        }
        const bool active = is_comp || is_halo;
        bool ok[V];
        T g[V], bph[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const int m = col + e - G;
            ok[e] = active && m >= 0 && m <= M;
            g[e] = ok[e] ? A.col_g[col + e] : (T)0;
            bph[e] = ok[e] ? A.col_bphi[col + e] * hh : (T)0;
        }
        const bool all_ok = ok[V - 1] && ok[0];
        __syncthreads(); /* sR ready */

        double pn[TS], pv[TS];
#pragma unroll
        for (int w = 0; w < TS; ++w) pn[w] = pv[w] = 0.0;

        const int j0 = lo0, j1 = min(n1 + 0, N + 1) - 1 + 2 * (NST - 1);
        int jm = ((j0 % NR) + NR) % NR; /* j mod NR */
        for (int j = j0; j <= j1; ++j) {
            /* old rows up to j+1 must have landed */
            const long long need = cbase + (long long)(min(j + 1, R1) - R0);
            while (waited < need) {
                ++waited;
                if (!mbar_wait(smem_u32(&bar[waited & (RS - 1)]), (uint32_t)((waited / RS) & 1)))
                    timed_out = true;
            }
            const long long gj = cbase + (j - R0);
            const int jm1 = (jm + NR - 1) % NR, jm3 = (jm + NR - 3) % NR, jm4 = (jm + NR - 4) % NR;

#pragma unroll
            for (int s = 0; s < NST; ++s) {
                const int e_s = NST - 1 - s;
                const int r = j - 2 * s;
                const int lo = max(n0 - e_s, 0), hi = min(n1 + e_s, N + 1);
                const bool part = is_comp || (is_halo && s < NST - 1);
                if (r < lo || r >= hi || !part) continue;
                /* inputs: own values (row r of the grid being advanced) and the
                 * stencil rows r-1, r+1 of the other grid */
                const T *oa_p, *ob_p, *ua, *ub, *da, *db;
                if (s == 0) {
                    const T* w = sW + (size_t)(gj & (RS - 1)) * 2 * LW;
                    oa_p = w + lcol;
                    ob_p = w + LW + lcol;
                    const T* fu = (r + 1 <= N) ? sF + (size_t)((gj + 1) & (RS - 1)) * 2 * LW : nullptr;
                    const T* fd = (r - 1 >= 0) ? sF + (size_t)((gj - 1) & (RS - 1)) * 2 * LW : nullptr;
                    ua = fu ? fu + lcol : zrow + lcol;
                    ub = fu ? fu + LW + lcol : zrow + lcol;
                    da = fd ? fd + lcol : zrow + lcol;
                    db = fd ? fd + LW + lcol : zrow + lcol;
                } else {
                    if (s == 1) {
                        const T* f = sF + (size_t)((gj - 2) & (RS - 1)) * 2 * LW;
                        oa_p = f + lcol;
                        ob_p = f + LW + lcol;
                    } else {
                        const T* o = sRing + (size_t)((s - 2) * NR + jm4) * 2 * RW;
                        oa_p = o + rcol;
                        ob_p = o + RW + rcol;
                    }
                    const T* prev = sRing + (size_t)(s - 1) * NR * 2 * RW;
                    const T* pu = (r + 1 <= N) ? prev + (size_t)jm1 * 2 * RW : nullptr;
                    const T* pd = (r - 1 >= 0) ? prev + (size_t)jm3 * 2 * RW : nullptr;
                    ua = pu ? pu + rcol : zrow + rcol;
                    ub = pu ? pu + RW + rcol : zrow + rcol;
                    da = pd ? pd + rcol : zrow + rcol;
                    db = pd ? pd + RW + rcol : zrow + rcol;
                }
                T oa[V], ob[V], Dau[V], Dbu[V], Dad[V], Dbd[V];
                ld_own<T, V>(oa_p, oa);
                ld_own<T, V>(ob_p, ob);
                row_diff<T, V>(ua, Dau);
                row_diff<T, V>(ub, Dbu);
                row_diff<T, V>(da, Dad);
                row_diff<T, V>(db, Dbd);
                const T nf = (T)r;
                const T chi = (r == 1) ? (T)2 : (T)1;
                const T ha0 = h * sR[r - lo0];
                const T nEs = nf * hh * Es[s], nEe = nf * hh * Ee[s];
                T an[V], bn[V];
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    T a_, b_;
                    cn_cell<T>(oa[e], ob[e], cc * (Dbu[e] - Dbd[e]), cc * (chi * Dad[e] - Dau[e]),
                               ha0 * g[e], fma_t<T>(nf, bph[e], nEs), fma_t<T>(nf, bph[e], nEe), nu,
                               xi, h, a_, b_);
                    an[e] = ok[e] ? a_ : (T)0;
                    bn[e] = (ok[e] && r > 0) ? b_ : (T)0;
                }
                if (s < NST - 1) {
                    T* o = sRing + (size_t)(s * NR + jm) * 2 * RW;
                    st_own<T, V>(o + rcol, an);
                    st_own<T, V>(o + RW + rcol, bn);
                }
                if (s >= NST - 2 && is_comp && r >= n0 && r < n1) {
                    T* dst = (s == NST - 2) ? oWa + (size_t)r * pitch + col
                                            : oFa + (size_t)r * pitch + col;
                    const size_t db_off = (s == NST - 2) ? dWb : dFb;
                    if (all_ok) {
                        st_own<T, V>(dst, an);
                        st_own<T, V>(dst + db_off, bn);
                    } else {
#pragma unroll
                        for (int e = 0; e < V; ++e)
                            if (ok[e]) {
                                dst[e] = an[e];
                                dst[db_off + e] = bn[e];
                            }
                    }
                }
                if ((s & 1) == 0 && n0 == 0 && is_comp && r <= 1) {
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        if (r == 0) pn[s / 2] += (double)an[e];
                        else pv[s / 2] += (double)bn[e];
                    }
                }
            }
            __syncthreads();
            if (tid == NTr) {
                /* old rows up to j-2 have been read for the last time */
                const long long f = (j == j1) ? cbase + S : gj - 1;
                if (f > p_freed) p_freed = f;
                fence_proxy_async_smem();
                pump();
            }
            /* ---- observables: row 1 of whole grid w is built at j = 4w + 1 ---- */
            if (n0 == 0) {
#pragma unroll
                for (int w = 0; w < TS; ++w) {
                    if (j == 4 * w + 1) {
                        const double sn = block_sum(pn[w], red);
                        const double sv = block_sum(pv[w], red);
                        if (tid == 0) {
                            A.part[(2 * w) * ntx + tx] = sn;
                            A.part[(2 * w + 1) * ntx + tx] = sv;
                            if (w == TS - 1) {
                                __threadfence();
                                const unsigned t = atomicAdd(A.ticket, 1u);
                                if (t == (unsigned)(ntx - 1)) {
                                    __threadfence();
                                    const volatile double* pvv = A.part;
                                    for (int ww = 0; ww < TS; ++ww) {
                                        double s_n = 0, s_v = 0;
                                        for (int u = 0; u < ntx; ++u) {
                                            s_n += pvv[(2 * ww) * ntx + u];
                                            s_v += pvv[(2 * ww + 1) * ntx + u];
                                        }
                                        A.trace_n[k + 1 + ww] = A.nscale * s_n;
                                        A.trace_v[k + 1 + ww] = A.vscale * s_v;
                                    }
                                    *A.ticket = 0u;
                                }
                            }
                        }
                    }
                }
            }
            jm = (jm + 1 == NR) ? 0 : jm + 1;
        }
        cbase += S;
    }
    if (timed_out) atomicExch(A.err, kErrTimeout);
}

}  // namespace

static int ok_or(cudaError_t e) { return e == cudaSuccess ? 0 : (int)e; }

template <typename T>
size_t step_smem_bytes(int tile_m, int chunk_n, int vec, int ts) {
    return smem_layout<T>(tile_m, chunk_n, vec, ts).total;
}

template <typename T>
int step_block_threads(int tile_m, int vec) {
    return round_warp(tile_m / vec) + 32;
}

template <typename T>
int step_max_tile(int vec) {
    if (sizeof(T) == 4 && vec == 2) return 2 * (MaxBlock<float, 2>::value - 32);
    if (sizeof(T) == 4) return 4 * (MaxBlock<float, 4>::value - 32);
    return 2 * (MaxBlock<double, 2>::value - 32);
}

template <typename T>
static const void* step_fn(int vec, int ts) {
    if constexpr (sizeof(T) == 4) {
        if (vec == 4)
            return ts == 2 ? reinterpret_cast<const void*>(&fused_step_kernel<float, 4, 2>)
                           : reinterpret_cast<const void*>(&fused_step_kernel<float, 4, 1>);
        return reinterpret_cast<const void*>(&fused_step_kernel<float, 2, 1>);
    } else {
        return reinterpret_cast<const void*>(&fused_step_kernel<double, 2, 1>);
    }
}

template <typename T>
int step_kernel_configure(int tile_m, int chunk_n, int vec, int ts, int* blocks_per_sm) {
    const size_t bytes = step_smem_bytes<T>(tile_m, chunk_n, vec, ts);
    const void* fn = step_fn<T>(vec, ts);
    cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, step_block_threads<T>(tile_m, vec),
                                                      bytes);
    if (e != cudaSuccess) return (int)e;
    *blocks_per_sm = nb;
    return 0;
}

template <typename T>
int launch_step(const StepArgs<T>& a, int ts, int i, int parity, bool pdl, void* stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.grid);
    cfg.blockDim = dim3(step_block_threads<T>(a.tile_m, a.vec));
    cfg.dynamicSmemBytes = step_smem_bytes<T>(a.tile_m, a.chunk_n, a.vec, ts);
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if constexpr (sizeof(T) == 4) {
        if (a.vec == 4)
            e = ts == 2 ? cudaLaunchKernelEx(&cfg, fused_step_kernel<float, 4, 2>, a, i, parity)
                        : cudaLaunchKernelEx(&cfg, fused_step_kernel<float, 4, 1>, a, i, parity);
        else
            e = cudaLaunchKernelEx(&cfg, fused_step_kernel<float, 2, 1>, a, i, parity);
    } else {
        e = cudaLaunchKernelEx(&cfg, fused_step_kernel<double, 2, 1>, a, i, parity);
    }
    if (e != cudaSuccess) return (int)e;
    return ok_or(cudaGetLastError());
}

#define BTE_STEP_INSTANTIATE(T)                                      \
    template size_t step_smem_bytes<T>(int, int, int, int);          \
    template int step_block_threads<T>(int, int);                    \
    template int step_max_tile<T>(int);                              \
    template int step_kernel_configure<T>(int, int, int, int, int*); \
    template int launch_step<T>(const StepArgs<T>&, int, int, int, bool, void*);
BTE_STEP_INSTANTIATE(float)
BTE_STEP_INSTANTIATE(double)

}  // namespace bte
