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
 *     c = B(t_s) dt / (4 dphi), t_s the time of the grid that supplies S.
 *
 * Work items.  A grid is cut into items of tile_m phi_y columns x chunk_n
 * harmonic rows.  Persistent CTAs take items q = blockIdx.x, +gridDim.x, ...
 * An item is walked upward in n with a one-row lag: at row j the CTA builds
 * the new whole-grid row j (its columns plus one halo column per side) and
 * then the new fractional row j-1, which needs the new whole rows j-2 and j.
 * In the batched form the items of many instances (parameter points, each
 * with its own grid, time step and drive) share one launch; an item first
 * looks up its instance.
 *
 * Threads.  Compute thread t owns V consecutive columns (V = 2 or 4) of the
 * tile.  One extra warp (the producer) issues the TMA bulk copies that
 * stream the old fractional and whole rows into a ring of RS shared-memory
 * stages (cp.async.bulk + mbarrier, RS-2 rows ahead of use, continuing
 * across items), and computes the two halo cells of each new whole row.
 *
 * Data reuse.  Every old fractional row is read from shared memory once per
 * thread when it arrives; its own values and central differences stay in
 * registers for the two rows that use them.  A new whole row goes to
 * shared memory once (for the neighbours' differences) and straight from
 * registers to global memory; the new fractional row goes from registers to
 * global memory.  One __syncthreads per row.
 *
 * Launch.  Programmatic dependent launch: the prologue (barrier set-up)
 * runs while the previous step drains; griddepcontrol.wait precedes the
 * first read of the state.
 *
 * Observables (Sec. 2, Eqs. v_dr_generic and norm_in_phi): items that own
 * rows 0 and 1 reduce sum_m a_{0,m} and sum_m b_{1,m} in FP64; the last of
 * them to arrive adds the per-tile partials in tile order, so the results
 * are bitwise reproducible.  A single instance writes the sample to its
 * trace; a batched instance adds it to its window sums (Eq. absorption_def).
 *
 * Every mbarrier wait is bounded (~2 s of %globaltimer).  A wait that gives
 * up on any thread ends the launch at the next row barrier: the producer
 * issues nothing more, waits (bounded again) for the bulk copies it already
 * issued, so that no copy is still writing shared memory when the CTA
 * exits, and the kernel records an error word that the host reports as
 * BTE_ETIMEOUT.
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
    static constexpr int H = Cols<T>::H;
    static constexpr int G = Cols<T>::G;
    static constexpr int RS = sizeof(T) == 4 ? 8 : 6; /* TMA ring stages */
};

/* largest block: 512 compute threads + producer warp for FP32 with V = 2,
 * 256 + 32 otherwise (FP64 needs the registers) */
template <typename T, int V>
struct MaxBlock {
    static constexpr int value = (sizeof(T) == 4 && V == 2) ? 544 : 288;
};

__host__ __device__ inline int round_warp(int n) { return (n + 31) / 32 * 32; }

template <typename T>
__host__ __device__ inline size_t smem_layout(int tile_m, int chunk_n, int V, size_t* offN,
                                              size_t* offR, size_t* offBar, size_t* offRed) {
    constexpr int H = StepCfg<T>::H, RS = StepCfg<T>::RS;
    const size_t LW = (size_t)tile_m + 2 * H;
    const size_t WN = (size_t)tile_m + 2 * V;
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

/* V consecutive values at p (vector loads; p is aligned to V elements or 16 bytes). */
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

/* Left and right neighbours p[-1], p[V] of a group. */
template <typename T, int V>
__device__ __forceinline__ void neighbours(const T* p, T& left, T& right) {
    if constexpr (sizeof(T) == 4) {
        left = reinterpret_cast<const float2*>(p - 2)->y;
        right = reinterpret_cast<const float2*>(p + V)->x;
    } else {
        left = p[-1];
        right = p[V];
    }
}

/* Central differences of a group from its own values and neighbours. */
template <typename T, int V>
__device__ __forceinline__ void diffs(const T (&own)[V], T left, T right, T (&d)[V]) {
    d[0] = own[1] - left;
#pragma unroll
    for (int e = 1; e < V - 1; ++e) d[e] = own[e + 1] - own[e - 1];
    d[V - 1] = right - own[V - 2];
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

/* What an item needs to know about its instance for the current step. */
template <typename T>
struct View {
    const T *gFa, *gFb, *gWa, *gWb; /* old state (set cur)          */
    T *oWa, *oFa;                    /* new state (set nxt)          */
    size_t dWb, dFb;                 /* b array offset from a array  */
    const T *row_a0, *col_g, *col_phi;
    double *part;
    unsigned* ticket;
    int N, M, pitch, ntx, inst, q0; /* q0: the instance's first item */
    long long k;
    bool active;                     /* instance still running       */
    T Ews, Ewe, Efs, Efe; /* E at the start / end of the whole and fractional half-steps */
    T Bws, Bwe, Bfs, Bfe; /* B at the same times                                         */
    T ccw, ccf;           /* stencil coefficients of the two half-steps                   */
    T h, hh, nu, xi;
};

/* Drive of the half-steps of step k (kk = k mod P): E and B at the start and
 * end of each half-step and the two stencil coefficients, from the
 * [3][stride] tables (FP64 values rounded to T once on the host, so no
 * conversion here). */
template <typename T>
__device__ __forceinline__ void drive(View<T>& v, const T* ew, const T* ef, int stride, int kk) {
    v.Ews = ew[kk];
    v.Ewe = ew[kk + 1];
    v.Efs = ef[kk];
    v.Efe = ef[kk + 1];
    v.Bws = ew[stride + kk];
    v.Bwe = ew[stride + kk + 1];
    v.Bfs = ef[stride + kk];
    v.Bfe = ef[stride + kk + 1];
    v.ccw = ew[2 * stride + kk];
    v.ccf = ef[2 * stride + kk];
}

/* Instance of item q: single-instance launches use A; batched ones look the
 * instance up in the item -> instance table. */
template <typename T, bool BATCH>
__device__ __forceinline__ void make_view(View<T>& v, int q, const StepArgs<T>& A,
                                          const BatchArgs<T>& Bt, long long kbase, int cur,
                                          bool with_drive) {
    if constexpr (!BATCH) {
        v.gFa = A.a_f[cur];
        v.gFb = A.b_f[cur];
        v.gWa = A.a_w[cur];
        v.gWb = A.b_w[cur];
        v.oWa = A.a_w[cur ^ 1];
        v.oFa = A.a_f[cur ^ 1];
        v.dWb = (size_t)(A.b_w[cur ^ 1] - v.oWa);
        v.dFb = (size_t)(A.b_f[cur ^ 1] - v.oFa);
        v.row_a0 = A.row_a0;
        v.col_g = A.col_g;
        v.col_phi = A.col_phi;
        /* a persistent launch may have several steps in flight: slot k % dring */
        const int slot = A.dring > 1 ? (int)(kbase % A.dring) : 0;
        v.part = A.part + (size_t)slot * 2 * A.ntx;
        v.ticket = A.ticket + slot;
        v.N = A.N;
        v.M = A.M;
        v.pitch = A.pitch;
        v.ntx = A.ntx;
        v.inst = 0;
        v.q0 = 0;
        v.k = kbase;
        v.active = true;
        if (with_drive) {
            const int kk = A.P > 0 ? (int)(kbase % A.P) : 0;
            drive<T>(v, A.e_whole, A.e_frac, A.dstride, kk);
            v.h = A.h;
            v.hh = A.hh;
            v.nu = A.nu;
            v.xi = A.xi;
        }
    } else {
        const int lo = __ldg(Bt.item_inst + q);
        const BatchInst<T>& I = Bt.inst[lo];
        v.inst = lo;
        v.q0 = I.item0;
        v.gFa = I.a_f[cur];
        v.gFb = I.b_f[cur];
        v.gWa = I.a_w[cur];
        v.gWb = I.b_w[cur];
        v.oWa = I.a_w[cur ^ 1];
        v.oFa = I.a_f[cur ^ 1];
        v.dWb = (size_t)(I.b_w[cur ^ 1] - v.oWa);
        v.dFb = (size_t)(I.b_f[cur ^ 1] - v.oFa);
        v.row_a0 = I.row_a0;
        v.col_g = I.col_g;
        v.col_phi = I.col_phi;
        v.part = I.part;
        v.ticket = I.ticket;
        v.N = I.N;
        v.M = I.M;
        v.pitch = I.pitch;
        v.ntx = I.ntx;
        v.k = kbase;
        v.active = kbase < I.K;
        if (with_drive && v.active) {
            const int kk = I.P > 0 ? (int)(kbase % I.P) : 0;
            drive<T>(v, I.e_whole, I.e_frac, I.dstride, kk);
            v.h = I.h;
            v.hh = I.hh;
            v.nu = I.nu;
            v.xi = I.xi;
        }
    }
}

/* Dependencies of item (tx, ty) before its step `target` of a persistent
 * launch: every item of the 3 x 3 block of tiles and chunks around it must
 * have completed `target` steps (it reads their rows and halo columns of
 * the step before, and overwrites the set they read in it).  Called by one
 * whole warp: lane i < 9 polls neighbour i, so the counters are read in
 * parallel; the spin is bounded by %globaltimer and stops early when
 * another CTA has recorded an error.  The result is the same on every
 * lane: false when the wait gave up. */
__device__ __forceinline__ bool wait_neighbours(const unsigned* done, int tx, int ty, int ntx,
                                                int nty, unsigned target, const int* err) {
    const int lane = threadIdx.x & 31;
    const int x = tx + lane % 3 - 1, y = ty + lane / 3 - 1;
    const bool mine = lane < 9 && lane != 4 && x >= 0 && x < ntx && y >= 0 && y < nty;
    const unsigned* c = done + (size_t)(mine ? y : 0) * ntx + (mine ? x : 0);
    bool ready = !mine || ld_acquire(c) >= target;
    if (__all_sync(0xffffffffu, ready)) return true;
    const uint64_t t0 = global_timer();
    for (;;) {
        if (!ready) ready = ld_acquire(c) >= target;
        if (__all_sync(0xffffffffu, ready)) return true;
        const bool stop = *reinterpret_cast<const volatile int*>(err) != 0 ||
                          global_timer() - t0 > kWaitLimitNs;
        if (__any_sync(0xffffffffu, stop)) return false;
    }
}

/* One launch: step base + launch_i (one step), or A.nsteps steps of a
 * persistent launch.  DOWN fixes the direction of the row walks (see the
 * consumer loop): where the state is larger than L2 the host alternates it
 * between consecutive one-step launches (launch_i even: upward, odd:
 * downward), so that every step starts with the rows the step before wrote
 * last -- the ones still in L2 (2049 x 8193 FP32: 537 MB of state against
 * 129 MB of L2).  The two
 * directions are separate instantiations, so each keeps its own register
 * allocation.  A persistent launch walks upward every step. */
template <typename T, int V, bool BATCH, bool PERSIST, bool DOWN>
__global__ void __launch_bounds__(MaxBlock<T, V>::value)
    fused_step_kernel(StepArgs<T> A, BatchArgs<T> Bt, int launch_i, int parity) {
    constexpr int H = StepCfg<T>::H;
    constexpr int G = StepCfg<T>::G;
    constexpr int RS = StepCfg<T>::RS;
    extern __shared__ __align__(128) unsigned char smem_raw[];

    const int Wt = BATCH ? Bt.tile_m : A.tile_m;
    const int chunk = BATCH ? Bt.chunk_n : A.chunk_n;
    const int NT = Wt / V;
    const int NTr = round_warp(NT);
    const int LW = Wt + 2 * H;
    const int WN = Wt + 2 * V;
    size_t offN, offR, offBar, offRed;
    smem_layout<T>(Wt, chunk, V, &offN, &offR, &offBar, &offRed);
    T* sF = reinterpret_cast<T*>(smem_raw);        /* [RS][2][LW] */
    T* sW = sF + (size_t)RS * 2 * LW;              /* [RS][2][LW] */
    T* sN = reinterpret_cast<T*>(smem_raw + offN); /* [2][2][WN]  */
    T* sR = reinterpret_cast<T*>(smem_raw + offR); /* [chunk_n+4] */
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + offBar);
    double* red = reinterpret_cast<double*>(smem_raw + offRed);

    const int tid = threadIdx.x;
    const bool is_comp = tid < NT;
    const bool is_prod = tid >= NTr;
    const int lane = tid & 31;
    const int items = BATCH ? Bt.items : A.ntx * A.nty;
    const uint32_t rowbytes = (uint32_t)(LW * sizeof(T));

    pdl_trigger();
    if (tid == NTr) {
        for (int s = 0; s < RS; ++s) mbar_init(smem_u32(&bar[s]), 1);
        fence_proxy_async_smem();
    }
    /* new-row buffers: entries outside the tile's columns +-1 stay zero */
    for (int q = tid; q < 4 * WN; q += blockDim.x) sN[q] = (T)0;
    /* only the counter kernel moves base */
    const long long kbase0 = *(BATCH ? Bt.base : A.base) + launch_i;
    const int cur0 = (parity + launch_i) & 1;
    __syncthreads();

    /* everything below reads the previous step's state */
    pdl_wait();

    /* ---- producer: issues the global stage sequence of this CTA's items ---- */
    int p_item = blockIdx.x, p_s = 0, p_S = 0, p_n0 = 0, p_n1 = 0, p_N = 0;
    size_t p_col0 = 0, p_pitch = 0;
    const T *p_Fa = nullptr, *p_Fb = nullptr, *p_Wa = nullptr, *p_Wb = nullptr;
    int p_slot = 0;
    long long p_issued = 0, p_freed = 0;
    /* first item at or after p_item whose instance is still running */
    auto p_load_item = [&](long long kb, int cr) {
        while (p_item < items) {
            View<T> v;
            make_view<T, BATCH>(v, p_item, A, Bt, kb, cr, false);
            if (v.active) {
                const int ql = p_item - v.q0;
                const int ty = ql / v.ntx;
                p_n0 = ty * chunk;
                p_n1 = min(p_n0 + chunk, v.N + 1);
                p_S = p_n1 - p_n0 + 4;
                p_N = v.N;
                p_pitch = (size_t)v.pitch;
                p_col0 = (size_t)(ql - ty * v.ntx) * Wt + (G - H);
                p_Fa = v.gFa;
                p_Fb = v.gFb;
                p_Wa = v.gWa;
                p_Wb = v.gWb;
                return;
            }
            p_item += gridDim.x;
        }
    };
    auto pump = [&](long long kb, int cr) {
        while (p_item < items && p_issued < p_freed + RS) {
            const int row = DOWN ? p_n1 + 1 - p_s : p_n0 - 2 + p_s;
            const uint32_t mb = smem_u32(&bar[p_slot]);
            if (row < 0 || row > p_N) {
                mbar_arrive(mb);
            } else {
                const bool wneed = row >= p_n0 - 1 && row <= p_n1;
                mbar_arrive_tx(mb, rowbytes * (wneed ? 4u : 2u));
                const size_t off = (size_t)row * p_pitch + p_col0;
                T* dF = sF + (size_t)p_slot * 2 * LW;
                bulk_g2s(smem_u32(dF), p_Fa + off, rowbytes, mb);
                bulk_g2s(smem_u32(dF + LW), p_Fb + off, rowbytes, mb);
                if (wneed) {
                    T* dW = sW + (size_t)p_slot * 2 * LW;
                    bulk_g2s(smem_u32(dW), p_Wa + off, rowbytes, mb);
                    bulk_g2s(smem_u32(dW + LW), p_Wb + off, rowbytes, mb);
                }
            }
            ++p_issued;
            p_slot = (p_slot + 1 == RS) ? 0 : p_slot + 1;
            if (++p_s == p_S) {
                p_s = 0;
                p_item += gridDim.x;
                p_load_item(kb, cr);
            }
        }
    };
    bool timed_out = false; /* a bounded wait of this thread gave up        */
    bool aborted = false;   /* some thread's did: the launch stops          */
    long long cbase = 0; /* global stage index of the current item's stage 0 */
    int c_slot = 0;      /* ring slot of the stage being consumed         */
    uint32_t c_phase = 0;

    /* One step: step kbase, reading ping-pong set cur.  A launch runs one
     * step, or A.nsteps steps of a persistent launch with a grid barrier
     * between them; the ring's stage counters and barrier phases run on
     * across steps, and the producer starts a step's copies only after the
     * barrier, when every CTA's writes of the step before are complete. */
    auto run_step = [&](const long long kbase, const int cur) {
        if (tid == NTr) {
            p_item = blockIdx.x;
            p_s = 0;
            p_load_item(kbase, cur);
            pump(kbase, cur);
        }

        for (int q = blockIdx.x; q < items; q += gridDim.x) {
            View<T> I;
            make_view<T, BATCH>(I, q, A, Bt, kbase, cur, true);
            if (!I.active) continue; /* uniform: every thread sees the same instance */
            const int N = I.N, M = I.M, pitch = I.pitch, ntx = I.ntx;
            const int ql = q - I.q0;
            const int ty = ql / ntx;
            const int tx = ql - ty * ntx;
            const int n0 = ty * chunk;
            const int n1 = min(n0 + chunk, N + 1);
            const int S = n1 - n0 + 4;
            const int p0 = G + tx * Wt; /* physical column of the tile's first column */
            using O = Rn<T>;
            const T h = I.h, hh = I.hh, ccw = I.ccw, ccf = I.ccf;
            const CnK<T> K = cn_constants<T>(h, I.nu, I.xi);

            __syncthreads(); /* the previous item is done with sR and sN */
            for (int r = tid; r < n1 - n0 + 2; r += blockDim.x) {
                const int n = n0 - 1 + r;
                sR[r] = (n >= 0 && n <= N) ? I.row_a0[n] : (T)0;
            }

            /* per-column constants of the thread's V columns */
            const int c = p0 + V * tid; /* physical column of the group      */
            const int lc = H + V * tid; /* its index in a streamed row       */
            const int ln = V + V * tid; /* its index in a new whole row      */
            bool ok[V];
            T g[V], ws[V], we[V], fs[V], fe[V];
    #pragma unroll
            for (int e = 0; e < V; ++e) {
                ok[e] = is_comp && (c + e - G) <= M;
                const T ph = ok[e] ? I.col_phi[c + e] : (T)0;
                g[e] = ok[e] ? I.col_g[c + e] : (T)0;
                ws[e] = rot_factor<T>(I.Ews, I.Bws, ph, hh);
                we[e] = rot_factor<T>(I.Ewe, I.Bwe, ph, hh);
                fs[e] = rot_factor<T>(I.Efs, I.Bfs, ph, hh);
                fe[e] = rot_factor<T>(I.Efe, I.Bfe, ph, hh);
            }
            const bool all_ok = ok[V - 1];

            /* producer lane 0: the halo columns p0-1 and p0+Wt of new whole
             * rows, as one pair of cells (the same paired arithmetic as the
             * compute threads' cells) */
            const bool hlane = is_prod && lane == 0;
            bool hok[2];
            int hlc[2], hidx[2];
            T hg[2], hbs[2], hbe[2];
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const int hcol = s2 == 0 ? p0 - 1 : p0 + Wt;
                hok[s2] = hlane && (hcol - G) >= 0 && (hcol - G) <= M;
                hlc[s2] = hcol - (p0 - H);
                hidx[s2] = s2 == 0 ? V - 1 : V + Wt;
                hg[s2] = hbs[s2] = hbe[s2] = (T)0;
                if (hok[s2]) {
                    hg[s2] = I.col_g[hcol];
                    const T ph = I.col_phi[hcol];
                    hbs[s2] = rot_factor<T>(I.Ews, I.Bws, ph, hh);
                    hbe[s2] = rot_factor<T>(I.Ewe, I.Bwe, ph, hh);
                }
            }
            __syncthreads(); /* sR ready */

            /* rolling windows (registers): old fractional rows j-1, j (own
             * values and central differences), central differences of new whole
             * rows j-2, j-1 */
            T fa_m1[V], fb_m1[V], fa_0[V], fb_0[V];
            T dfa_m1[V], dfb_m1[V], dfa_0[V], dfb_0[V];
            T dwa_m2[V], dwb_m2[V], dwa_m1[V], dwb_m1[V];
    #pragma unroll
            for (int e = 0; e < V; ++e) {
                fa_m1[e] = fb_m1[e] = fa_0[e] = fb_0[e] = (T)0;
                dfa_m1[e] = dfb_m1[e] = dfa_0[e] = dfb_0[e] = (T)0;
                dwa_m2[e] = dwb_m2[e] = dwa_m1[e] = dwb_m1[e] = (T)0;
            }
            double part_n = 0.0, part_v = 0.0;
            int slot_m1 = 0, slot_m2 = 0; /* ring slots of the two previous stages */

            /* Row walk.  Upward (even steps): iteration j (j =
             * n0 - 3 .. n1, stage si = j - n0 + 3) works on new whole row j
             * after old row j + 1 arrived, and on new fractional row j - 1.
             * Downward (odd steps), the mirror image: j = n1 + 2 .. n0 - 1
             * (stage si = n1 + 2 - j), old row j - 1 arrives, fractional row
             * j + 1 follows.  Each step then starts
             * with the rows the previous step wrote last, which are still in
             * L2.  The per-cell arithmetic is the same either way.  Stages 0
             * and 1 are consumed by the load-only first two iterations. */
            constexpr int dj = DOWN ? -1 : 1;
            for (int j = DOWN ? n1 + 2 : n0 - 3; DOWN ? j >= n0 - 1 : j <= n1; j += dj) {
                if (!mbar_wait(smem_u32(&bar[c_slot]), c_phase)) timed_out = true;
                const T* ra = sF + (size_t)c_slot * 2 * LW; /* the old fractional row that arrived */
                const int jn = DOWN ? j - 1 : j + 1;         /* its index */

                T fa_p1[V], fb_p1[V], dfa_p1[V], dfb_p1[V]; /* row jn */
                if (jn >= 0 && jn <= N && is_comp) {
                    T l, r;
                    ld_own<T, V>(ra + lc, fa_p1);
                    neighbours<T, V>(ra + lc, l, r);
                    diffs<T, V>(fa_p1, l, r, dfa_p1);
                    ld_own<T, V>(ra + LW + lc, fb_p1);
                    neighbours<T, V>(ra + LW + lc, l, r);
                    diffs<T, V>(fb_p1, l, r, dfb_p1);
                } else {
    #pragma unroll
                    for (int e = 0; e < V; ++e) fa_p1[e] = fb_p1[e] = dfa_p1[e] = dfb_p1[e] = (T)0;
                }

                if (DOWN ? j <= n1 : j >= n0 - 1) { /* from the third stage on */
                    /* ---- new whole-grid row j ---- */
                    const bool wrow_ok = j >= 0 && j <= N;
                    T wa_n[V], wb_n[V];
                    T* na = sN + (size_t)(j & 1) * 2 * WN;
                    if (wrow_ok) {
                        const T nf = (T)j;
                        const T chi = (j == 1) ? (T)2 : (T)1;
                        const T hr = O::mul(h, sR[j - n0 + 1]);
                        const T* wa = sW + (size_t)slot_m1 * 2 * LW; /* old whole row j */
                        if (is_comp) {
                            T oa[V], ob[V];
                            ld_own<T, V>(wa + lc, oa);
                            ld_own<T, V>(wa + LW + lc, ob);
                                T an[V], bn[V];
                            /* differences of old fractional rows j + 1 (next) and j - 1 (prev) */
                            if constexpr (!DOWN)
                                cn_row<T, V>(oa, ob, dfb_p1, dfb_m1, dfa_m1, dfa_p1, ccw, chi, hr, g,
                                             nf, ws, we, K, an, bn);
                            else
                                cn_row<T, V>(oa, ob, dfb_m1, dfb_p1, dfa_p1, dfa_m1, ccw, chi, hr, g,
                                             nf, ws, we, K, an, bn);
#pragma unroll
                            for (int e = 0; e < V; ++e) {
                                wa_n[e] = ok[e] ? an[e] : (T)0;
                                wb_n[e] = (ok[e] && j > 0) ? bn[e] : (T)0;
                            }
                            st_own<T, V>(na + ln, wa_n);
                            st_own<T, V>(na + WN + ln, wb_n);
                            if (j >= n0 && j < n1) {
                                T* wrow = I.oWa + (size_t)j * pitch + c;
                                if (all_ok) {
                                    st_own<T, V>(wrow, wa_n);
                                    st_own<T, V>(wrow + I.dWb, wb_n);
                                } else {
    #pragma unroll
                                    for (int e = 0; e < V; ++e)
                                        if (ok[e]) {
                                            wrow[e] = wa_n[e];
                                            wrow[I.dWb + e] = wb_n[e];
                                        }
                                }
                            }
                            if (n0 == 0 && j <= 1) {
    #pragma unroll
                                for (int e = 0; e < V; ++e) {
                                    if (j == 0) part_n += (double)wa_n[e];
                                    if (j == 1) part_v += (double)wb_n[e];
                                }
                            }
                        } else if (hlane) {
                            /* old fractional rows j - 1 and j + 1: the one that
                             * arrived now and the one two stages back */
                            const T* f2 = sF + (size_t)slot_m2 * 2 * LW;
                            const T* fd = DOWN ? ra : f2; /* row j - 1 */
                            const T* fu = DOWN ? f2 : ra; /* row j + 1 */
                            const bool dn = j - 1 >= 0, up = j + 1 <= N;
                            T oa2[2], ob2[2], dad[2], dbd[2], dau[2], dbu[2], an2[2], bn2[2];
#pragma unroll
                            for (int s2 = 0; s2 < 2; ++s2) {
                                const int c2 = hlc[s2];
                                oa2[s2] = wa[c2];
                                ob2[s2] = wa[LW + c2];
                                dad[s2] = dn ? fd[c2 + 1] - fd[c2 - 1] : (T)0;
                                dbd[s2] = dn ? fd[LW + c2 + 1] - fd[LW + c2 - 1] : (T)0;
                                dau[s2] = up ? fu[c2 + 1] - fu[c2 - 1] : (T)0;
                                dbu[s2] = up ? fu[LW + c2 + 1] - fu[LW + c2 - 1] : (T)0;
                            }
                            cn_row<T, 2>(oa2, ob2, dbu, dbd, dad, dau, ccw, chi, hr, hg, nf, hbs,
                                         hbe, K, an2, bn2);
#pragma unroll
                            for (int s2 = 0; s2 < 2; ++s2) {
                                na[hidx[s2]] = hok[s2] ? an2[s2] : (T)0;
                                na[WN + hidx[s2]] = (hok[s2] && j > 0) ? bn2[s2] : (T)0;
                            }
                        }
                    }
                    /* the row barrier; it also ends the launch when a wait gave up */
                    if (__syncthreads_or(timed_out)) {
                        aborted = true;
                        if (tid == 0) atomicExch(BATCH ? Bt.err : A.err, kErrTimeout);
                        break;
                    }
                    if (tid == NTr) {
                        /* every stage before stage si - 1 (si: this iteration's
                         * stage) has been read for the last time; all of them
                         * after the last iteration */
                        const long long si = DOWN ? n1 + 2 - j : j - n0 + 3;
                        const long long f = (si == S - 1) ? cbase + S : cbase + si - 1;
                        if (f > p_freed) p_freed = f;
                        fence_proxy_async_smem();
                        pump(kbase, cur);
                    }

                    /* ---- new fractional row j-1 ---- */
                    T dwa_0[V], dwb_0[V];
                    if (wrow_ok && is_comp) {
                        T l, r;
                        neighbours<T, V>(na + ln, l, r);
                        diffs<T, V>(wa_n, l, r, dwa_0);
                        neighbours<T, V>(na + WN + ln, l, r);
                        diffs<T, V>(wb_n, l, r, dwb_0);
                    } else {
    #pragma unroll
                        for (int e = 0; e < V; ++e) dwa_0[e] = dwb_0[e] = (T)0;
                    }
                    /* ---- new fractional row r, one behind: it needs new whole
                     * rows r - 1 and r + 1, the one just made (dw_0) and the
                     * one two rows back (dw_m2) ---- */
                    const int r = DOWN ? j + 1 : j - 1;
                    if (r >= n0 && r < n1 && is_comp && ok[0]) {
                        const T nf = (T)r;
                        const T chi = (r == 1) ? (T)2 : (T)1;
                        const T hr = O::mul(h, sR[r - n0 + 1]);
                        T fa_n[V], fb_n[V];
                        if constexpr (!DOWN)
                            cn_row<T, V>(fa_m1, fb_m1, dwb_0, dwb_m2, dwa_m2, dwa_0, ccf, chi, hr, g,
                                         nf, fs, fe, K, fa_n, fb_n);
                        else
                            cn_row<T, V>(fa_m1, fb_m1, dwb_m2, dwb_0, dwa_0, dwa_m2, ccf, chi, hr, g,
                                         nf, fs, fe, K, fa_n, fb_n);
                        if (r == 0) {
#pragma unroll
                            for (int e = 0; e < V; ++e) fb_n[e] = (T)0;
                        }
                        T* frow = I.oFa + (size_t)r * pitch + c;
                        if (all_ok) {
                            st_own<T, V>(frow, fa_n);
                            st_own<T, V>(frow + I.dFb, fb_n);
                        } else {
    #pragma unroll
                            for (int e = 0; e < V; ++e)
                                if (ok[e]) {
                                    frow[e] = fa_n[e];
                                    frow[I.dFb + e] = fb_n[e];
                                }
                        }
                    }

                    /* ---- observables of rows 0 and 1, once both are made ---- */
                    if (n0 == 0 && j == (DOWN ? 0 : 1)) {
                        const double sn = block_sum(part_n, red);
                        const double sv = block_sum(part_v, red);
                        if (tid == 0) {
                            I.part[tx] = sn;
                            I.part[ntx + tx] = sv;
                            __threadfence();
                            const unsigned t = atomicAdd(I.ticket, 1u);
                            if (t == (unsigned)(ntx - 1)) {
                                __threadfence();
                                double s_n = 0, s_v = 0;
                                const volatile double* pv = I.part;
                                for (int u = 0; u < ntx; ++u) {
                                    s_n += pv[u];
                                    s_v += pv[ntx + u];
                                }
                                if constexpr (!BATCH) {
                                    A.trace_n[kbase + 1] = A.nscale * s_n;
                                    A.trace_v[kbase + 1] = A.vscale * s_v;
                                } else {
                                    /* window sums of Eq. absorption_def, FP64, one writer
                                     * per instance and step */
                                    const BatchInst<T>& B = Bt.inst[I.inst];
                                    const double vv = B.vscale * s_v, nn = B.nscale * s_n;
                                    const long long k1 = kbase + 1;
                                    double* acc = B.acc;
                                    if (k1 > B.K - B.Kw) {
                                        const double ang =
                                            B.P > 0 ? 6.283185307179586476925286766559 *
                                                          (double)(k1 % B.P) / (double)B.P
                                                    : B.omega * (double)k1 * B.dt_eff;
                                        acc[0] += vv * cos(ang);
                                        acc[1] += vv;
                                    }
                                    acc[2] = fmax(acc[2], fabs(nn - 1.0));
                                    if (!isfinite(vv) || !isfinite(nn)) acc[3] = 1.0;
                                    acc[4] = vv;
                                    acc[5] = nn;
                                }
                                *I.ticket = 0u;
                            }
                        }
                    }
    #pragma unroll
                    for (int e = 0; e < V; ++e) {
                        dwa_m2[e] = dwa_m1[e];
                        dwb_m2[e] = dwb_m1[e];
                        dwa_m1[e] = dwa_0[e];
                        dwb_m1[e] = dwb_0[e];
                    }
                }
    #pragma unroll
                for (int e = 0; e < V; ++e) {
                    fa_m1[e] = fa_0[e];
                    fb_m1[e] = fb_0[e];
                    fa_0[e] = fa_p1[e];
                    fb_0[e] = fb_p1[e];
                    dfa_m1[e] = dfa_0[e];
                    dfb_m1[e] = dfb_0[e];
                    dfa_0[e] = dfa_p1[e];
                    dfb_0[e] = dfb_p1[e];
                }
                slot_m2 = slot_m1;
                slot_m1 = c_slot;
                if (++c_slot == RS) {
                    c_slot = 0;
                    c_phase ^= 1u;
                }
            }
            if (aborted) break;
            cbase += S;
        }
    };
    if constexpr (!PERSIST) {
        run_step(kbase0, cur0);
    } else {
        /* one item per CTA (gridDim.x == ntx * nty), every step */
        const int tx = (int)blockIdx.x % A.ntx, ty = (int)blockIdx.x / A.ntx;
        for (int st = 0; st < A.nsteps; ++st) {
            if (st > 0) {
                bool gave_up = false;
                if (tid < 32)
                    gave_up = !wait_neighbours(A.done, tx, ty, A.ntx, A.nty, (unsigned)st, A.err);
                if (__syncthreads_or(gave_up)) {
                    aborted = true;
                    if (tid == 0) atomicExch(A.err, kErrTimeout);
                    break;
                }
                /* the neighbours' stores, seen by this CTA's bulk copies (async proxy) */
                if (tid == NTr) asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            run_step(kbase0 + st, (cur0 + st) & 1);
            if (aborted) break;
            /* this thread's stores of the step, before another CTA's bulk
             * copies read them; then the item's completion count */
            asm volatile("fence.proxy.async.global;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                st_release(A.done + blockIdx.x, (unsigned)(st + 1));
            }
        }
    }
    if (aborted && tid == NTr) {
        /* Drain: every stage issued and not yet seen complete lies among the
         * last RS issued (a slot is re-armed only after a row barrier that no
         * timeout preceded), and no slot holds two of them, so stage s
         * completes phase (s / RS) & 1 of slot s % RS. */
        const long long first = p_issued > RS ? p_issued - RS : 0;
        for (long long s = first; s < p_issued; ++s)
            if (!mbar_wait(smem_u32(&bar[(int)(s % RS)]), (uint32_t)((s / RS) & 1))) break;
    }
    if ((timed_out || aborted) && tid == 0) atomicExch(BATCH ? Bt.err : A.err, kErrTimeout);
}

}  // namespace

static int ok_or(cudaError_t e) { return e == cudaSuccess ? 0 : (int)e; }

template <typename T>
size_t step_smem_bytes(int tile_m, int chunk_n, int vec) {
    size_t a, b, c, d;
    return smem_layout<T>(tile_m, chunk_n, vec, &a, &b, &c, &d);
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

template <typename T, bool BATCH, bool PERSIST, bool DOWN>
static const void* step_fn(int vec) {
    if constexpr (sizeof(T) == 4)
        return vec == 4
                   ? reinterpret_cast<const void*>(&fused_step_kernel<float, 4, BATCH, PERSIST, DOWN>)
                   : reinterpret_cast<const void*>(&fused_step_kernel<float, 2, BATCH, PERSIST, DOWN>);
    else
        return reinterpret_cast<const void*>(&fused_step_kernel<double, 2, BATCH, PERSIST, DOWN>);
}

template <typename T, bool BATCH, bool PERSIST>
static int configure(int tile_m, int chunk_n, int vec, int* blocks_per_sm) {
    const size_t bytes = step_smem_bytes<T>(tile_m, chunk_n, vec);
    const void* fn = step_fn<T, BATCH, PERSIST, false>(vec);
    cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    if (!PERSIST) {
        e = cudaFuncSetAttribute(step_fn<T, BATCH, PERSIST, true>(vec),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return (int)e;
    }
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, step_block_threads<T>(tile_m, vec),
                                                      bytes);
    if (e != cudaSuccess) return (int)e;
    *blocks_per_sm = nb;
    return 0;
}

template <typename T>
int step_kernel_configure(int tile_m, int chunk_n, int vec, int* blocks_per_sm) {
    return configure<T, false, false>(tile_m, chunk_n, vec, blocks_per_sm);
}

template <typename T>
int step_kernel_configure_persist(int tile_m, int chunk_n, int vec, int* blocks_per_sm) {
    return configure<T, false, true>(tile_m, chunk_n, vec, blocks_per_sm);
}

template <typename T>
int step_kernel_configure_batch(int tile_m, int chunk_n, int vec, int* blocks_per_sm) {
    return configure<T, true, false>(tile_m, chunk_n, vec, blocks_per_sm);
}

template <typename T, bool BATCH, bool PERSIST>
static int launch(const StepArgs<T>& a, const BatchArgs<T>& b, int grid, int tile_m, int chunk_n,
                  int vec, int i, int parity, bool pdl, void* stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(step_block_threads<T>(tile_m, vec));
    cfg.dynamicSmemBytes = step_smem_bytes<T>(tile_m, chunk_n, vec);
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    if (PERSIST) {
        /* every CTA must be resident at once (the grid barrier waits for all) */
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
    } else {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    }
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    /* one-step launches of a state larger than L2 alternate the row-walk
     * direction with launch_i */
    const bool down = !PERSIST && (BATCH ? b.alt : a.alt) && (i & 1);
    if constexpr (sizeof(T) == 4) {
        if (vec == 4)
            e = down ? cudaLaunchKernelEx(&cfg, fused_step_kernel<float, 4, BATCH, PERSIST, !PERSIST>, a, b, i, parity)
                     : cudaLaunchKernelEx(&cfg, fused_step_kernel<float, 4, BATCH, PERSIST, false>, a, b, i, parity);
        else
            e = down ? cudaLaunchKernelEx(&cfg, fused_step_kernel<float, 2, BATCH, PERSIST, !PERSIST>, a, b, i, parity)
                     : cudaLaunchKernelEx(&cfg, fused_step_kernel<float, 2, BATCH, PERSIST, false>, a, b, i, parity);
    } else {
        e = down ? cudaLaunchKernelEx(&cfg, fused_step_kernel<double, 2, BATCH, PERSIST, !PERSIST>, a, b, i, parity)
                 : cudaLaunchKernelEx(&cfg, fused_step_kernel<double, 2, BATCH, PERSIST, false>, a, b, i, parity);
    }
    if (e != cudaSuccess) return (int)e;
    return ok_or(cudaGetLastError());
}

template <typename T>
int launch_step(const StepArgs<T>& a, int i, int parity, bool pdl, void* stream) {
    BatchArgs<T> none = {};
    return launch<T, false, false>(a, none, a.grid, a.tile_m, a.chunk_n, a.vec, i, parity, pdl,
                                   stream);
}

template <typename T>
int launch_step_persist(const StepArgs<T>& a, int parity, void* stream) {
    BatchArgs<T> none = {};
    return launch<T, false, true>(a, none, a.grid, a.tile_m, a.chunk_n, a.vec, 0, parity, false,
                                  stream);
}

template <typename T>
int launch_step_batch(const BatchArgs<T>& b, int i, int parity, bool pdl, void* stream) {
    StepArgs<T> none = {};
    return launch<T, true, false>(none, b, b.grid, b.tile_m, b.chunk_n, b.vec, i, parity, pdl,
                                  stream);
}

#define BTE_STEP_INSTANTIATE(T)                                                    \
    template size_t step_smem_bytes<T>(int, int, int);                             \
    template int step_block_threads<T>(int, int);                                  \
    template int step_max_tile<T>(int);                                            \
    template int step_kernel_configure<T>(int, int, int, int*);                    \
    template int step_kernel_configure_batch<T>(int, int, int, int*);              \
    template int step_kernel_configure_persist<T>(int, int, int, int*);            \
    template int launch_step<T>(const StepArgs<T>&, int, int, bool, void*);        \
    template int launch_step_persist<T>(const StepArgs<T>&, int, void*);           \
    template int launch_step_batch<T>(const BatchArgs<T>&, int, int, bool, void*);
BTE_STEP_INSTANTIATE(float)
BTE_STEP_INSTANTIATE(double)

}  // namespace bte
