/*
 * bte_kernels.cu -- sm_103a kernels of the single-instance solver.
 *
 * The hot kernel is fused_step_kernel: one launch performs one full
 * leap-frog step of Sec. 3 (Eqs. leap_frog_1 and leap_frog_2):
 *     whole grid       z^{t+1}   = T(z^t;       S(z^{t+1/2}))
 *     fractional grid  z^{t+3/2} = T(z^{t+1/2}; S(z^{t+1}))
 * where T is the Crank-Nicolson operator of Eqs. a_t_plus_1 / b_t_plus_1 and
 * S the 4-point diagonal stencil of the paper's A^t, B^t terms.
 *
 * Work decomposition.  A CTA owns tile_m consecutive phi_y columns and
 * chunk_n consecutive harmonic rows.  It walks its rows upward with a
 * one-row lag: at row j it builds the new whole-grid row j (on its columns
 * plus one halo column per side) and then the new fractional row j-1, which
 * needs new whole rows j-2 and j (kept in a 3-row shared-memory ring).  The
 * old fractional and whole rows stream in through a ring of RS shared-memory
 * stages filled by TMA bulk copies (cp.async.bulk + mbarrier), RS-2 rows
 * ahead of use, so every old value is read from HBM/L2 once per CTA.  New
 * rows are written straight from registers with coalesced stores.  Chunks
 * recompute the two boundary whole rows they need (two extra rows of work
 * per chunk).
 *
 * Observables (Sec. 2, Eq. v_dr_generic and Eq. norm_in_phi) are folded in:
 * the CTAs that own rows 0 and 1 reduce sum_m a_{0,m} and sum_m b_{1,m} in
 * FP64 (warp shuffles), and the last of them to arrive sums the per-tile
 * partials in tile order, so the trace is bitwise reproducible.
 *
 * Every mbarrier wait is bounded (about 2 s of %globaltimer); on expiry the
 * kernel records an error word that the host reports as BTE_ETIMEOUT.
 */
#include <cuda_runtime.h>

#include <cstdint>

#include "bte_internal.h"

namespace bte {

namespace {

constexpr int kMaxThreads = 1024;

template <typename T>
struct Ring {
    static constexpr int RS = sizeof(T) == 4 ? 8 : 6;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            bar),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

/* Bounded wait: false after ~2 s without the phase completing. */
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer() - t0 > 2000000000ull) return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <typename T>
__device__ __forceinline__ T recip(T x);
template <>
__device__ __forceinline__ float recip<float>(float x) {
    return __frcp_rn(x);
}
template <>
__device__ __forceinline__ double recip<double>(double x) {
    return 1.0 / x;
}

/* Crank-Nicolson update of one cell (Eqs. a_t_plus_1, b_t_plus_1 with the
 * sign of b' that solves nu a' + th1 b' = g, -th1 a' + nu b' = q), written as
 * increments so that FP32 keeps the O(h) relaxation balance:
 *   D  = nu^2 + th1^2
 *   da = [nu (Sa + h a0) - th1 Sb - a (nu h + th1 (th + th1)) - b (th nu + xi th1)] / D
 *   db = [th1 (Sa + h a0) + nu Sb + a (th nu + xi th1) - b (nu h + th1 (th + th1))] / D
 * (algebraically identical to a' = (g nu - q th1)/D, b' = (g th1 + q nu)/D
 * with g = a xi - b th + Sa + h a0, q = b xi + a th + Sb). */
template <typename T>
__device__ __forceinline__ void cn_cell(T a, T b, T Sa, T Sb, T ha0, T th, T th1, T nu, T xi,
                                        T h, T& an, T& bn) {
    const T D = nu * nu + th1 * th1;
    const T inv = recip<T>(D);
    const T src = Sa + ha0;
    const T ca = nu * h + th1 * (th + th1);
    const T cb = th * nu + xi * th1;
    const T da = (nu * src - th1 * Sb - a * ca - b * cb) * inv;
    const T db = (th1 * src + nu * Sb + a * cb - b * ca) * inv;
    an = a + da;
    bn = b + db;
}

template <typename T>
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int q = 0; q < nw; ++q) s += red[q];
    }
    return s; /* valid in thread 0 */
}

/* ---------------------------------------------------------------------- */
/* fused leap-frog step                                                    */
/* ---------------------------------------------------------------------- */
template <typename T>
__global__ void __launch_bounds__(kMaxThreads) fused_step_kernel(StepArgs<T> A, int i) {
    constexpr int H = 16 / (int)sizeof(T); /* ghost / halo columns (16 bytes) */
    constexpr int RS = Ring<T>::RS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int Wt = A.tile_m;
    const int LW = Wt + 2 * H; /* columns of a streamed row segment */
    const int NW = Wt + 2;     /* columns of a new whole-grid row   */
    T* sF = reinterpret_cast<T*>(smem_raw);          /* [RS][2][LW] old fractional rows */
    T* sW = sF + (size_t)RS * 2 * LW;                 /* [RS][2][LW] old whole rows      */
    T* sN = sW + (size_t)RS * 2 * LW;                 /* [3][2][LW]  new whole rows      */
    T* zrow = sN + (size_t)3 * 2 * LW;                /* [LW] zeros                      */
    uint64_t* bar = reinterpret_cast<uint64_t*>(zrow + LW);
    double* red = reinterpret_cast<double*>(bar + RS);

    const int tid = threadIdx.x;
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int N = A.N, M = A.M, pitch = A.pitch;
    const int p0 = H + tx * Wt; /* physical column of the first owned column */
    const int n0 = ty * A.chunk_n;
    const int n1 = min(n0 + A.chunk_n, N + 1);
    const long long k = *A.base + i;
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

    const int S_tot = n1 - n0 + 4; /* stages: rows n0-2 .. n1+1 */

    for (int q = tid; q < LW; q += blockDim.x) zrow[q] = (T)0;
    if (tid == 0) {
        for (int s = 0; s < RS; ++s) mbar_init(smem_u32(&bar[s]), 1);
        fence_proxy_async_smem();
    }
    __syncthreads();

    auto issue = [&](int s) {
        const int slot = s % RS;
        const int row = n0 - 2 + s;
        const uint32_t mb = smem_u32(&bar[slot]);
        if (row < 0 || row > N) {
            mbar_arrive(mb);
            return;
        }
        const bool wneed = row >= n0 - 1 && row <= n1;
        const uint32_t rb = (uint32_t)(LW * sizeof(T));
        mbar_arrive_tx(mb, rb * (wneed ? 4u : 2u));
        const size_t off = (size_t)row * pitch + (p0 - H);
        bulk_g2s(smem_u32(sF + (size_t)slot * 2 * LW), gFa + off, rb, mb);
        bulk_g2s(smem_u32(sF + (size_t)slot * 2 * LW + LW), gFb + off, rb, mb);
        if (wneed) {
            bulk_g2s(smem_u32(sW + (size_t)slot * 2 * LW), gWa + off, rb, mb);
            bulk_g2s(smem_u32(sW + (size_t)slot * 2 * LW + LW), gWb + off, rb, mb);
        }
    };
    if (tid == 0) {
        const int pre = S_tot < RS ? S_tot : RS;
        for (int s = 0; s < pre; ++s) issue(s);
    }

    /* per-column constants of the (at most two) whole-grid columns and the
     * one fractional-grid column this thread updates */
    T wg[2], wbs[2], wbe[2];
    bool wok[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int q = tid + u * blockDim.x;
        const int c = p0 - 1 + q;
        const int m = c - H;
        wok[u] = q < NW && m >= 0 && m <= M;
        wg[u] = wok[u] ? A.col_g[c] : (T)0;
        const T bp = wok[u] ? A.col_bphi[c] : (T)0;
        wbs[u] = (Ews + bp) * hh;
        wbe[u] = (Ewe + bp) * hh;
    }
    const int cf = p0 + tid;
    const bool fok = tid < Wt && (cf - H) <= M;
    const T fg = fok ? A.col_g[cf] : (T)0;
    const T fbp = fok ? A.col_bphi[cf] : (T)0;
    const T fbs = (Efs + fbp) * hh, fbe = (Efe + fbp) * hh;

    int waited = -1;
    bool timed_out = false;
    double part_n = 0.0, part_v = 0.0;

    for (int j = n0 - 1; j <= n1; ++j) {
        const int need = j - n0 + 3;
        while (waited < need && waited + 1 < S_tot) {
            ++waited;
            if (!mbar_wait(smem_u32(&bar[waited % RS]), (uint32_t)((waited / RS) & 1)))
                timed_out = true;
        }
        /* ---- new whole-grid row j ---- */
        T* nrow_a = sN + (size_t)((j + 3) % 3) * 2 * LW;
        T* nrow_b = nrow_a + LW;
        if (j >= 0 && j <= N) {
            const int sd = (j - 1 - (n0 - 2)) % RS, su = (j + 1 - (n0 - 2)) % RS;
            const int sj = (j - (n0 - 2)) % RS;
            const T* fa_dn = (j - 1 >= 0) ? sF + (size_t)sd * 2 * LW : zrow;
            const T* fb_dn = (j - 1 >= 1) ? sF + (size_t)sd * 2 * LW + LW : zrow;
            const T* fa_up = (j + 1 <= N) ? sF + (size_t)su * 2 * LW : zrow;
            const T* fb_up = (j + 1 <= N) ? sF + (size_t)su * 2 * LW + LW : zrow;
            const T* wa = sW + (size_t)sj * 2 * LW;
            const T* wb = wa + LW;
            const T nf = (T)j;
            const T chi = (j == 1) ? (T)2 : (T)1;
            const T ha0 = h * A.row_a0[j];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int q = tid + u * blockDim.x;
                if (q < NW) {
                    T an = (T)0, bn = (T)0;
                    if (wok[u]) {
                        const int lc = q - 1 + H; /* local column in the streamed rows */
                        const T Sa = cc * ((fb_up[lc + 1] - fb_up[lc - 1]) -
                                           (fb_dn[lc + 1] - fb_dn[lc - 1]));
                        const T Sb = cc * (chi * (fa_dn[lc + 1] - fa_dn[lc - 1]) -
                                           (fa_up[lc + 1] - fa_up[lc - 1]));
                        cn_cell<T>(wa[lc], wb[lc], Sa, Sb, ha0 * wg[u], nf * wbs[u],
                                   nf * wbe[u], nu, xi, h, an, bn);
                        if (j == 0) bn = (T)0;
                        const int c = p0 - 1 + q;
                        if (j >= n0 && j < n1 && q >= 1 && q <= Wt) {
                            const size_t g = (size_t)j * pitch + c;
                            oWa[g] = an;
                            oWb[g] = bn;
                        }
                        if (n0 == 0 && q >= 1 && q <= Wt) {
                            if (j == 0) part_n += (double)an;
                            if (j == 1) part_v += (double)bn;
                        }
                    }
                    nrow_a[q] = an;
                    nrow_b[q] = bn;
                }
            }
        }
        __syncthreads();
        /* ---- new fractional row j-1 ---- */
        const int r = j - 1;
        if (r >= n0 && r < n1) {
            const int sr = (r - (n0 - 2)) % RS;
            const T* fa = sF + (size_t)sr * 2 * LW;
            const T* fb = fa + LW;
            const T* na_dn = (r - 1 >= 0) ? sN + (size_t)((r - 1 + 3) % 3) * 2 * LW : zrow;
            const T* nb_dn = (r - 1 >= 1) ? sN + (size_t)((r - 1 + 3) % 3) * 2 * LW + LW : zrow;
            const T* na_up = (r + 1 <= N) ? sN + (size_t)((r + 1) % 3) * 2 * LW : zrow;
            const T* nb_up = (r + 1 <= N) ? sN + (size_t)((r + 1) % 3) * 2 * LW + LW : zrow;
            if (fok) {
                const int ln = tid + 1;  /* column in the new whole rows   */
                const int lc = tid + H;  /* column in the streamed rows    */
                const T nf = (T)r;
                const T chi = (r == 1) ? (T)2 : (T)1;
                const T Sa = cc * ((nb_up[ln + 1] - nb_up[ln - 1]) - (nb_dn[ln + 1] - nb_dn[ln - 1]));
                const T Sb = cc * (chi * (na_dn[ln + 1] - na_dn[ln - 1]) -
                                   (na_up[ln + 1] - na_up[ln - 1]));
                T an, bn;
                cn_cell<T>(fa[lc], fb[lc], Sa, Sb, h * A.row_a0[r] * fg, nf * fbs, nf * fbe, nu, xi,
                           h, an, bn);
                if (r == 0) bn = (T)0;
                const size_t g = (size_t)r * pitch + cf;
                oFa[g] = an;
                oFb[g] = bn;
            }
        }
        /* ---- observables of rows 0 and 1 ---- */
        if (n0 == 0 && j == 1) {
            const double sn = block_sum<T>(part_n, red);
            const double sv = block_sum<T>(part_v, red);
            if (tid == 0) {
                A.part[tx] = sn;
                A.part[A.ntx + tx] = sv;
                __threadfence();
                const unsigned t = atomicAdd(A.ticket, 1u);
                if (t == (unsigned)(A.ntx - 1)) {
                    __threadfence();
                    double s_n = 0, s_v = 0;
                    const volatile double* pv = A.part;
                    for (int q = 0; q < A.ntx; ++q) {
                        s_n += pv[q];
                        s_v += pv[A.ntx + q];
                    }
                    A.trace_n[k + 1] = A.nscale * s_n;
                    A.trace_v[k + 1] = A.vscale * s_v;
                    *A.ticket = 0u;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            const int s = j - n0 + 1 + RS;
            if (s < S_tot) {
                fence_proxy_async_smem();
                issue(s);
            }
        }
    }
    if (timed_out) atomicExch(A.err, kErrTimeout);
}

/* ---------------------------------------------------------------------- */
/* initial state, start-up half step, plain observables                  */
/* ---------------------------------------------------------------------- */
template <typename T>
__global__ void init_kernel(T* a_w, T* b_w, const T* row_a0, const T* col_g, int N, int M,
                            int pitch) {
    constexpr int G = 16 / (int)sizeof(T);
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (m > M || n > N) return;
    const size_t g = (size_t)n * pitch + G + m;
    a_w[g] = row_a0[n] * col_g[G + m];
    b_w[g] = (T)0;
}

template <typename T>
__device__ __forceinline__ T ld_or0(const T* x, int n, int c, int N, int pitch) {
    return (n < 0 || n > N) ? (T)0 : x[(size_t)n * pitch + c];
}

template <typename T>
__global__ void apply_kernel(ApplyArgs<T> A) {
    constexpr int G = 16 / (int)sizeof(T);
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (m > A.M || n > A.N) return;
    const int c = G + m;
    const T chi = (n == 1) ? (T)2 : (T)1;
    const T bp = A.col_bphi[c];
    const T th = (T)n * (((T)A.E_start + bp) * A.hh);
    const T th1 = (T)n * (((T)A.E_end + bp) * A.hh);
    const int N = A.N, P = A.pitch;
    const T bu = ld_or0(A.bs, n + 1, c + 1, N, P) - ld_or0(A.bs, n + 1, c - 1, N, P);
    const T bd = (n - 1 >= 1) ? ld_or0(A.bs, n - 1, c + 1, N, P) - ld_or0(A.bs, n - 1, c - 1, N, P)
                              : (T)0;
    const T ad = ld_or0(A.as, n - 1, c + 1, N, P) - ld_or0(A.as, n - 1, c - 1, N, P);
    const T au = ld_or0(A.as, n + 1, c + 1, N, P) - ld_or0(A.as, n + 1, c - 1, N, P);
    const T Sa = A.c * (bu - bd);
    const T Sb = A.c * (chi * ad - au);
    const size_t g = (size_t)n * P + c;
    T an, bn;
    cn_cell<T>(A.a[g], A.b[g], Sa, Sb, A.h * A.row_a0[n] * A.col_g[c], th, th1, A.nu, A.xi, A.h,
               an, bn);
    if (n == 0) bn = (T)0;
    A.an[g] = an;
    A.bn[g] = bn;
}

template <typename T>
__global__ void observe_kernel(const T* a_w, const T* b_w, int M, int pitch, double vscale,
                               double nscale, double* trace_v, double* trace_n, long long slot) {
    constexpr int G = 16 / (int)sizeof(T);
    __shared__ double red[32];
    double sn = 0, sv = 0;
    for (int m = threadIdx.x; m <= M; m += blockDim.x) {
        sn += (double)a_w[G + m];
        sv += (double)b_w[(size_t)pitch + G + m];
    }
    const double tn = block_sum<T>(sn, red);
    const double tv = block_sum<T>(sv, red);
    if (threadIdx.x == 0) {
        trace_n[slot] = nscale * tn;
        trace_v[slot] = vscale * tv;
    }
}

__global__ void advance_base_kernel(long long* base, long long by) { *base += by; }

/* Window averages (Eq. absorption_def) and norm error from the trace, in
 * FP64 with a fixed-order reduction. */
__global__ void finalize_kernel(FinalArgs A) {
    __shared__ double s_cos[1024], s_sum[1024], s_err[1024];
    __shared__ int s_bad[1024];
    const int t = threadIdx.x;
    double sc = 0, ss = 0, er = 0;
    int bad = 0;
    const long long k0 = A.K - A.Kw + 1;
    for (long long q = t; q <= A.k; q += blockDim.x) {
        const double v = A.trace_v[q], nr = A.trace_n[q];
        if (!isfinite(v) || !isfinite(nr)) bad = 1;
        er = fmax(er, fabs(nr - 1.0));
        if (q >= k0 && q <= A.K) {
            double ang;
            if (A.P > 0)
                ang = 6.283185307179586476925286766559 * (double)(q % A.P) / (double)A.P;
            else
                ang = A.omega * (double)q * A.dt_eff;
            sc += v * cos(ang);
            ss += v;
        }
    }
    s_cos[t] = sc;
    s_sum[t] = ss;
    s_err[t] = er;
    s_bad[t] = bad;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            s_cos[t] += s_cos[t + o];
            s_sum[t] += s_sum[t + o];
            s_err[t] = fmax(s_err[t], s_err[t + o]);
            s_bad[t] |= s_bad[t + o];
        }
        __syncthreads();
    }
    if (t == 0) {
        const double inv = 1.0 / (double)A.Kw;
        A.out[0] = 2.0 * A.inv_r1 * s_cos[0] * inv;
        A.out[1] = s_sum[0] * inv;
        A.out[2] = s_err[0];
        A.out[3] = (double)s_bad[0];
    }
}

}  // namespace

/* ---------------------------------------------------------------------- */
/* launchers                                                               */
/* ---------------------------------------------------------------------- */
static int ok_or(cudaError_t e) { return e == cudaSuccess ? 0 : (int)e; }

template <typename T>
size_t step_smem_bytes(int tile_m) {
    constexpr int H = 16 / (int)sizeof(T);
    const size_t LW = (size_t)tile_m + 2 * H;
    const int RS = Ring<T>::RS;
    return (2 * RS * 2 + 3 * 2 + 1) * LW * sizeof(T) + RS * sizeof(uint64_t) + 32 * sizeof(double);
}

template <typename T>
int step_kernel_configure(int tile_m) {
    const size_t bytes = step_smem_bytes<T>(tile_m);
    return ok_or(cudaFuncSetAttribute(fused_step_kernel<T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

template <typename T>
int launch_step(const StepArgs<T>& a, int i, void* stream) {
    dim3 grid(a.ntx, a.nty);
    fused_step_kernel<T><<<grid, a.tile_m, step_smem_bytes<T>(a.tile_m), (cudaStream_t)stream>>>(
        a, i);
    return ok_or(cudaGetLastError());
}

template <typename T>
int launch_init(T* a_w, T* b_w, const T* row_a0, const T* col_g, int N, int M, int pitch,
                void* stream) {
    dim3 grid((M + 1 + 255) / 256, N + 1);
    init_kernel<T><<<grid, 256, 0, (cudaStream_t)stream>>>(a_w, b_w, row_a0, col_g, N, M, pitch);
    return ok_or(cudaGetLastError());
}

template <typename T>
int launch_apply(const ApplyArgs<T>& a, void* stream) {
    dim3 grid((a.M + 1 + 255) / 256, a.N + 1);
    apply_kernel<T><<<grid, 256, 0, (cudaStream_t)stream>>>(a);
    return ok_or(cudaGetLastError());
}

template <typename T>
int launch_observe(const T* a_w, const T* b_w, int M, int pitch, double vscale, double nscale,
                   double* trace_v, double* trace_n, long long slot, void* stream) {
    observe_kernel<T><<<1, 512, 0, (cudaStream_t)stream>>>(a_w, b_w, M, pitch, vscale, nscale,
                                                           trace_v, trace_n, slot);
    return ok_or(cudaGetLastError());
}

int launch_advance_base(long long* base, long long by, void* stream) {
    advance_base_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(base, by);
    return ok_or(cudaGetLastError());
}

int launch_finalize(const FinalArgs& a, void* stream) {
    finalize_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(a);
    return ok_or(cudaGetLastError());
}

#define BTE_INSTANTIATE(T)                                                                     \
    template size_t step_smem_bytes<T>(int);                                                   \
    template int step_kernel_configure<T>(int);                                                \
    template int launch_step<T>(const StepArgs<T>&, int, void*);                               \
    template int launch_init<T>(T*, T*, const T*, const T*, int, int, int, void*);             \
    template int launch_apply<T>(const ApplyArgs<T>&, void*);                                  \
    template int launch_observe<T>(const T*, const T*, int, int, double, double, double*,      \
                                   double*, long long, void*);
BTE_INSTANTIATE(float)
BTE_INSTANTIATE(double)

}  // namespace bte
