/*
 * bte_device.cuh -- device helpers shared by the library's kernels:
 * mbarrier / TMA bulk-copy wrappers (inline PTX, sm_90+ forms valid on
 * sm_103a), bounded waits, the per-cell Crank-Nicolson update and a
 * fixed-order block reduction.
 */
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace bte {
namespace dev {

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

/* The same test with a suspend-time hint: the thread may sleep in the
 * barrier unit for up to `ns` nanoseconds (it wakes when the phase
 * completes) instead of returning at once, so a waiting warp takes few
 * issue slots from the warps doing work. */
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

/* Default limit of a bounded wait: 2 s of %globaltimer. */
constexpr uint64_t kWaitLimitNs = 2000000000ull;

/* Bounded wait on an mbarrier phase: false once limit_ns of %globaltimer
 * have passed without the phase completing.  Retries sleep in the barrier
 * unit (up to 10 us each, woken by the phase; never past the limit). */
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer();
    for (;;) {
        const uint64_t el = global_timer() - t0;
        if (el > limit_ns) return false;
        const uint64_t left = limit_ns - el;
        if (mbar_try_wait_sleep(bar, parity, left < 10000u ? (uint32_t)left + 1u : 10000u)) return true;
    }
}

/* TMA bulk copy global -> shared, completion counted on an mbarrier.  Both
 * addresses 16-byte aligned, size a multiple of 16. */
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

/* 1/x for the Crank-Nicolson denominator D = nu^2 + theta'^2 >= 1: the
 * hardware approximate reciprocal in FP32 (PTX rcp.approx.ftz.f32, about one
 * ulp; D is never subnormal, zero or infinite), the correctly rounded
 * division in FP64. */
template <typename T>
__device__ __forceinline__ T recip(T x);
template <>
__device__ __forceinline__ float recip<float>(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <>
__device__ __forceinline__ double recip<double>(double x) {
    return 1.0 / x;
}

/* Arithmetic with exactly one rounding per operation and no contraction
 * left to the compiler (the _rn intrinsics are never fused or reordered).
 * Every kernel that applies the per-cell update -- streamed, persistent,
 * on-chip, start-up -- goes through these, so they all perform the same
 * sequence of roundings and agree bit for bit. */
template <typename T>
struct Rn;
template <>
struct Rn<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <>
struct Rn<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

/* Constants of the Crank-Nicolson operator T_h (Sec. 3): nu = 1 + h/2,
 * xi = 1 - h/2 and the products nu^2, nu h. */
template <typename T>
struct CnK {
    T h, nu, xi, nu2, nuh;
};
template <typename T>
__device__ __forceinline__ CnK<T> cn_constants(T h, T nu, T xi) {
    return CnK<T>{h, nu, xi, Rn<T>::mul(nu, nu), Rn<T>::mul(nu, h)};
}

/* Rotation factor (E + B phi_y) h/2 of one column at one time (the theta of
 * Eqs. a_t_plus_1, b_t_plus_1 is n times it). */
template <typename T>
__device__ __forceinline__ T rot_factor(T E, T B, T phi, T hh) {
    return Rn<T>::mul(Rn<T>::fma(B, phi, E), hh);
}

/* The paper's stencil terms from central differences D x_r(m) of the other
 * grid: B^t = c (D b_{n+1} - D b_{n-1}) acts on a, A^t = c (chi(n) D a_{n-1}
 * - D a_{n+1}) on b (chi(1) = 2: the n = 1 row reads a_0 twice, Sec. 3). */
template <typename T>
__device__ __forceinline__ T stencil_a(T c, T db_next, T db_prev) {
    return Rn<T>::mul(c, Rn<T>::sub(db_next, db_prev));
}
template <typename T>
__device__ __forceinline__ T stencil_b(T c, T chi, T da_prev, T da_next) {
    return Rn<T>::mul(c, Rn<T>::fma(chi, da_prev, -da_next));
}

/* Crank-Nicolson update of one cell (Sec. 3, Eqs. a_t_plus_1, b_t_plus_1,
 * with the sign of b' that solves nu a' + th1 b' = g, -th1 a' + nu b' = q),
 * written as increments so that FP32 keeps the O(h) relaxation balance:
 *   D  = nu^2 + th1^2
 *   da = [nu (Sa + h a0) - th1 Sb - a (nu h + th1 (th + th1)) - b (th nu + xi th1)] / D
 *   db = [th1 (Sa + h a0) + nu Sb + a (th nu + xi th1) - b (nu h + th1 (th + th1))] / D
 * which equals a' - a, b' - b for a' = (g nu - q th1)/D, b' = (g th1 + q nu)/D,
 * g = a xi - b th + Sa + h a0, q = b xi + a th + Sb.  Sa is the paper's B^t
 * stencil term (acts on a), Sb its A^t term (acts on b); h a0 = hr g with
 * hr = h times the row factor and g the column factor of the separable
 * equilibrium.  Each product, sum and fused multiply-add below is one
 * rounding, in this order. */
template <typename T>
struct CnCoef {
    T th1, inv, ca, cb;
};
/* The part of the update that depends on the cell's (n, m) and the drive
 * only, not on the state: 1/D and the two coefficients of a and b. */
template <typename T>
__device__ __forceinline__ CnCoef<T> cn_coef(T th, T th1, const CnK<T>& k) {
    using O = Rn<T>;
    CnCoef<T> c;
    c.th1 = th1;
    const T D = O::fma(th1, th1, k.nu2);
    c.inv = recip<T>(D);
    c.ca = O::fma(th1, O::add(th, th1), k.nuh);
    c.cb = O::fma(k.xi, th1, O::mul(th, k.nu));
    return c;
}
/* The rest: the new a, b from the old ones and the stencil terms. */
template <typename T>
__device__ __forceinline__ void cn_update(T a, T b, T Sa, T Sb, T hr, T g, const CnCoef<T>& c,
                                          const CnK<T>& k, T& an, T& bn) {
    using O = Rn<T>;
    const T src = O::fma(hr, g, Sa);
    T t = O::fma(k.nu, src, -O::mul(c.th1, Sb));
    t = O::fma(-a, c.ca, t);
    t = O::fma(-b, c.cb, t);
    T u = O::fma(c.th1, src, O::mul(k.nu, Sb));
    u = O::fma(a, c.cb, u);
    u = O::fma(-b, c.ca, u);
    an = O::add(a, O::mul(t, c.inv));
    bn = O::add(b, O::mul(u, c.inv));
}
template <typename T>
__device__ __forceinline__ void cn_cell(T a, T b, T Sa, T Sb, T hr, T g, T th, T th1,
                                        const CnK<T>& k, T& an, T& bn) {
    cn_update<T>(a, b, Sa, Sb, hr, g, cn_coef<T>(th, th1, k), k, an, bn);
}

/* The update of V consecutive columns of one row (V = 2 or 4): the stencil
 * terms from the other grid's differences in rows n+1 (next) and n-1 (prev),
 * the rotations n w0, n w1 (w = rot_factor at the half-step's start and end)
 * and cn_cell.  FP32 runs two columns per instruction with Blackwell's paired
 * FP32 operations (__ffma2_rn, __fadd2_rn, __fmul2_rn), which round each
 * component exactly as the scalar _rn form: the same bits as cn_cell on
 * each column, in half the issue slots.  FP64 runs cn_cell per column. */
__device__ __forceinline__ float2 pair(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

template <typename T, int V>
__device__ __forceinline__ void cn_row(const T (&a)[V], const T (&b)[V], const T (&db_next)[V],
                                       const T (&db_prev)[V], const T (&da_prev)[V],
                                       const T (&da_next)[V], T cc, T chi, T hr, const T (&g)[V],
                                       T nf, const T (&w0)[V], const T (&w1)[V], const CnK<T>& k,
                                       T (&an)[V], T (&bn)[V]) {
    if constexpr (sizeof(T) == 4 && V % 2 == 0) {
        const float2 cc2 = pair(cc, cc), chi2 = pair(chi, chi), hr2 = pair(hr, hr);
        const float2 nf2 = pair(nf, nf), nu2 = pair(k.nu2, k.nu2), nuh2 = pair(k.nuh, k.nuh);
        const float2 nu = pair(k.nu, k.nu), xi = pair(k.xi, k.xi);
#pragma unroll
        for (int e = 0; e < V; e += 2) {
            const float2 A = pair(a[e], a[e + 1]), Bv = pair(b[e], b[e + 1]);
            const float2 Sa = __fmul2_rn(cc2, __fadd2_rn(pair(db_next[e], db_next[e + 1]),
                                                         neg2(pair(db_prev[e], db_prev[e + 1]))));
            const float2 Sb = __fmul2_rn(cc2, __ffma2_rn(chi2, pair(da_prev[e], da_prev[e + 1]),
                                                         neg2(pair(da_next[e], da_next[e + 1]))));
            const float2 th = __fmul2_rn(nf2, pair(w0[e], w0[e + 1]));
            const float2 th1 = __fmul2_rn(nf2, pair(w1[e], w1[e + 1]));
            const float2 D = __ffma2_rn(th1, th1, nu2);
            const float2 inv = pair(recip<float>(D.x), recip<float>(D.y));
            const float2 src = __ffma2_rn(hr2, pair(g[e], g[e + 1]), Sa);
            const float2 ca = __ffma2_rn(th1, __fadd2_rn(th, th1), nuh2);
            const float2 cb = __ffma2_rn(xi, th1, __fmul2_rn(th, nu));
            float2 t = __ffma2_rn(nu, src, neg2(__fmul2_rn(th1, Sb)));
            t = __ffma2_rn(neg2(A), ca, t);
            t = __ffma2_rn(neg2(Bv), cb, t);
            float2 u = __ffma2_rn(th1, src, __fmul2_rn(nu, Sb));
            u = __ffma2_rn(A, cb, u);
            u = __ffma2_rn(neg2(Bv), ca, u);
            const float2 na = __fadd2_rn(A, __fmul2_rn(t, inv));
            const float2 nb = __fadd2_rn(Bv, __fmul2_rn(u, inv));
            an[e] = na.x;
            an[e + 1] = na.y;
            bn[e] = nb.x;
            bn[e + 1] = nb.y;
        }
    } else {
        using O = Rn<T>;
#pragma unroll
        for (int e = 0; e < V; ++e)
            cn_cell<T>(a[e], b[e], stencil_a<T>(cc, db_next[e], db_prev[e]),
                       stencil_b<T>(cc, chi, da_prev[e], da_next[e]), hr, g[e],
                       O::mul(nf, w0[e]), O::mul(nf, w1[e]), k, an[e], bn[e]);
    }
}


/* Split cluster barrier (all threads of every CTA of the cluster): the
 * arrive releases this thread's earlier writes (distributed shared memory
 * included), the wait acquires those of every thread that arrived. */
__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

/* Acquire load and release store of a counter at GPU scope (completion
 * counters that CTAs of one launch poll). */
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

/* Drive of one half-step: E and B at its start (E0, B0) and end (E1, B1),
 * and its stencil coefficient, read from a [3][stride] drive table (E, B,
 * coefficient; FP64 values rounded to T once on the host) at row kk. */
template <typename T>
struct Half {
    T E0, E1, B0, B1, cc;
};
template <typename T>
__device__ __forceinline__ Half<T> half_drive(const T* tab, int stride, int kk) {
    Half<T> d;
    d.E0 = tab[kk];
    d.E1 = tab[kk + 1];
    d.B0 = tab[stride + kk];
    d.B1 = tab[stride + kk + 1];
    d.cc = tab[2 * stride + kk];
    return d;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

/* Sums of FP32 values carried as unevaluated pairs hi + lo of FP32 numbers
 * (Knuth's error-free TwoSum, so the pair keeps about 48 bits): the per-step
 * row sums of FP32 states need FP64-grade accuracy, and FP32 operations run
 * at many times the rate of FP64 ones on this GPU. */
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return F2{s, e};
}
__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
    const F2 s = two_sum(x.hi, y.hi);
    return two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
/* x + v with the pair's error term kept */
__device__ __forceinline__ F2 f2_add1(F2 x, float v) {
    const F2 t = two_sum(x.hi, v);
    return F2{t.hi, __fadd_rn(x.lo, t.lo)};
}
__device__ __forceinline__ double warp_sum_f2(F2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = f2_add(v, F2{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)});
    return (double)v.hi + (double)v.lo;
}

/* Sum over the block in a fixed order (warp shuffles, then warp partials
 * in warp order); the result is valid in thread 0.  `red` holds >= 32
 * doubles; every thread of the block must call it. */
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
    return s;
}

}  // namespace dev
}  // namespace bte
