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

/* Bounded wait on an mbarrier phase: false after ~2 s of %globaltimer. */
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer() - t0 > 2000000000ull) return false;
    }
    return true;
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

/* a * b + c with one rounding. */
template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) {
    return fmaf(a, b, c);
}
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) {
    return fma(a, b, c);
}

/* Crank-Nicolson update of one cell (Sec. 3, Eqs. a_t_plus_1, b_t_plus_1,
 * with the sign of b' that solves nu a' + th1 b' = g, -th1 a' + nu b' = q),
 * written as increments so that FP32 keeps the O(h) relaxation balance:
 *   D  = nu^2 + th1^2
 *   da = [nu (Sa + h a0) - th1 Sb - a (nu h + th1 (th + th1)) - b (th nu + xi th1)] / D
 *   db = [th1 (Sa + h a0) + nu Sb + a (th nu + xi th1) - b (nu h + th1 (th + th1))] / D
 * which equals a' - a, b' - b for a' = (g nu - q th1)/D, b' = (g th1 + q nu)/D,
 * g = a xi - b th + Sa + h a0, q = b xi + a th + Sb.  Sa is the paper's B^t
 * stencil term (acts on a), Sb its A^t term (acts on b). */
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
