/*
 * bte_sur_kernels.cu -- CUDA kernels of the MLP surrogate (sm_103a).
 *
 * The two 256 x 256 hidden layers and their backward products run on the
 * fifth-generation BF16 tensor cores (tcgen05.mma, FP32 accumulators in
 * tensor memory) in one GEMM kernel whose epilogue fuses the bias, the SiLU
 * activation and its derivative.  The thin layers (5 inputs, 2 outputs) are
 * FP32 FMA kernels; batch reductions are two-pass and deterministic; Adam
 * keeps FP32 master weights and refreshes the BF16 operand copies in the
 * same pass.
 */
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bte_device.cuh"
#include "bte_sur_internal.h"
#include "bte_tc.cuh"

namespace bte {
namespace sur {
namespace {

/* tcgen05 GEMM tile: 128 x 128 outputs per CTA (one MMA of M = N = 128
 * per 16 of K), K in stages of 64, two stages in shared memory. */
constexpr int GM = 128, GN = 128, GK = 64;
constexpr int kGThreads = 256; /* 8 warps: two per tensor-memory lane quadrant */
constexpr uint32_t kGTileBytes = (uint32_t)GM * GK * 2; /* 16 KB per operand tile */
constexpr uint32_t kGCore = 128;                        /* one 8 x 8 core matrix */
constexpr uint32_t kGGroup = (GK / 8) * kGCore;         /* 1024: next 8-row group */
constexpr size_t kGSmem = 4 * (size_t)kGTileBytes + 64 + 1024; /* 2 stages x (A, B), barriers, align */

/* sigmoid(z) = 1 / (1 + exp(-z)) with the fast exponential and reciprocal
 * (relative error ~1e-7, so the bfloat16 rounding that follows matches an
 * exact evaluation; exp(-z) = inf gives 0) */
__device__ __forceinline__ float sigmoid_f(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_f(float z) { return z * sigmoid_f(z); }
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = sigmoid_f(z);
    return s * (1.0f + z * (1.0f - s));
}

/* byte offset of element (r, k) of a [128][64] K-major stage tile in the
 * tensor cores' canonical layout without swizzle (8 x 8 core matrices of
 * 128 contiguous bytes, K-adjacent core matrices 128 bytes apart, 8-row
 * groups 1024 bytes apart) */
__device__ __forceinline__ uint32_t gcanon(int r, int k) {
    return (uint32_t)(((r >> 3) * (GK / 8) + (k >> 3)) * kGCore + (r & 7) * 16 + (k & 7) * 2);
}

/* One 128-row x 64-k operand tile into shared memory (canonical layout).
 * K-major source ([row][k], leading dimension ld): 1024 chunks of 8 k, four
 * per thread; a quarter-warp writes one core matrix (8 rows of one chunk
 * column, 128 contiguous bytes).  MN-major source ([k][row]): 128 blocks
 * of 8 k x 8 rows, one per thread of `first` .. `first + 127`, read as
 * eight 16-byte rows and transposed in registers (byte permutes) into the
 * eight 16-byte rows of one core matrix. */
template <bool MN>
__device__ __forceinline__ void load_stage(unsigned char* s, const __nv_bfloat16* g, long long ld,
                                           int row0, int k0, int first) {
    const int t = threadIdx.x;
    if constexpr (!MN) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = t + q * kGThreads;
            const int r = (c & 7) + 8 * (c >> 6), kc = (c >> 3) & 7;
            const uint4 v =
                __ldg(reinterpret_cast<const uint4*>(g + (long long)(row0 + r) * ld + k0 + kc * 8));
            *reinterpret_cast<uint4*>(s + gcanon(r, kc * 8)) = v;
        }
    } else {
        const int b = t - first;
        if (b < 0 || b >= 128) return;
        const int rb = b & 15, kb = b >> 4; /* 16 row blocks x 8 k blocks */
        uint32_t w[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(
                g + (long long)(k0 + kb * 8 + i) * ld + row0 + rb * 8));
            w[i][0] = v.x;
            w[i][1] = v.y;
            w[i][2] = v.z;
            w[i][3] = v.w;
        }
        unsigned char* dst = s + (uint32_t)((rb * (GK / 8) + kb) * kGCore);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            /* row j of the core matrix: element j of input rows 0..7 */
            const uint32_t sel = (j & 1) ? 0x7632u : 0x5410u;
            uint4 o;
            o.x = __byte_perm(w[0][j >> 1], w[1][j >> 1], sel);
            o.y = __byte_perm(w[2][j >> 1], w[3][j >> 1], sel);
            o.z = __byte_perm(w[4][j >> 1], w[5][j >> 1], sel);
            o.w = __byte_perm(w[6][j >> 1], w[7][j >> 1], sel);
            *reinterpret_cast<uint4*>(dst + j * 16) = o;
        }
    }
}

/* C = A B^T on the tensor cores (see GemmArgs).  One CTA per 128 x 128
 * output tile of one member (blockIdx.z).  K advances in stages of 64: the
 * CTA's threads fill stage s (global loads, transposed where the operand
 * is stored MN-major) while the tensor cores still work on the other
 * stage; one thread issues the four M = N = 128, K = 16 MMAs of a stage
 * into 128 columns of tensor memory and commits them to the stage's
 * mbarrier, which tells the threads when they may refill it.  The
 * epilogue reads the accumulators back with tcgen05.ld (warp w: lanes
 * 32 (w mod 4) .., columns 64 (w / 4) ..).  Every wait is bounded; a wait
 * that gives up sets the error word, and the CTA still frees its tensor
 * memory before it exits. */
template <bool AMN, bool BMN, int EPI>
__global__ void __launch_bounds__(kGThreads) gemm_tc_kernel(GemmArgs a) {
    extern __shared__ unsigned char gsm_raw[];
    unsigned char* gsm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~(uintptr_t)1023);
    /* stage s: A tile at s * 16 KB, B tile at (2 + s) * 16 KB; barrier s at 64 KB + 8 s */
    uint64_t* bars = reinterpret_cast<uint64_t*>(gsm + 4 * kGTileBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gsm + 4 * kGTileBytes + 32);
    const uint32_t bar0 = dev::smem_u32(bars);

    const int mem = blockIdx.z;
    const __nv_bfloat16* A = a.A + mem * a.sA;
    const __nv_bfloat16* B = a.B + mem * a.sB;
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    bool ok = true;

    if (tid == 0) {
        dev::mbar_init(bar0, 1);
        dev::mbar_init(bar0 + 8, 1);
        dev::fence_proxy_async_smem();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         dev::smem_u32(tmem_slot)),
                     "r"(GN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = tc::instr_desc(GM, GN);

    const int nk = a.K / GK;
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        unsigned char* sA = gsm + st * kGTileBytes;
        unsigned char* sB = gsm + (2 + st) * kGTileBytes;
        const uint32_t bar = bar0 + 8 * st;
        /* the MMAs that read this stage two rounds ago are complete */
        if (kt >= 2 && !dev::mbar_wait(bar, (uint32_t)(((kt - 2) >> 1) & 1))) ok = false;
        if (__syncthreads_or(!ok)) break;
        load_stage<AMN>(sA, A, a.lda, m0, kt * GK, 0);
        load_stage<BMN>(sB, B, a.ldb, n0, kt * GK, AMN ? 128 : 0);
        /* generic-proxy writes -> visible to the tensor cores */
        dev::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after();
            const uint32_t aA = dev::smem_u32(sA), aB = dev::smem_u32(sB);
#pragma unroll
            for (int ks = 0; ks < GK / 16; ++ks) {
                const uint64_t ad = tc::smem_desc(aA + ks * 2 * kGCore, kGCore, kGGroup);
                const uint64_t bd = tc::smem_desc(aB + ks * 2 * kGCore, kGCore, kGGroup);
                tc::tc_mma(tmem, ad, bd, idesc, (kt > 0 || ks > 0) ? 1u : 0u);
            }
            tc::tc_commit(bar);
        }
    }
    /* the last commit covers every MMA issued before it */
    if (ok && nk > 0 && !dev::mbar_wait(bar0 + 8 * ((nk - 1) & 1), (uint32_t)(((nk - 1) >> 1) & 1)))
        ok = false;
    if (ok && nk > 1 && !dev::mbar_wait(bar0 + 8 * (nk & 1), (uint32_t)(((nk - 2) >> 1) & 1)))
        ok = false;
    tc::tc_fence_after();

    if (ok) {
        const int sub = warp & 3, half = warp >> 2;
        const int row = m0 + sub * 32 + lane;
#pragma unroll 1
        for (int cb = 0; cb < GN / 2; cb += 32) {
            const int cl = half * (GN / 2) + cb; /* column within the tile */
            float v[32];
            tc::tc_ld32(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)cl, v);
            const int col = n0 + cl;
            if (EPI == EPI_FWD) {
                const float* bias = a.bias + mem * a.sBias + col;
                const long long o = mem * a.sZ + (long long)row * a.ldz + col;
#pragma unroll
                for (int c8 = 0; c8 < 32; c8 += 8) {
                    float z[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) z[e] = v[c8 + e] + bias[c8 + e];
                    if (a.Z) {
                        *reinterpret_cast<float4*>(a.Z + o + c8) = make_float4(z[0], z[1], z[2], z[3]);
                        *reinterpret_cast<float4*>(a.Z + o + c8 + 4) = make_float4(z[4], z[5], z[6], z[7]);
                    }
                    __nv_bfloat162 pk[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        pk[e] = __floats2bfloat162_rn(silu_f(z[2 * e]), silu_f(z[2 * e + 1]));
                    *reinterpret_cast<uint4*>(a.Hout + o + c8) = *reinterpret_cast<const uint4*>(pk);
                }
            } else if (EPI == EPI_BWD) {
                const long long o = mem * a.sZ + (long long)row * a.ldz + col;
#pragma unroll
                for (int c8 = 0; c8 < 32; c8 += 8) {
                    const float4 z0 = *reinterpret_cast<const float4*>(a.Zin + o + c8);
                    const float4 z1 = *reinterpret_cast<const float4*>(a.Zin + o + c8 + 4);
                    const float z[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
                    __nv_bfloat162 pk[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        pk[e] = __floats2bfloat162_rn(v[c8 + 2 * e] * silu_grad_f(z[2 * e]),
                                                      v[c8 + 2 * e + 1] * silu_grad_f(z[2 * e + 1]));
                    *reinterpret_cast<uint4*>(a.Dout + o + c8) = *reinterpret_cast<const uint4*>(pk);
                }
            } else {
                const long long o = mem * a.sC + (long long)row * a.ldc + col;
#pragma unroll
                for (int c4 = 0; c4 < 32; c4 += 4)
                    *reinterpret_cast<float4*>(a.C + o + c4) =
                        make_float4(v[c4], v[c4 + 1], v[c4 + 2], v[c4 + 3]);
            }
        }
    }
    if (!ok && tid == 0 && a.err) atomicExch(a.err, 1);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GN)
                     : "memory");
}

__device__ __forceinline__ void load_xh(const float* x, const int* idx, long long row0, int r,
                                        int nvalid, const Scale& sc, float (&xh)[kIn]) {
    if (r < nvalid) {
        const long long s = idx ? (long long)idx[r] : row0 + r;
#pragma unroll
        for (int i = 0; i < kIn; ++i) xh[i] = 2.0f * (x[s * kIn + i] - sc.x_lo[i]) * sc.x_inv[i] - 1.0f;
    } else {
#pragma unroll
        for (int i = 0; i < kIn; ++i) xh[i] = 0.0f;
    }
}

__global__ void l1_kernel(L1Args a) {
    const int mem = blockIdx.y;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)a.Bp * a.H) return;
    const int r = (int)(e / a.H), o = (int)(e - (long long)r * a.H);
    const int* idx = a.idx ? a.idx + (long long)mem * a.Bp : nullptr;
    float xh[kIn];
    load_xh(a.x, idx, a.row0, r, a.nvalid, a.sc, xh);
    const float* P = a.params + mem * a.pstride;
    float z = P[a.ob1 + o];
#pragma unroll
    for (int i = 0; i < kIn; ++i) z = fmaf(P[a.oW1 + (long long)o * kIn + i], xh[i], z);
    const long long out = ((long long)mem * a.Bp + r) * a.H + o;
    if (a.Z1) a.Z1[out] = z;
    a.H1[out] = __float2bfloat16_rn(silu_f(z));
}

/* one warp per sample; lane l covers hidden units 8l .. 8l+7 (H = 256) */
__global__ void head_kernel(HeadArgs a) {
    const int mem = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + warp;
    if (r >= a.Bp) return;
    const float* P = a.params + mem * a.pstride;
    const long long base = ((long long)mem * a.Bp + r) * a.H;
    float y0 = 0.0f, y1 = 0.0f;
    float hv[8];
    for (int c0 = lane * 8; c0 < a.H; c0 += 256) {
        const uint4 raw = *reinterpret_cast<const uint4*>(a.H3 + base + c0);
        const __nv_bfloat162* hp = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(hp[i]);
            hv[2 * i] = f.x;
            hv[2 * i + 1] = f.y;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            y0 = fmaf(P[a.oW4 + c0 + i], hv[i], y0);
            y1 = fmaf(P[a.oW4 + a.H + c0 + i], hv[i], y1);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        y0 += __shfl_xor_sync(0xffffffffu, y0, o);
        y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    }
    y0 += P[a.ob4];
    y1 += P[a.ob4 + 1];
    const long long yo = ((long long)mem * a.Bp + r) * kOut;
    if (lane == 0 && a.Yh) {
        a.Yh[yo] = y0;
        a.Yh[yo + 1] = y1;
    }
    if (!a.y) return;
    /* training: loss gradient and the output layer's backward product */
    float d0 = 0.0f, d1 = 0.0f;
    if (r < a.nvalid) {
        const int* idx = a.idx ? a.idx + (long long)mem * a.Bp : nullptr;
        const long long s = idx ? (long long)idx[r] : a.row0 + r;
        const float t0 = (a.y[s * kOut] - a.sc.y_mean[0]) / a.sc.y_std[0];
        const float t1 = (a.y[s * kOut + 1] - a.sc.y_mean[1]) / a.sc.y_std[1];
        d0 = (y0 - t0) * a.inv_n;
        d1 = (y1 - t1) * a.inv_n;
        if (lane == 0) {
            const double l = 0.5 * ((double)(y0 - t0) * (y0 - t0) + (double)(y1 - t1) * (y1 - t1));
            atomicAdd(a.loss + mem, l * a.inv_n);
        }
    }
    if (lane == 0) {
        a.DY[yo] = d0;
        a.DY[yo + 1] = d1;
    }
    for (int c0 = lane * 8; c0 < a.H; c0 += 256) {
        __nv_bfloat162 outv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float v[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int c = c0 + 2 * i + u;
                const float dh = d0 * P[a.oW4 + c] + d1 * P[a.oW4 + a.H + c];
                v[u] = dh * silu_grad_f(a.Z3[base + c]);
            }
            outv[i] = __floats2bfloat162_rn(v[0], v[1]);
        }
        *reinterpret_cast<uint4*>(a.DZ3 + base + c0) = *reinterpret_cast<const uint4*>(outv);
    }
}

/* values per 128-sample block: b1, W1 (5 per unit), b2, b3, W4 (2 per unit), b4 */
__host__ __device__ inline int red_count(int H) { return H * (1 + kIn + 1 + 1 + kOut) + kOut; }

__global__ void reduce_partial_kernel(RedArgs a) {
    const int mem = blockIdx.y, chunk = blockIdx.x;
    const int r0 = chunk * 128;
    __shared__ float sxh[128][kIn];
    __shared__ float sdy[128][kOut];
    const int* idx = a.idx ? a.idx + (long long)mem * a.Bp : nullptr;
    for (int r = threadIdx.x; r < 128; r += blockDim.x) {
        float xh[kIn];
        load_xh(a.x, idx, a.row0, r0 + r, a.nvalid, a.sc, xh);
#pragma unroll
        for (int i = 0; i < kIn; ++i) sxh[r][i] = xh[i];
        const long long yo = ((long long)mem * a.Bp + r0 + r) * kOut;
        sdy[r][0] = a.DY[yo];
        sdy[r][1] = a.DY[yo + 1];
    }
    __syncthreads();
    const int nred = red_count(a.H);
    float* out = a.partial + ((long long)mem * (a.Bp / 128) + chunk) * nred;
    for (int o = threadIdx.x; o < a.H; o += blockDim.x) {
        float gb1 = 0, gw1[kIn] = {0, 0, 0, 0, 0}, gb2 = 0, gb3 = 0, gw4[kOut] = {0, 0};
        for (int r = 0; r < 128; ++r) {
            const long long e = ((long long)mem * a.Bp + r0 + r) * a.H + o;
            const float d1 = __bfloat162float(a.DZ1[e]);
            gb1 += d1;
#pragma unroll
            for (int i = 0; i < kIn; ++i) gw1[i] = fmaf(d1, sxh[r][i], gw1[i]);
            gb2 += __bfloat162float(a.DZ2[e]);
            gb3 += __bfloat162float(a.DZ3[e]);
            const float h3 = __bfloat162float(a.H3[e]);
            gw4[0] = fmaf(sdy[r][0], h3, gw4[0]);
            gw4[1] = fmaf(sdy[r][1], h3, gw4[1]);
        }
        out[o] = gb1;
#pragma unroll
        for (int i = 0; i < kIn; ++i) out[a.H + o * kIn + i] = gw1[i];
        out[a.H * (1 + kIn) + o] = gb2;
        out[a.H * (2 + kIn) + o] = gb3;
        out[a.H * (3 + kIn) + o] = gw4[0];
        out[a.H * (4 + kIn) + o] = gw4[1];
    }
    if (threadIdx.x < kOut) {
        float s = 0;
        for (int r = 0; r < 128; ++r) s += sdy[r][threadIdx.x];
        out[a.H * (3 + kIn + kOut) + threadIdx.x] = s;
    }
}

__global__ void reduce_final_kernel(RedArgs a) {
    const int mem = blockIdx.y;
    const int nred = red_count(a.H);
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nred) return;
    const int nch = a.Bp / 128;
    const float* part = a.partial + (long long)mem * nch * nred;
    float s = 0;
    for (int c = 0; c < nch; ++c) s += part[(long long)c * nred + q];
    /* destination of value q in the packed member */
    const int H = a.H;
    long long dst;
    if (q < H) dst = a.off.b1 + q;
    else if (q < H * (1 + kIn)) dst = a.off.W1 + (q - H);
    else if (q < H * (2 + kIn)) dst = a.off.b2 + (q - H * (1 + kIn));
    else if (q < H * (3 + kIn)) dst = a.off.b3 + (q - H * (2 + kIn));
    else if (q < H * (4 + kIn)) dst = a.off.W4 + (q - H * (3 + kIn));
    else if (q < H * (5 + kIn)) dst = a.off.W4 + H + (q - H * (4 + kIn));
    else dst = a.off.b4 + (q - H * (5 + kIn));
    a.grad[mem * a.pstride + dst] = s;
}

__global__ void adam_kernel(AdamArgs a) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.pstride * a.members) return;
    const int mem = (int)(e / a.pstride);
    const long long q = e - (long long)mem * a.pstride;
    if (q >= a.count) return;
    const float g = a.g[e];
    const float m = a.beta1 * a.m[e] + (1.0f - a.beta1) * g;
    const float v = a.beta2 * a.v[e] + (1.0f - a.beta2) * g * g;
    a.m[e] = m;
    a.v[e] = v;
    const float p = a.p[e] - a.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
    a.p[e] = p;
    const long long HH = (long long)a.H * a.H;
    if (q >= a.oW2 && q < a.oW2 + HH)
        a.wb[(long long)mem * 2 * HH + (q - a.oW2)] = __float2bfloat16_rn(p);
    else if (q >= a.oW3 && q < a.oW3 + HH)
        a.wb[(long long)mem * 2 * HH + HH + (q - a.oW3)] = __float2bfloat16_rn(p);
}

__global__ void refresh_kernel(AdamArgs a) {
    const long long HH = (long long)a.H * a.H;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * HH * a.members) return;
    const int mem = (int)(e / (2 * HH));
    const long long q = e - mem * 2 * HH;
    const long long src = mem * a.pstride + (q < HH ? a.oW2 + q : a.oW3 + (q - HH));
    a.wb[e] = __float2bfloat16_rn(a.p[src]);
}

__global__ void ensemble_kernel(EnsArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n) return;
    float mean[kOut] = {0, 0}, sq[kOut] = {0, 0};
    for (int m = 0; m < a.members; ++m)
#pragma unroll
        for (int o = 0; o < kOut; ++o)
            mean[o] += a.Yh[((long long)m * a.Bp + r) * kOut + o] * a.sc.y_std[o] + a.sc.y_mean[o];
#pragma unroll
    for (int o = 0; o < kOut; ++o) mean[o] /= (float)a.members;
    for (int m = 0; m < a.members; ++m)
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            const float d =
                a.Yh[((long long)m * a.Bp + r) * kOut + o] * a.sc.y_std[o] + a.sc.y_mean[o] - mean[o];
            sq[o] += d * d;
        }
    float worst = 0.0f;
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
        const float s = sqrtf(sq[o] / (float)a.members);
        a.mean[(long long)r * kOut + o] = mean[o];
        a.stdv[(long long)r * kOut + o] = s;
        worst = fmaxf(worst, s);
    }
    /* NaN anywhere also sends the point to the solver */
    if (a.mask) a.mask[r] = !(worst <= a.threshold);
}

int ok_or(cudaError_t e) { return e == cudaSuccess ? 0 : (int)e; }

}  // namespace

int reduce_count(int H) { return red_count(H); }

template <bool AMN, bool BMN, int EPI>
static int launch_tc(const GemmArgs& a, int members, cudaStream_t s) {
    const void* fn = reinterpret_cast<const void*>(&gemm_tc_kernel<AMN, BMN, EPI>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem);
    if (e != cudaSuccess) return (int)e;
    const dim3 grid(a.N / GN, a.M / GM, members);
    gemm_tc_kernel<AMN, BMN, EPI><<<grid, kGThreads, kGSmem, s>>>(a);
    return ok_or(cudaGetLastError());
}

int launch_gemm(const GemmArgs& a, bool a_kmajor, bool b_kmajor, int epi, int members,
                void* stream) {
    if (a.M % GM || a.N % GN || a.K % GK || a.M <= 0 || a.N <= 0 || a.K <= 0)
        return (int)cudaErrorInvalidValue;
    cudaStream_t s = (cudaStream_t)stream;
    if (!a_kmajor && !b_kmajor && epi == EPI_FWD) return launch_tc<false, false, EPI_FWD>(a, members, s);
    if (!a_kmajor && b_kmajor && epi == EPI_BWD) return launch_tc<false, true, EPI_BWD>(a, members, s);
    if (a_kmajor && b_kmajor && epi == EPI_F32) return launch_tc<true, true, EPI_F32>(a, members, s);
    if (!a_kmajor && !b_kmajor && epi == EPI_F32) return launch_tc<false, false, EPI_F32>(a, members, s);
    return (int)cudaErrorInvalidValue;
}

int launch_l1(const L1Args& a, int members, void* stream) {
    const long long n = (long long)a.Bp * a.H;
    const dim3 grid((unsigned)((n + 255) / 256), members);
    l1_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
    return ok_or(cudaGetLastError());
}

int launch_head(const HeadArgs& a, int members, void* stream) {
    const dim3 grid((unsigned)((a.Bp + 7) / 8), members);
    head_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
    return ok_or(cudaGetLastError());
}

int launch_reduce(const RedArgs& a, int members, void* stream) {
    reduce_partial_kernel<<<dim3(a.Bp / 128, members), 256, 0, (cudaStream_t)stream>>>(a);
    int rc = ok_or(cudaGetLastError());
    if (rc) return rc;
    const int nred = red_count(a.H);
    reduce_final_kernel<<<dim3((nred + 255) / 256, members), 256, 0, (cudaStream_t)stream>>>(a);
    return ok_or(cudaGetLastError());
}

int launch_adam(const AdamArgs& a, void* stream) {
    const long long n = a.pstride * a.members;
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(a);
    return ok_or(cudaGetLastError());
}

int launch_refresh_bf16(const AdamArgs& a, void* stream) {
    const long long n = 2ll * a.H * a.H * a.members;
    refresh_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(a);
    return ok_or(cudaGetLastError());
}

int launch_ensemble(const EnsArgs& a, void* stream) {
    ensemble_kernel<<<(a.n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(a);
    return ok_or(cudaGetLastError());
}

}  // namespace sur
}  // namespace bte
