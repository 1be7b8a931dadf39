/*
 * bte_sur_tc.cu -- ensemble inference of the surrogate MLP on the fifth-
 * generation tensor cores (tcgen05, sm_103a).
 *
 * One CTA takes two 128-row tiles of one member, one after the other.  The
 * 5-input layer runs on the FP32 cores and writes h1 (BF16) into shared
 * memory in the tensor cores' canonical K-major layout (8 x 8 core
 * matrices, no swizzle).  Each 256 x 256
 * layer is 2 x 16 tcgen05.mma instructions (M = 128, N = 128, K = 16, BF16
 * in, FP32 accumulate) issued by one thread into 256 columns of tensor
 * memory; the weight halves (64 KB each) arrive by bulk copy into two
 * shared-memory buffers, the next layer's while the epilogue runs.  The
 * epilogue reads the accumulators back (tcgen05.ld), adds the bias, applies
 * SiLU and writes the next layer's BF16 operand in place.  The 2-output
 * layer reads h3 from shared memory on the FP32 cores.
 *
 * Every wait on an mbarrier is bounded (about 2 s of %globaltimer); a wait
 * that gives up sets the error word and the CTA still frees its tensor
 * memory before it exits.
 */
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bte_device.cuh"
#include "bte_sur_internal.h"
#include "bte_tc.cuh"

namespace bte {
namespace sur {
namespace {

using namespace tc;

constexpr int TM = 128;             /* rows per CTA (MMA M) */
constexpr int TH = 256;             /* hidden width */
constexpr int TN = 128;             /* MMA N (one weight half) */
constexpr int TK = 16;              /* MMA K */
constexpr int kThreadsTC = 512; /* 16 warps: 4 per tensor-memory lane quadrant */
constexpr int kTPC = 2;         /* row tiles per CTA, one after another */
constexpr uint32_t kHalfBytes = (uint32_t)TN * TH * 2; /* 64 KB */
constexpr uint32_t kOpBytes = (uint32_t)TM * TH * 2;   /* 64 KB */
constexpr uint32_t kCoreStride = 128;                  /* bytes of one 8 x 8 core matrix */
constexpr uint32_t kGroupStride = (TH / 8) * kCoreStride; /* 4096: next 8-row group */
/* dynamic shared memory: operand h, two weight halves, inputs, barriers */
constexpr size_t kOffH = 0;
constexpr size_t kOffW0 = kOffH + kOpBytes;
constexpr size_t kOffW1 = kOffW0 + kHalfBytes;
constexpr size_t kOffX = kOffW1 + kHalfBytes;
constexpr size_t kOffBias = kOffX + (size_t)TM * kIn * 4; /* b2, b3 */
constexpr size_t kOffW4 = kOffBias + 2 * (size_t)TH * 4;  /* W4 [2][256], b4 [2] */
constexpr size_t kOffBar = kOffW4 + (2 * (size_t)TH + 4) * 4;
constexpr size_t kSmemTC = kOffBar + 64 + 1024; /* + alignment slack */

/* silu(z) = z / (1 + exp(-z)), fast exponential and reciprocal (as in training) */
__device__ __forceinline__ float silu_tc(float z) { return z * __fdividef(1.0f, 1.0f + __expf(-z)); }

/* byte offset of element (r, k) of a [rows][256] K-major operand in the
 * canonical no-swizzle layout */
__host__ __device__ __forceinline__ uint32_t canon(int r, int k) {
    return (uint32_t)(((r >> 3) * (TH / 8) + (k >> 3)) * kCoreStride + (r & 7) * 16 + (k & 7) * 2);
}

__global__ void __launch_bounds__(kThreadsTC, 1) infer_tc_kernel(InferArgs a) {
    extern __shared__ unsigned char tsm_raw[];
    /* 1024-byte aligned base (descriptor addresses are 16-byte units) */
    unsigned char* tsm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tsm_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* hS = tsm + kOffH;
    float* sx = reinterpret_cast<float*>(tsm + kOffX);
    float* sb = reinterpret_cast<float*>(tsm + kOffBias);
    float* sw4 = reinterpret_cast<float*>(tsm + kOffW4);
    uint64_t* bars = reinterpret_cast<uint64_t*>(tsm + kOffBar); /* w0, w1, mma */
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tsm + kOffBar + 32);
    const uint32_t aH = dev::smem_u32(hS);
    const uint32_t aW[2] = {dev::smem_u32(tsm + kOffW0), dev::smem_u32(tsm + kOffW1)};
    const uint32_t bW[2] = {dev::smem_u32(&bars[0]), dev::smem_u32(&bars[1])};
    const uint32_t bM = dev::smem_u32(&bars[2]);

    const int mem = blockIdx.y, ntile = a.Bp / TM;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* P = a.params + mem * a.pstride;
    const unsigned char* Wg = reinterpret_cast<const unsigned char*>(a.wti) + (size_t)mem * 4 * kHalfBytes;
    bool ok = true;

    /* every global parameter load of the CTA is issued here, so that their
     * latencies overlap (biases of layers 2, 3 and the output layer's weights
     * go to shared memory).  Layer 1: the thread computes units
     * 8 ug1 .. 8 ug1 + 7 of rows 8 (rb1 + 2k) + (lane & 7), k = 0..7, so
     * that a quarter-warp writes one 8 x 8 core matrix (128 contiguous bytes)
     * with one 16-byte store per lane. */
    const int q1 = 4 * warp + (lane >> 3);
    const int ug1 = q1 & 31, rb1 = q1 >> 5;
    float w1[8][kIn], b1[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
        for (int i = 0; i < kIn; ++i) w1[u][i] = P[a.off.W1 + (long long)(8 * ug1 + u) * kIn + i];
        b1[u] = P[a.off.b1 + 8 * ug1 + u];
    }
    if (tid < TH) {
        sb[tid] = P[a.off.b2 + tid];
        sb[TH + tid] = P[a.off.b3 + tid];
    }
    sw4[tid] = P[a.off.W4 + tid]; /* 512 threads: both output rows */
    if (tid < kOut) sw4[2 * TH + tid] = P[a.off.b4 + tid];

    if (tid == 0) {
        dev::mbar_init(bW[0], 1);
        dev::mbar_init(bW[1], 1);
        dev::mbar_init(bM, 1);
        dev::fence_proxy_async_smem();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         dev::smem_u32(tmem_slot)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    /* weight halves of layer `l` into both buffers (4 bulk copies of 16 KB each) */
    auto load_layer = [&](int l) {
        for (int hh = 0; hh < 2; ++hh) {
            dev::mbar_arrive_tx(bW[hh], kHalfBytes);
            const unsigned char* src = Wg + (size_t)(2 * l + hh) * kHalfBytes;
            for (int c = 0; c < 4; ++c)
                dev::bulk_g2s(aW[hh] + c * (kHalfBytes / 4), src + c * (kHalfBytes / 4), kHalfBytes / 4,
                              bW[hh]);
        }
    };
    if (tid == 0) load_layer(0);

    /* the CTA's row tiles, one after another with the same member: set-up,
     * tensor memory and the small parameters serve both, and the next
     * tile's first weight layer streams in under this tile's last
     * epilogue.  Each barrier completes once per layer, so its wait parity
     * is the layer index in every tile. */
    for (int it = 0; it < kTPC; ++it) {
        const int tile = blockIdx.x * kTPC + it;
        if (tile >= ntile) break;
        const int r0 = tile * TM;

        /* ---- layer 1 on the FP32 cores: h1 = silu(W1 xh + b1) ---- */
        for (int r = tid; r < TM; r += kThreadsTC) {
            const int row = r0 + r;
            float xh[kIn];
            if (row < a.nvalid) {
                const long long s = a.row0 + row;
    #pragma unroll
                for (int i = 0; i < kIn; ++i)
                    xh[i] = 2.0f * (a.x[s * kIn + i] - a.sc.x_lo[i]) * a.sc.x_inv[i] - 1.0f;
            } else {
    #pragma unroll
                for (int i = 0; i < kIn; ++i) xh[i] = 0.0f;
            }
    #pragma unroll
            for (int i = 0; i < kIn; ++i) sx[r * kIn + i] = xh[i];
        }
        __syncthreads();
    #pragma unroll 1
        for (int k = 0; k < TM / 16; ++k) {
            const int r = 8 * (rb1 + 2 * k) + (lane & 7);
            float xv[kIn];
    #pragma unroll
            for (int i = 0; i < kIn; ++i) xv[i] = sx[r * kIn + i];
            __nv_bfloat162 pk[4];
    #pragma unroll
            for (int u = 0; u < 8; u += 2) {
                float z0 = b1[u], z1 = b1[u + 1];
    #pragma unroll
                for (int i = 0; i < kIn; ++i) {
                    z0 = fmaf(w1[u][i], xv[i], z0);
                    z1 = fmaf(w1[u + 1][i], xv[i], z1);
                }
                pk[u / 2] = __floats2bfloat162_rn(silu_tc(z0), silu_tc(z1));
            }
            *reinterpret_cast<uint4*>(hS + canon(r, 8 * ug1)) = *reinterpret_cast<const uint4*>(pk);
        }

        /* ---- layers 2 and 3 ---- */
        constexpr uint32_t idesc = instr_desc(TM, TN);
        const int sub = warp & 3;             /* TMEM lanes 32 sub .. 32 sub + 31 */
        const int cq = warp >> 2;             /* accumulator columns 64 cq .. 64 cq + 63 */
        for (int l = 0; l < 2; ++l) {
            /* operand written by the generic proxy -> visible to the tensor cores */
            dev::fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                for (int hh = 0; hh < 2; ++hh)
                    if (!dev::mbar_wait(bW[hh], (uint32_t)l)) ok = false;
                tc_fence_after();
                for (int hh = 0; hh < 2; ++hh)
                    for (int ks = 0; ks < TH / TK; ++ks) {
                        const uint64_t ad = smem_desc(aH + ks * 2 * kCoreStride, kCoreStride, kGroupStride);
                        const uint64_t bd =
                            smem_desc(aW[hh] + ks * 2 * kCoreStride, kCoreStride, kGroupStride);
                        tc_mma(tmem + hh * TN, ad, bd, idesc, ks > 0 ? 1u : 0u);
                    }
                tc_commit(bM);
            }
            if (!dev::mbar_wait(bM, (uint32_t)l)) ok = false;
            tc_fence_after();
            /* the weight buffers are free: fetch the next layer's */
            if (tid == 0 && l == 0) load_layer(1);
            if (tid == 0 && l == 1 && it + 1 < kTPC && tile + 1 < ntile) load_layer(0);
            /* epilogue: bias + SiLU, BF16, written as the next operand (row = TMEM lane) */
            const float* bias = sb + l * TH;
            const int row = sub * 32 + lane;
            for (int cb = 0; cb < TH / 4; cb += 32) {
                const int col0 = cq * (TH / 4) + cb;
                float v[32];
                tc_ld32(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)col0, v);
    #pragma unroll
                for (int c8 = 0; c8 < 32; c8 += 8) {
                    __nv_bfloat162 pk[4];
    #pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int col = col0 + c8 + 2 * e;
                        pk[e] = __floats2bfloat162_rn(silu_tc(v[c8 + 2 * e] + bias[col]),
                                                      silu_tc(v[c8 + 2 * e + 1] + bias[col + 1]));
                    }
                    *reinterpret_cast<uint4*>(hS + canon(row, col0 + c8)) =
                        *reinterpret_cast<const uint4*>(pk);
                }
            }
        }
        tc_fence_before();
        __syncthreads();

        /* ---- output layer (N = 2): one warp per row, lane c reads units 8c .. 8c+7 ---- */
        float w40[8], w41[8];
    #pragma unroll
        for (int i = 0; i < 8; ++i) {
            w40[i] = sw4[lane * 8 + i];
            w41[i] = sw4[TH + lane * 8 + i];
        }
        const float b40 = sw4[2 * TH], b41 = sw4[2 * TH + 1];
        for (int r = warp; r < TM; r += kThreadsTC / 32) {
            const uint4 raw = *reinterpret_cast<const uint4*>(hS + canon(r, lane * 8));
            const __nv_bfloat162* hp = reinterpret_cast<const __nv_bfloat162*>(&raw);
            float y0 = 0.0f, y1 = 0.0f;
    #pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 f = __bfloat1622float2(hp[i]);
                y0 = fmaf(w40[2 * i], f.x, y0);
                y0 = fmaf(w40[2 * i + 1], f.y, y0);
                y1 = fmaf(w41[2 * i], f.x, y1);
                y1 = fmaf(w41[2 * i + 1], f.y, y1);
            }
    #pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                y0 += __shfl_xor_sync(0xffffffffu, y0, o);
                y1 += __shfl_xor_sync(0xffffffffu, y1, o);
            }
            if (lane == 0) {
                const long long yo = ((long long)mem * a.Bp + r0 + r) * kOut;
                a.Yh[yo] = y0 + b40;
                a.Yh[yo + 1] = y1 + b41;
            }
        }
        __syncthreads(); /* h and the inputs are free for the next tile */
    }
    if (!ok) atomicExch(a.err, 1);
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256)
                     : "memory");
}

/* W2, W3 of every member as BF16 in the canonical layout: [member][layer][half][128 x 256] */
__global__ void canon_weights_kernel(const float* params, long long pstride, ParamOffsets off,
                                     __nv_bfloat16* wti, int members) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per = 2ll * TH * TH;
    if (e >= per * members) return;
    const int mem = (int)(e / per);
    const long long q = e - mem * per;
    const int l = (int)(q / (TH * TH));
    const int n = (int)((q / TH) % TH), k = (int)(q % TH);
    const float v = params[mem * pstride + (l == 0 ? off.W2 : off.W3) + (long long)n * TH + k];
    unsigned char* dst = reinterpret_cast<unsigned char*>(wti) +
                         ((size_t)mem * 4 + 2 * l + n / TN) * kHalfBytes + canon(n % TN, k);
    *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
}

}  // namespace

int launch_canon_weights(const float* params, long long pstride, const ParamOffsets& off,
                         __nv_bfloat16* wti, int members, void* stream) {
    const long long n = 2ll * TH * TH * members;
    canon_weights_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        params, pstride, off, wti, members);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : (int)e;
}

int launch_infer_tc(const InferArgs& a, int members, void* stream) {
    cudaError_t e = cudaFuncSetAttribute(infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemTC);
    if (e != cudaSuccess) return (int)e;
    const dim3 grid((a.Bp / TM + kTPC - 1) / kTPC, members);
    infer_tc_kernel<<<grid, kThreadsTC, kSmemTC, (cudaStream_t)stream>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace sur
}  // namespace bte
