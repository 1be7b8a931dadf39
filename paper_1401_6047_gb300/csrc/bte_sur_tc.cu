/*
 * bte_sur_tc.cu -- ensemble inference of the surrogate MLP on the fifth-
 * generation tensor cores (tcgen05, sm_103a).
 *
 * Persistent CTAs: about one per SM, each bound to one ensemble member and
 * walking that member's 128-row tiles.  Sixteen compute warps and one MMA
 * warp share shared memory through mbarriers:
 *
 *   compute warps   layer 1 (5 inputs, FP32 cores) -> h1 in four K-chunks
 *                   of 64 columns, each chunk signalled when written;
 *                   epilogue of layer 2 (tcgen05.ld, bias, SiLU, BF16) ->
 *                   h2 in place, again chunk by chunk; epilogue of layer 3
 *                   fused with the 2-output layer (h3 never stored)
 *   MMA warp        per chunk as it is signalled, the layer's 2 x 4
 *                   tcgen05.mma (M = 128, N = 128, K = 16, BF16 in, FP32
 *                   accumulators: layer 2 in tensor-memory columns 0..255,
 *                   layer 3 in 256..511), a commit per layer; the weight
 *                   halves of the next layer by bulk copy as soon as the
 *                   previous layer's MMAs are complete
 *
 * so each layer's MMAs run under the epilogue that produces their operand,
 * chunk by chunk.  Operands sit in the tensor cores' canonical K-major
 * layout without swizzle (8 x 8 core matrices; K-adjacent ones 128 bytes
 * apart, 8-row groups 4096 bytes apart).
 *
 * Every wait on an mbarrier is bounded (about 2 s of %globaltimer).  A wait
 * that gives up raises the CTA's abort flag: every later wait returns at
 * once, no further MMA or copy is issued, the work of the remaining tiles
 * is skipped (named barriers are still passed, so no warp waits forever),
 * copies already issued are waited for (bounded), the error word is set and
 * the tensor memory is freed before the CTA exits.
 */
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "bte_device.cuh"
#include "bte_sur_internal.h"
#include "bte_tc.cuh"

namespace bte {
namespace sur {
namespace {

using namespace tc;

constexpr int TM = 128;             /* rows per tile (MMA M) */
constexpr int TH = 256;             /* hidden width */
constexpr int TN = 128;             /* MMA N (one weight half) */
constexpr int TK = 16;              /* MMA K */
constexpr int kChunk = 64;          /* K columns per signalled chunk */
constexpr int kNChunk = TH / kChunk;
constexpr int kCompWarps = 16;      /* 4 per tensor-memory lane quadrant */
constexpr int kCompThreads = kCompWarps * 32;
constexpr int kThreadsTC = kCompThreads + 32; /* + the MMA warp */
constexpr uint32_t kHalfBytes = (uint32_t)TN * TH * 2; /* 64 KB */
constexpr uint32_t kOpBytes = (uint32_t)TM * TH * 2;   /* 64 KB */
constexpr uint32_t kCoreStride = 128;                  /* bytes of one 8 x 8 core matrix */
constexpr uint32_t kGroupStride = (TH / 8) * kCoreStride; /* 4096: next 8-row group */
/* dynamic shared memory: operand h, two weight halves, small parameters,
 * output partial sums, barriers */
constexpr size_t kOffH = 0;
constexpr size_t kOffW0 = kOffH + kOpBytes;
constexpr size_t kOffW1 = kOffW0 + kHalfBytes;
constexpr size_t kOffW1s = kOffW1 + kHalfBytes;           /* W1 [256][5] */
constexpr size_t kOffB = kOffW1s + (size_t)TH * kIn * 4;  /* b1, b2, b3 [256] each */
constexpr size_t kOffW4 = kOffB + 3 * (size_t)TH * 4;     /* W4 [2][256], b4 [2] */
constexpr size_t kOffRed = kOffW4 + (2 * (size_t)TH + 4) * 4; /* [4][128][2] partial outputs */
constexpr size_t kOffX = kOffRed + 4 * (size_t)TM * 2 * 4;      /* [128][5] raw inputs */
constexpr size_t kOffBar = kOffX + (size_t)TM * kIn * 4;
/* barriers: wbar[2] (weight halves), cbar[4] (h chunks), mbar (MMA commits) */
constexpr size_t kSmemTC = kOffBar + 128 + 1024; /* + alignment slack */

/* silu(z) = z / (1 + exp(-z)), fast exponential and reciprocal (as in training) */
__device__ __forceinline__ float silu_tc(float z) { return z * __fdividef(1.0f, 1.0f + __expf(-z)); }

/* byte offset of element (r, k) of a [rows][256] K-major operand in the
 * canonical no-swizzle layout */
__host__ __device__ __forceinline__ uint32_t canon(int r, int k) {
    return (uint32_t)(((r >> 3) * (TH / 8) + (k >> 3)) * kCoreStride + (r & 7) * 16 + (k & 7) * 2);
}

/* Bounded mbarrier wait that also gives up at once when another thread of
 * the CTA has raised the abort flag; a wait that runs out raises it.  Each
 * retry may sleep up to 10 us in the barrier unit (woken by the phase). */
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort) {
    if (dev::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = dev::global_timer();
    while (!dev::mbar_try_wait_sleep(bar, parity, 10000u)) {
        if (*abort) return false;
        if (dev::global_timer() - t0 > dev::kWaitLimitNs) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void comp_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kCompThreads) : "memory");
}

__global__ void __launch_bounds__(kThreadsTC, 1) infer_tc_kernel(InferArgs a) {
    extern __shared__ unsigned char tsm_raw[];
    /* 1024-byte aligned base (descriptor addresses are 16-byte units) */
    unsigned char* tsm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tsm_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* hS = tsm + kOffH;
    float* sW1 = reinterpret_cast<float*>(tsm + kOffW1s);
    float* sB = reinterpret_cast<float*>(tsm + kOffB);
    float* sW4 = reinterpret_cast<float*>(tsm + kOffW4);
    float* red = reinterpret_cast<float*>(tsm + kOffRed);
    float* sX = reinterpret_cast<float*>(tsm + kOffX);
    uint64_t* bars = reinterpret_cast<uint64_t*>(tsm + kOffBar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tsm + kOffBar + 64);
    volatile int* abort = reinterpret_cast<volatile int*>(tsm + kOffBar + 72);
    const uint32_t aH = dev::smem_u32(hS);
    const uint32_t aW0 = dev::smem_u32(tsm + kOffW0);
    const uint32_t bW0 = dev::smem_u32(&bars[0]); /* half h: bW0 + 8 h */
    const uint32_t bC0 = dev::smem_u32(&bars[2]); /* chunk c: bC0 + 8 c */
    const uint32_t bM = dev::smem_u32(&bars[6]);

    const int mem = blockIdx.y, ntile = a.Bp / TM;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* P = a.params + mem * a.pstride;
    const unsigned char* Wg = reinterpret_cast<const unsigned char*>(a.wti) + (size_t)mem * 4 * kHalfBytes;

    /* small parameters of the member into shared memory */
    for (int i = tid; i < TH * kIn; i += kThreadsTC) sW1[i] = P[a.off.W1 + i];
    for (int i = tid; i < TH; i += kThreadsTC) {
        sB[i] = P[a.off.b1 + i];
        sB[TH + i] = P[a.off.b2 + i];
        sB[2 * TH + i] = P[a.off.b3 + i];
    }
    for (int i = tid; i < kOut * TH; i += kThreadsTC) sW4[i] = P[a.off.W4 + i];
    if (tid < kOut) sW4[kOut * TH + tid] = P[a.off.b4 + tid];
    if (tid == 0) {
        dev::mbar_init(bW0, 1);
        dev::mbar_init(bW0 + 8, 1);
        for (int c = 0; c < kNChunk; ++c) dev::mbar_init(bC0 + 8 * c, kCompWarps);
        dev::mbar_init(bM, 1);
        *abort = 0;
        dev::fence_proxy_async_smem();
    }
    if (warp == kCompWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         dev::smem_u32(tmem_slot)),
                     "r"(2 * TH)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == kCompWarps) {
        /* ---------------- MMA warp (lane 0 issues) ---------------- */
        if (lane == 0) {
            int pend_w = 0; /* weight-layer loads issued and not yet waited for */
            uint32_t wpar = 0;
            auto load_layer = [&](int l) {
                for (int hh = 0; hh < 2; ++hh) {
                    dev::mbar_arrive_tx(bW0 + 8 * hh, kHalfBytes);
                    const unsigned char* src = Wg + (size_t)(2 * l + hh) * kHalfBytes;
                    for (int c = 0; c < 4; ++c)
                        dev::bulk_g2s(aW0 + hh * kHalfBytes + c * (kHalfBytes / 4), src + c * (kHalfBytes / 4),
                                      kHalfBytes / 4, bW0 + 8 * hh);
                }
                ++pend_w;
            };
            auto wait_layer = [&]() {
                const bool ok = wait_or_abort(bW0, wpar, abort) && wait_or_abort(bW0 + 8, wpar, abort);
                if (ok) {
                    --pend_w;
                    wpar ^= 1u;
                }
                return ok;
            };
            constexpr uint32_t idesc = instr_desc(TM, TN);
            bool first = true;
            for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
                if (*abort) break;
                if (first) load_layer(0);
                first = false;
                for (int l = 0; l < 2; ++l) {
                    /* layer l + 2: weights, then each chunk of its operand as it is written */
                    if (!wait_layer()) break;
                    tc_fence_after();
                    const uint32_t acc = tmem + (uint32_t)(l * TH);
                    bool ok = true;
                    for (int c = 0; c < kNChunk && ok; ++c) {
                        ok = wait_or_abort(bC0 + 8 * c, (uint32_t)l, abort);
                        if (!ok) break;
                        tc_fence_after();
                        for (int hh = 0; hh < 2; ++hh)
                            for (int k4 = 0; k4 < kChunk / TK; ++k4) {
                                const int ks = c * (kChunk / TK) + k4;
                                const uint64_t ad = smem_desc(aH + ks * 2 * kCoreStride, kCoreStride, kGroupStride);
                                const uint64_t bd = smem_desc(aW0 + hh * kHalfBytes + ks * 2 * kCoreStride,
                                                              kCoreStride, kGroupStride);
                                tc_mma(acc + hh * TN, ad, bd, idesc, ks > 0 ? 1u : 0u);
                            }
                    }
                    if (!ok) break;
                    tc_commit(bM);
                    /* the layer's MMAs are complete: the weight buffers are free */
                    if (!wait_or_abort(bM, (uint32_t)l, abort)) break;
                    if (l == 0) load_layer(1);
                    else if (tile + (int)gridDim.x < ntile) load_layer(0);
                }
            }
            /* copies still in flight (only after an abort) land before the CTA exits */
            for (int i = 0; i < pend_w; ++i) {
                dev::mbar_wait(bW0, wpar);
                dev::mbar_wait(bW0 + 8, wpar);
                wpar ^= 1u;
            }
        }
        __syncwarp();
    } else {
        /* ---------------- compute warps ---------------- */
        const int q = warp & 3;   /* tensor-memory lane quadrant: rows 32 q .. 32 q + 31 */
        const int sc = warp >> 2; /* column sub-block of the epilogues */
        const int ug = warp & 7;  /* layer 1: unit group (8 units) of each chunk */
        const int rl0 = (warp >> 3) * 64 + lane; /* layer 1: rows rl0, rl0 + 32 */
        const int erow = q * 32 + lane;          /* epilogue row (tensor-memory lane) */
        const uint32_t tl = (uint32_t)(q * 32) << 16;
        /* the raw inputs of a tile's 128 rows go to shared memory by
         * asynchronous 4-byte copies (zero-filled past nvalid), issued one
         * tile ahead by warps 0 and 8 (rows rl0, rl0 + 32 of each lane) */
        auto fetch_x = [&](int tile) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int rl = rl0 + 32 * j, row = tile * TM + rl;
                const bool in = row < a.nvalid;
                const float* src = a.x + (in ? (a.row0 + row) * kIn : 0);
#pragma unroll
                for (int i = 0; i < kIn; ++i)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                                     dev::smem_u32(sX + rl * kIn + i)),
                                 "l"(src + i), "r"(in ? 4 : 0)
                                 : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        if (blockIdx.x < ntile && ug == 0) fetch_x(blockIdx.x);
        for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
            const bool run = !*abort;
            const int r0 = tile * TM;
            /* ---- layer 1 on the FP32 cores, chunk by chunk ---- */
            if (ug == 0) asm volatile("cp.async.wait_all;" ::: "memory");
            comp_sync(); /* every row's inputs have landed */
            float xh[2][kIn];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int rl = rl0 + 32 * j;
                const bool in = r0 + rl < a.nvalid;
#pragma unroll
                for (int i = 0; i < kIn; ++i)
                    xh[j][i] = in ? 2.0f * (sX[rl * kIn + i] - a.sc.x_lo[i]) * a.sc.x_inv[i] - 1.0f : 0.0f;
            }
            for (int c = 0; c < kNChunk; ++c) {
                if (run) {
                    const int u0 = c * kChunk + 8 * ug;
                    /* W1 rows u0 .. u0 + 7 (40 values) and b1, as 16-byte loads */
                    float w[8][kIn], b[8];
                    {
                        float wf[8 * kIn];
                        const float4* w4 = reinterpret_cast<const float4*>(sW1 + u0 * kIn);
#pragma unroll
                        for (int q4 = 0; q4 < 2 * kIn; ++q4) {
                            const float4 t = w4[q4];
                            wf[4 * q4] = t.x;
                            wf[4 * q4 + 1] = t.y;
                            wf[4 * q4 + 2] = t.z;
                            wf[4 * q4 + 3] = t.w;
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u)
#pragma unroll
                            for (int i = 0; i < kIn; ++i) w[u][i] = wf[u * kIn + i];
                        const float4 b0 = reinterpret_cast<const float4*>(sB + u0)[0];
                        const float4 b1v = reinterpret_cast<const float4*>(sB + u0)[1];
                        b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
                        b[4] = b1v.x; b[5] = b1v.y; b[6] = b1v.z; b[7] = b1v.w;
                    }
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        __nv_bfloat162 pk[4];
#pragma unroll
                        for (int u = 0; u < 8; u += 2) {
                            float z0 = b[u], z1 = b[u + 1];
#pragma unroll
                            for (int i = 0; i < kIn; ++i) {
                                z0 = fmaf(w[u][i], xh[j][i], z0);
                                z1 = fmaf(w[u + 1][i], xh[j][i], z1);
                            }
                            pk[u / 2] = __floats2bfloat162_rn(silu_tc(z0), silu_tc(z1));
                        }
                        *reinterpret_cast<uint4*>(hS + canon(rl0 + 32 * j, u0)) =
                            *reinterpret_cast<const uint4*>(pk);
                    }
                }
                /* the chunk's operand bytes -> visible to the tensor cores */
                dev::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) dev::mbar_arrive(bC0 + 8 * c);
            }
            /* ---- layer 2 epilogue -> h2, chunk by chunk ---- */
            const bool ok2 = run && wait_or_abort(bM, 0u, abort);
            tc_fence_after();
            for (int c = 0; c < kNChunk; ++c) {
                if (ok2) {
                    const int col0 = c * kChunk + sc * 16;
                    float v[16];
                    tc_ld16(tmem + tl + (uint32_t)col0, v);
                    float bias[16];
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const float4 t = reinterpret_cast<const float4*>(sB + TH + col0)[q4];
                        bias[4 * q4] = t.x;
                        bias[4 * q4 + 1] = t.y;
                        bias[4 * q4 + 2] = t.z;
                        bias[4 * q4 + 3] = t.w;
                    }
#pragma unroll
                    for (int h8 = 0; h8 < 16; h8 += 8) {
                        __nv_bfloat162 pk[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            pk[e] = __floats2bfloat162_rn(silu_tc(v[h8 + 2 * e] + bias[h8 + 2 * e]),
                                                          silu_tc(v[h8 + 2 * e + 1] + bias[h8 + 2 * e + 1]));
                        *reinterpret_cast<uint4*>(hS + canon(erow, col0 + h8)) =
                            *reinterpret_cast<const uint4*>(pk);
                    }
                }
                tc_fence_before();
                dev::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) dev::mbar_arrive(bC0 + 8 * c);
            }
            /* ---- layer 3 epilogue fused with the output layer (N = 2) ---- */
            const bool ok3 = ok2 && wait_or_abort(bM, 1u, abort);
            tc_fence_after();
            /* the next tile's inputs (layer 1 of this tile has read sX) */
            if (ug == 0 && tile + (int)gridDim.x < ntile) fetch_x(tile + gridDim.x);
            float y0 = 0.0f, y1 = 0.0f;
            if (ok3) {
#pragma unroll 1
                for (int q4 = 0; q4 < 4; ++q4) {
                    const int col0 = sc * 64 + 16 * q4;
                    float v[16];
                    tc_ld16(tmem + tl + (uint32_t)(TH + col0), v);
                    float bias[16], w40[16], w41[16];
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        const float4 tb = reinterpret_cast<const float4*>(sB + 2 * TH + col0)[k4];
                        const float4 t0 = reinterpret_cast<const float4*>(sW4 + col0)[k4];
                        const float4 t1 = reinterpret_cast<const float4*>(sW4 + TH + col0)[k4];
                        bias[4 * k4] = tb.x; bias[4 * k4 + 1] = tb.y; bias[4 * k4 + 2] = tb.z; bias[4 * k4 + 3] = tb.w;
                        w40[4 * k4] = t0.x; w40[4 * k4 + 1] = t0.y; w40[4 * k4 + 2] = t0.z; w40[4 * k4 + 3] = t0.w;
                        w41[4 * k4] = t1.x; w41[4 * k4 + 1] = t1.y; w41[4 * k4 + 2] = t1.z; w41[4 * k4 + 3] = t1.w;
                    }
#pragma unroll
                    for (int e = 0; e < 16; e += 2) {
                        /* h3 rounded to BF16 as the operand of a tensor-core layer would be */
                        const float2 hf = __bfloat1622float2(
                            __floats2bfloat162_rn(silu_tc(v[e] + bias[e]), silu_tc(v[e + 1] + bias[e + 1])));
                        y0 = fmaf(w40[e], hf.x, y0);
                        y0 = fmaf(w40[e + 1], hf.y, y0);
                        y1 = fmaf(w41[e], hf.x, y1);
                        y1 = fmaf(w41[e + 1], hf.y, y1);
                    }
                }
            }
            red[(sc * TM + erow) * 2] = y0;
            red[(sc * TM + erow) * 2 + 1] = y1;
            tc_fence_before();
            comp_sync();
            if (tid < TM && ok3) {
                float o0 = sW4[kOut * TH], o1 = sW4[kOut * TH + 1];
#pragma unroll
                for (int s4 = 0; s4 < 4; ++s4) {
                    o0 += red[(s4 * TM + tid) * 2];
                    o1 += red[(s4 * TM + tid) * 2 + 1];
                }
                const long long yo = ((long long)mem * a.Bp + r0 + tid) * kOut;
                a.Yh[yo] = o0;
                a.Yh[yo + 1] = o1;
            }
            comp_sync(); /* red is free for the next tile */
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kCompWarps)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TH)
                     : "memory");
    if (tid == 0 && *abort) atomicExch(a.err, 1);
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
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    /* about one CTA per SM: ceil(SMs / members) per member, each walking
     * every gridDim.x-th tile of its member */
    const int ntile = a.Bp / TM;
    const int per = std::max(1, std::min(ntile, (sms + members - 1) / members));
    const dim3 grid(per, members);
    infer_tc_kernel<<<grid, kThreadsTC, kSmemTC, (cudaStream_t)stream>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace sur
}  // namespace bte
