/*
 * bte_sur_kernels.cu -- CUDA kernels of the MLP surrogate (sm_103a).
 *
 * The two 256 x 256 hidden layers and their backward products run on the
 * BF16 tensor cores (mma.sync m16n8k16, FP32 accumulation) in one GEMM
 * kernel whose epilogue fuses the bias, the SiLU activation and its
 * derivative.  The thin layers (5 inputs, 2 outputs) are FP32 FMA kernels;
 * batch reductions are two-pass and deterministic; Adam keeps FP32 master
 * weights and refreshes the BF16 operand copies in the same pass.
 */
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bte_sur_internal.h"

namespace bte {
namespace sur {
namespace {

constexpr int BM = 128, BN = 128, BK = 32;
constexpr int kThreads = 256; /* 8 warps: 2 along M x 4 along N, warp tile 64 x 32 */
constexpr int PAD = 8;        /* bf16 elements of row padding (16 bytes) */
/* one stage: the larger of the [128][32+8] and [32][128+8] tile shapes */
constexpr int kTileElems = (BM * (BK + PAD) > BK * (BM + PAD)) ? BM * (BK + PAD) : BK * (BM + PAD);

/* sigmoid(z) = 1 / (1 + exp(-z)) with the fast exponential and reciprocal
 * (relative error ~1e-7, so the bfloat16 rounding that follows matches an
 * exact evaluation; exp(-z) = inf gives 0) */
__device__ __forceinline__ float sigmoid_f(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_f(float z) { return z * sigmoid_f(z); }
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = sigmoid_f(z);
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

/* Copies one 128 x 32 operand tile into shared memory.  kmajor = false:
 * global [row][k] (row = m or n), shared [128][32+PAD]; kmajor = true:
 * global [k][row], shared [32][128+PAD]. */
template <bool KMAJOR>
__device__ __forceinline__ void load_tile(__nv_bfloat16* s, const __nv_bfloat16* g, long long ld,
                                          int row0, int k0) {
    const int t = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int c = t + q * kThreads; /* 512 chunks of 8 elements */
        if (!KMAJOR) {
            const int r = c >> 2, kc = (c & 3) * 8;
            cp_async16(s + r * (BK + PAD) + kc, g + (long long)(row0 + r) * ld + k0 + kc);
        } else {
            const int k = c >> 4, rc = (c & 15) * 8;
            cp_async16(s + k * (BM + PAD) + rc, g + (long long)(k0 + k) * ld + row0 + rc);
        }
    }
}

template <bool AK, bool BKM, int EPI>
__global__ void __launch_bounds__(kThreads) gemm_kernel(GemmArgs a) {
    __shared__ __align__(128) __nv_bfloat16 sA[2][kTileElems];
    __shared__ __align__(128) __nv_bfloat16 sB[2][kTileElems];
    const int mem = blockIdx.z;
    const __nv_bfloat16* A = a.A + mem * a.sA;
    const __nv_bfloat16* B = a.B + mem * a.sB;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;

    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;

    const int nk = a.K / BK;
    load_tile<AK>(sA[0], A, a.lda, m0, 0);
    load_tile<BKM>(sB[0], B, a.ldb, n0, 0);
    cp_async_commit();
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) {
            load_tile<AK>(sA[st ^ 1], A, a.lda, m0, (kt + 1) * BK);
            load_tile<BKM>(sB[st ^ 1], B, a.ldb, n0, (kt + 1) * BK);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const __nv_bfloat16* tA = sA[st];
        const __nv_bfloat16* tB = sB[st];
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[4][4];
            const int j = lane >> 3, r = lane & 7;
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const int mb = wm + mi * 16;
                if (!AK) {
                    ldsm_x4(af[mi], tA + (mb + (lane & 15)) * (BK + PAD) + kk + (lane >> 4) * 8);
                } else {
                    ldsm_x4_t(af[mi], tA + (kk + (j >> 1) * 8 + r) * (BM + PAD) + mb + (j & 1) * 8);
                }
            }
            uint32_t bf[4][2];
#pragma unroll
            for (int ni = 0; ni < 4; ni += 2) {
                const int nb = wn + ni * 8;
                uint32_t t4[4];
                if (!BKM) {
                    ldsm_x4(t4, tB + (nb + (j >> 1) * 8 + r) * (BK + PAD) + kk + (j & 1) * 8);
                } else {
                    ldsm_x4_t(t4, tB + (kk + (j & 1) * 8 + r) * (BN + PAD) + nb + (j >> 1) * 8);
                }
                bf[ni][0] = t4[0];
                bf[ni][1] = t4[1];
                bf[ni + 1][0] = t4[2];
                bf[ni + 1][1] = t4[3];
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bf[ni][0], bf[ni][1]);
        }
        __syncthreads();
    }

    /* epilogue: thread holds rows g, g+8 and columns 2q, 2q+1 of each 16 x 8 tile */
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm + mi * 16 + g + 8 * h;
                const int col = n0 + wn + ni * 8 + 2 * q;
                const float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
                if (EPI == EPI_FWD) {
                    const float* bias = a.bias + mem * a.sBias;
                    const float z0 = v0 + bias[col], z1 = v1 + bias[col + 1];
                    const long long o = mem * a.sZ + (long long)row * a.ldz + col;
                    if (a.Z) *reinterpret_cast<float2*>(a.Z + o) = make_float2(z0, z1);
                    *reinterpret_cast<__nv_bfloat162*>(a.Hout + o) =
                        __floats2bfloat162_rn(silu_f(z0), silu_f(z1));
                } else if (EPI == EPI_BWD) {
                    const long long o = mem * a.sZ + (long long)row * a.ldz + col;
                    const float2 z = *reinterpret_cast<const float2*>(a.Zin + o);
                    *reinterpret_cast<__nv_bfloat162*>(a.Dout + o) =
                        __floats2bfloat162_rn(v0 * silu_grad_f(z.x), v1 * silu_grad_f(z.y));
                } else {
                    const long long o = mem * a.sC + (long long)row * a.ldc + col;
                    *reinterpret_cast<float2*>(a.C + o) = make_float2(v0, v1);
                }
            }
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

int launch_gemm(const GemmArgs& a, bool a_kmajor, bool b_kmajor, int epi, int members,
                void* stream) {
    const dim3 grid(a.N / BN, a.M / BM, members);
    cudaStream_t s = (cudaStream_t)stream;
    if (!a_kmajor && !b_kmajor && epi == EPI_FWD)
        gemm_kernel<false, false, EPI_FWD><<<grid, kThreads, 0, s>>>(a);
    else if (!a_kmajor && b_kmajor && epi == EPI_BWD)
        gemm_kernel<false, true, EPI_BWD><<<grid, kThreads, 0, s>>>(a);
    else if (a_kmajor && b_kmajor && epi == EPI_F32)
        gemm_kernel<true, true, EPI_F32><<<grid, kThreads, 0, s>>>(a);
    else if (!a_kmajor && !b_kmajor && epi == EPI_F32)
        gemm_kernel<false, false, EPI_F32><<<grid, kThreads, 0, s>>>(a);
    else
        return (int)cudaErrorInvalidValue;
    return ok_or(cudaGetLastError());
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
