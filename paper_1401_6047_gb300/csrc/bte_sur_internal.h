/*
 * bte_sur_internal.h -- structures shared by the surrogate's host code and
 * its CUDA kernels.  Not part of the public ABI.
 *
 * Device layout of one ensemble (M members, hidden width H, 5 inputs, 2
 * outputs).  Parameters of a member are packed as W1 [H][5], b1 [H],
 * W2 [H][H], b2 [H], W3 [H][H], b3 [H], W4 [2][H], b4 [2]; members sit
 * `pstride` floats apart (pstride = the packed count rounded up to 8 so
 * every member starts on a 32-byte boundary).  BF16 copies of W2 and W3
 * (the tensor-core operands) sit in `wb` as [M][2][H][H].  Activations of a
 * batch of Bp samples (Bp a multiple of 128) are [M][Bp][H], row-major.
 */
#pragma once
#include <cuda_bf16.h>

#include <cstddef>
#include <cstdint>

namespace bte {
namespace sur {

constexpr int kIn = 5;
constexpr int kOut = 2;

/* Offsets of the parameter tensors inside one packed member. */
struct ParamOffsets {
    long long W1, b1, W2, b2, W3, b3, W4, b4, count;
};

inline ParamOffsets param_offsets(int H) {
    ParamOffsets o;
    long long q = 0;
    o.W1 = q; q += (long long)H * kIn;
    o.b1 = q; q += H;
    o.W2 = q; q += (long long)H * H;
    o.b2 = q; q += H;
    o.W3 = q; q += (long long)H * H;
    o.b3 = q; q += H;
    o.W4 = q; q += (long long)kOut * H;
    o.b4 = q; q += kOut;
    o.count = q;
    return o;
}

/* Input normalisation and output scaling shared by the kernels. */
struct Scale {
    float x_lo[kIn], x_inv[kIn]; /* xh = 2 (x - lo) * inv - 1, inv = 1/(hi - lo) */
    float y_mean[kOut], y_std[kOut];
};

enum Epi { EPI_FWD = 0, EPI_BWD = 1, EPI_F32 = 2 };

/* C[M][N] = sum_k A(m, k) B(k, n) per member (blockIdx.z), BF16 operands,
 * FP32 accumulation, then one epilogue:
 *   EPI_FWD: z = acc + bias[n]; Z[m][n] = z (if Z), Hout[m][n] = bf16(silu(z))
 *   EPI_BWD: Dout[m][n] = bf16(acc * silu'(Zin[m][n]))
 *   EPI_F32: C[m][n] = acc
 * A is stored [m][k] (a_kmajor = false) or [k][m]; B is stored [n][k]
 * (b_kmajor = false) or [k][n].  M, N multiples of 128; K of 64; every
 * leading dimension a multiple of 8 elements, bases 16-byte aligned. */
struct GemmArgs {
    const __nv_bfloat16* A;
    long long lda, sA;
    const __nv_bfloat16* B;
    long long ldb, sB;
    int M, N, K;
    const float* bias;
    long long sBias;
    float* Z;
    __nv_bfloat16* Hout;
    const float* Zin;
    __nv_bfloat16* Dout;
    long long ldz, sZ; /* leading dimension / member stride of Z, Hout, Zin, Dout */
    float* C;
    long long ldc, sC;
    int* err; /* set to 1 when a bounded wait gives up (may be null) */
};

/* Layer 1 (K = 5, FP32 FMAs): Z1 = W1 xh + b1, H1 = bf16(silu(Z1)), for
 * rows r < Bp; sample of row r is idx[r] (or row0 + r when idx is null);
 * rows r >= nvalid use xh = 0. */
struct L1Args {
    const float* x; /* [n][5] raw inputs */
    const int* idx; /* [M][Bp] per-member sample indices, or null */
    long long row0;
    int nvalid, Bp, H;
    const float* params;
    long long pstride;
    long long oW1, ob1;
    float* Z1;       /* may be null (inference) */
    __nv_bfloat16* H1;
    Scale sc;
};

/* Output layer (N = 2, FP32 FMAs, one warp per sample).  Inference writes
 * Yh [M][Bp][2].  Training also reads the targets, writes DY = (yh - th)/n
 * [M][Bp][2] and DZ3 = (DY W4) * silu'(Z3) as BF16, and adds the loss of
 * each member into loss[m] (FP64). */
struct HeadArgs {
    const __nv_bfloat16* H3;
    const float* Z3;
    const float* params;
    long long pstride, oW4, ob4;
    int Bp, H, nvalid;
    float* Yh;
    /* training */
    const float* y;  /* [n][2] raw targets, or null (inference) */
    const int* idx;
    long long row0;
    float inv_n;
    float* DY;
    __nv_bfloat16* DZ3;
    double* loss;
    Scale sc;
};

/* Gradients that are reductions over the batch with one small side:
 * b1, W1 (from DZ1 and xh), b2, b3, W4, b4 (from DY and H3). Two passes in
 * a fixed order: per-128-sample partial sums, then their sum. */
struct RedArgs {
    const __nv_bfloat16 *DZ1, *DZ2, *DZ3, *H3;
    const float* DY;
    const float* x;
    const int* idx;
    long long row0;
    int nvalid, Bp, H;
    float* partial; /* [M][Bp/128][nred] */
    float* grad;    /* [M][pstride] */
    long long pstride;
    ParamOffsets off;
    Scale sc;
};

struct AdamArgs {
    float* p;
    float* g;
    float* m;
    float* v;
    __nv_bfloat16* wb; /* [M][2][H][H] BF16 copies of W2, W3 */
    long long pstride, count, oW2, oW3;
    int H, members;
    float lr, beta1, beta2, eps, c1, c2; /* c1 = 1/(1-beta1^t), c2 = 1/(1-beta2^t) */
};

/* Fused inference of every member (blockIdx.y) on 128 rows per CTA: the
 * 5-input layer, both 256 x 256 layers (tcgen05 tensor cores, activations
 * in shared memory, accumulators in tensor memory) and the 2-output layer;
 * writes Yh [M][Bp][2].  Rows r < nvalid read x[row0 + r]; H = 256. */
struct InferArgs {
    const float* x;
    long long row0;
    int nvalid, Bp;
    const float* params;
    long long pstride;
    ParamOffsets off;
    const __nv_bfloat16* wb;  /* [M][2][H][H] */
    const __nv_bfloat16* wti; /* W2, W3 in the tensor cores' canonical layout */
    float* Yh;
    int* err;                 /* set to 1 when a bounded wait gives up */
    Scale sc;
};

struct EnsArgs {
    const float* Yh; /* [M][Bp][2] */
    int members, Bp, n;
    float* mean;     /* [n][2] */
    float* stdv;     /* [n][2] */
    unsigned char* mask;
    float threshold;
    Scale sc;
};

int launch_gemm(const GemmArgs& a, bool a_kmajor, bool b_kmajor, int epi, int members,
                void* stream);
int launch_l1(const L1Args& a, int members, void* stream);
int launch_head(const HeadArgs& a, int members, void* stream);
int launch_reduce(const RedArgs& a, int members, void* stream);
int launch_adam(const AdamArgs& a, void* stream);
int launch_refresh_bf16(const AdamArgs& a, void* stream);
int launch_ensemble(const EnsArgs& a, void* stream);
/* tcgen05 inference (bte_sur_tc.cu) and the canonical-layout weight copy it reads */
int launch_infer_tc(const InferArgs& a, int members, void* stream);
int launch_canon_weights(const float* params, long long pstride, const ParamOffsets& off,
                         __nv_bfloat16* wti, int members, void* stream);
/* number of values each 128-sample block writes in the reduction */
int reduce_count(int H);

}  // namespace sur
}  // namespace bte
