/*
 * bte_sur_host.cpp -- host side of the surrogate ABI (include/bte_surrogate.h):
 * device buffers of the ensemble, the launch sequence of one training step
 * and of inference, and the surrogate-with-solver-fallback routine.  All
 * arithmetic runs in the kernels of bte_sur_kernels.cu (and, for fallback
 * points, in the batched solver).
 */
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/bte_surrogate.h"
#include "bte_internal.h"
#include "bte_sur_internal.h"

using bte::sur::kIn;
using bte::sur::kOut;
typedef __nv_bfloat16 bf16;

struct bte_sur {
    int M, H, cap;
    bte::sur::ParamOffsets off;
    long long pstride;
    bte::sur::Scale sc;
    cudaStream_t stream;
    bool own_stream;
    unsigned char* mem;
    float *p, *g, *m, *v;
    bf16* wb;
    bf16* wti; /* W2, W3 in the tensor cores' canonical layout (inference) */
    int* err;
    float *Z1, *Z2, *Z3, *DY, *Yh, *partial;
    bf16 *H1, *H2, *H3, *DZ1, *DZ2, *DZ3;
    double* loss;
    int* idx;
    float *xd, *yd;
    long long nd;
    long long t; /* Adam steps taken */
    /* host-array inference: two buffer sets, so that the copies of one
     * chunk overlap the inference of the other, on two copy streams */
    float *xin[2], *mean_d[2], *std_d[2];
    unsigned char* mask_d[2];
    cudaStream_t cs_in, cs_out;
    cudaEvent_t ev_in[2], ev_comp[2], ev_out[2];
    bool pipe_ready;
};

namespace {

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return bte::report_error(code, buf);
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(BTE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

#define KL(call)                                                                         \
    do {                                                                                 \
        int r_ = (call);                                                                 \
        if (r_) return fail(BTE_ECUDA, "%s: %s", #call, cudaGetErrorString((cudaError_t)r_)); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

const double kTwoPi = 6.283185307179586476925286766559;

/* Forward pass of every member over rows [0, Bp) of the activation buffers;
 * Z buffers are written only when `train`. */
int forward(bte_sur* h, const float* x, const int* idx, long long row0, int nvalid, int Bp,
            bool train) {
    const int H = h->H;
    bte::sur::L1Args l1{};
    l1.x = x;
    l1.idx = idx;
    l1.row0 = row0;
    l1.nvalid = nvalid;
    l1.Bp = Bp;
    l1.H = H;
    l1.params = h->p;
    l1.pstride = h->pstride;
    l1.oW1 = h->off.W1;
    l1.ob1 = h->off.b1;
    l1.Z1 = train ? h->Z1 : nullptr;
    l1.H1 = h->H1;
    l1.sc = h->sc;
    /* activations are [member][Bp][H] for the current batch */
    KL(bte::sur::launch_l1(l1, h->M, h->stream));
    for (int layer = 0; layer < 2; ++layer) {
        bte::sur::GemmArgs a{};
        a.A = layer == 0 ? h->H1 : h->H2;
        a.lda = H;
        a.sA = (long long)Bp * H;
        a.B = h->wb + (long long)layer * H * H;
        a.ldb = H;
        a.sB = 2ll * H * H;
        a.M = Bp;
        a.N = H;
        a.K = H;
        a.bias = h->p + (layer == 0 ? h->off.b2 : h->off.b3);
        a.sBias = h->pstride;
        a.Z = train ? (layer == 0 ? h->Z2 : h->Z3) : nullptr;
        a.Hout = layer == 0 ? h->H2 : h->H3;
        a.ldz = H;
        a.sZ = (long long)Bp * H;
        a.err = h->err;
        KL(bte::sur::launch_gemm(a, false, false, bte::sur::EPI_FWD, h->M, h->stream));
    }
    return BTE_OK;
}

/* Loss, gradients into h->g; forward must have run with train = true. */
int backward(bte_sur* h, const float* x, const float* y, const int* idx, long long row0,
             int nvalid, int Bp) {
    const int H = h->H;
    const long long sAct = (long long)Bp * H;
    bte::sur::HeadArgs hd{};
    hd.H3 = h->H3;
    hd.Z3 = h->Z3;
    hd.params = h->p;
    hd.pstride = h->pstride;
    hd.oW4 = h->off.W4;
    hd.ob4 = h->off.b4;
    hd.Bp = Bp;
    hd.H = H;
    hd.nvalid = nvalid;
    hd.Yh = nullptr;
    hd.y = y;
    hd.idx = idx;
    hd.row0 = row0;
    hd.inv_n = 1.0f / (float)nvalid;
    hd.DY = h->DY;
    hd.DZ3 = h->DZ3;
    hd.loss = h->loss;
    hd.sc = h->sc;
    KL(bte::sur::launch_head(hd, h->M, h->stream));
    /* layers 3 and 2: weight gradient dZ^T H_prev, then dZ_prev = (dZ W) * silu'(Z_prev) */
    for (int layer = 1; layer >= 0; --layer) {
        const bf16* dZ = layer == 1 ? h->DZ3 : h->DZ2;
        const bf16* Hprev = layer == 1 ? h->H2 : h->H1;
        bte::sur::GemmArgs gw{};
        gw.A = dZ;
        gw.lda = H;
        gw.sA = sAct;
        gw.B = Hprev;
        gw.ldb = H;
        gw.sB = sAct;
        gw.M = H;
        gw.N = H;
        gw.K = Bp;
        gw.C = h->g + (layer == 1 ? h->off.W3 : h->off.W2);
        gw.ldc = H;
        gw.sC = h->pstride;
        gw.err = h->err;
        KL(bte::sur::launch_gemm(gw, true, true, bte::sur::EPI_F32, h->M, h->stream));
        bte::sur::GemmArgs dh{};
        dh.A = dZ;
        dh.lda = H;
        dh.sA = sAct;
        dh.B = h->wb + (long long)layer * H * H;
        dh.ldb = H;
        dh.sB = 2ll * H * H;
        dh.M = Bp;
        dh.N = H;
        dh.K = H;
        dh.Zin = layer == 1 ? h->Z2 : h->Z1;
        dh.Dout = layer == 1 ? h->DZ2 : h->DZ1;
        dh.ldz = H;
        dh.sZ = sAct;
        dh.err = h->err;
        KL(bte::sur::launch_gemm(dh, false, true, bte::sur::EPI_BWD, h->M, h->stream));
    }
    bte::sur::RedArgs r{};
    r.DZ1 = h->DZ1;
    r.DZ2 = h->DZ2;
    r.DZ3 = h->DZ3;
    r.H3 = h->H3;
    r.DY = h->DY;
    r.x = x;
    r.idx = idx;
    r.row0 = row0;
    r.nvalid = nvalid;
    r.Bp = Bp;
    r.H = H;
    r.partial = h->partial;
    r.grad = h->g;
    r.pstride = h->pstride;
    r.off = h->off;
    r.sc = h->sc;
    KL(bte::sur::launch_reduce(r, h->M, h->stream));
    return BTE_OK;
}

bte::sur::AdamArgs adam_args(bte_sur* h) {
    bte::sur::AdamArgs a{};
    a.p = h->p;
    a.g = h->g;
    a.m = h->m;
    a.v = h->v;
    a.wb = h->wb;
    a.pstride = h->pstride;
    a.count = h->off.count;
    a.oW2 = h->off.W2;
    a.oW3 = h->off.W3;
    a.H = h->H;
    a.members = h->M;
    a.beta1 = 0.9f;
    a.beta2 = 0.999f;
    a.eps = 1e-8f;
    return a;
}

int round128(long long n) { return (int)((n + 127) / 128 * 128); }

int predict_chunks(bte_sur* h, const float* x_dev, long long n, float* mean, float* stdv,
                   unsigned char* mask, double threshold) {
    KL(bte::sur::launch_canon_weights(h->p, h->pstride, h->off, h->wti, h->M, h->stream));
    for (long long r0 = 0; r0 < n; r0 += h->cap) {
        const int rows = (int)std::min<long long>(h->cap, n - r0);
        const int Bp = round128(rows);
        bte::sur::InferArgs ia{};
        ia.x = x_dev;
        ia.row0 = r0;
        ia.nvalid = rows;
        ia.Bp = Bp;
        ia.params = h->p;
        ia.pstride = h->pstride;
        ia.off = h->off;
        ia.wb = h->wb;
        ia.wti = h->wti;
        ia.Yh = h->Yh;
        ia.err = h->err;
        ia.sc = h->sc;
        KL(bte::sur::launch_infer_tc(ia, h->M, h->stream));
        bte::sur::EnsArgs e{};
        e.Yh = h->Yh;
        e.members = h->M;
        e.Bp = Bp;
        e.n = rows;
        e.mean = mean + r0 * kOut;
        e.stdv = stdv + r0 * kOut;
        e.mask = mask ? mask + r0 : nullptr;
        e.threshold = (float)threshold;
        e.sc = h->sc;
        KL(bte::sur::launch_ensemble(e, h->stream));
    }
    return BTE_OK;
}

/* copy streams and events of the host-array inference, made on first use */
int make_pipe(bte_sur* h) {
    CU(cudaStreamCreateWithFlags(&h->cs_in, cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&h->cs_out, cudaStreamNonBlocking));
    for (int s = 0; s < 2; ++s) {
        CU(cudaEventCreateWithFlags(&h->ev_in[s], cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&h->ev_comp[s], cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&h->ev_out[s], cudaEventDisableTiming));
    }
    h->pipe_ready = true;
    return BTE_OK;
}

}  // namespace

extern "C" {

int bte_sur_create(const bte_sur_config* cfg, bte_sur** out) {
    if (!cfg || !out) return fail(BTE_EINVAL, "NULL argument");
    *out = nullptr;
    const int M = cfg->members ? cfg->members : 8;
    const int H = cfg->width ? cfg->width : 256;
    const int cap = cfg->batch_capacity ? cfg->batch_capacity : 16384;
    if (M < 1 || M > 64) return fail(BTE_EINVAL, "members must be 1..64");
    if (H != 256) return fail(BTE_EINVAL, "only width 256 is supported");
    if (cap < 128 || cap % 128 || cap > (1 << 22))
        return fail(BTE_EINVAL, "batch_capacity must be a multiple of 128 in 128..4194304");
    if (cfg->reserved) return fail(BTE_EINVAL, "reserved field must be 0");
    bte::sur::Scale sc{};
    for (int i = 0; i < kIn; ++i) {
        if (!std::isfinite(cfg->x_lo[i]) || !std::isfinite(cfg->x_hi[i]) || !(cfg->x_hi[i] > cfg->x_lo[i]))
            return fail(BTE_EINVAL, "input box dimension %d is empty or not finite", i);
        sc.x_lo[i] = (float)cfg->x_lo[i];
        sc.x_inv[i] = (float)(1.0 / (cfg->x_hi[i] - cfg->x_lo[i]));
    }
    for (int o = 0; o < kOut; ++o) {
        if (!std::isfinite(cfg->y_mean[o]) || !std::isfinite(cfg->y_std[o]) || !(cfg->y_std[o] > 0))
            return fail(BTE_EINVAL, "output scaling %d must be finite with y_std > 0", o);
        sc.y_mean[o] = (float)cfg->y_mean[o];
        sc.y_std[o] = (float)cfg->y_std[o];
    }
    bte_sur* h = new (std::nothrow) bte_sur();
    if (!h) return fail(BTE_ENOMEM, "host allocation failed");
    h->M = M;
    h->H = H;
    h->cap = cap;
    h->off = bte::sur::param_offsets(H);
    h->pstride = (long long)align_up((size_t)h->off.count, 8);
    h->sc = sc;
    /* one allocation: parameters, gradients, moments, BF16 weights,
     * activations, reduction scratch, indices, inference buffers */
    const size_t P = (size_t)h->pstride * M * 4;
    const size_t act32 = (size_t)M * cap * H * 4, act16 = (size_t)M * cap * H * 2;
    const size_t nred = (size_t)bte::sur::reduce_count(H);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align_up(bytes, 256);
        return at;
    };
    const size_t op = take(P), og = take(P), om = take(P), ov = take(P);
    const size_t owb = take((size_t)M * 2 * H * H * 2);
    const size_t owti = take((size_t)M * 2 * H * H * 2);
    const size_t oerr = take(256);
    const size_t oz1 = take(act32), oz2 = take(act32), oz3 = take(act32);
    const size_t oh1 = take(act16), oh2 = take(act16), oh3 = take(act16);
    const size_t od1 = take(act16), od2 = take(act16), od3 = take(act16);
    const size_t ody = take((size_t)M * cap * kOut * 4), oyh = take((size_t)M * cap * kOut * 4);
    const size_t opart = take((size_t)M * (cap / 128) * nred * 4);
    const size_t oloss = take((size_t)M * 8);
    const size_t oidx = take((size_t)M * cap * 4);
    size_t oxin[2], omean[2], ostd[2], omask[2];
    for (int s = 0; s < 2; ++s) {
        oxin[s] = take((size_t)cap * kIn * 4);
        omean[s] = take((size_t)cap * kOut * 4);
        ostd[s] = take((size_t)cap * kOut * 4);
        omask[s] = take((size_t)cap);
    }
    cudaError_t e = cudaMalloc(&h->mem, o);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(BTE_ENOMEM, "surrogate workspace of %zu bytes: %s", o, cudaGetErrorString(e));
    }
    unsigned char* b = h->mem;
    h->p = (float*)(b + op);
    h->g = (float*)(b + og);
    h->m = (float*)(b + om);
    h->v = (float*)(b + ov);
    h->wb = (bf16*)(b + owb);
    h->wti = (bf16*)(b + owti);
    h->err = (int*)(b + oerr);
    h->Z1 = (float*)(b + oz1);
    h->Z2 = (float*)(b + oz2);
    h->Z3 = (float*)(b + oz3);
    h->H1 = (bf16*)(b + oh1);
    h->H2 = (bf16*)(b + oh2);
    h->H3 = (bf16*)(b + oh3);
    h->DZ1 = (bf16*)(b + od1);
    h->DZ2 = (bf16*)(b + od2);
    h->DZ3 = (bf16*)(b + od3);
    h->DY = (float*)(b + ody);
    h->Yh = (float*)(b + oyh);
    h->partial = (float*)(b + opart);
    h->loss = (double*)(b + oloss);
    h->idx = (int*)(b + oidx);
    for (int s = 0; s < 2; ++s) {
        h->xin[s] = (float*)(b + oxin[s]);
        h->mean_d[s] = (float*)(b + omean[s]);
        h->std_d[s] = (float*)(b + ostd[s]);
        h->mask_d[s] = (unsigned char*)(b + omask[s]);
    }
    if (cfg->stream) {
        h->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaFree(h->mem);
            delete h;
            return fail(BTE_ECUDA, "cudaStreamCreate failed");
        }
        h->own_stream = true;
    }
    if (cudaMemsetAsync(h->mem, 0, o, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        bte_sur_destroy(h);
        return fail(BTE_ECUDA, "workspace clear failed");
    }
    *out = h;
    return BTE_OK;
}

int64_t bte_sur_param_count(const bte_sur* h) { return h ? h->off.count : 0; }

int bte_sur_set_params(bte_sur* h, const float* p) {
    if (!h || !p) return fail(BTE_EINVAL, "NULL argument");
    for (long long i = 0; i < (long long)h->M * h->off.count; ++i)
        if (!std::isfinite(p[i])) return fail(BTE_EINVAL, "non-finite parameter at %lld", i);
    for (int m = 0; m < h->M; ++m)
        CU(cudaMemcpyAsync(h->p + m * h->pstride, p + (long long)m * h->off.count,
                           h->off.count * 4, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemsetAsync(h->m, 0, (size_t)h->pstride * h->M * 4, h->stream));
    CU(cudaMemsetAsync(h->v, 0, (size_t)h->pstride * h->M * 4, h->stream));
    h->t = 0;
    KL(bte::sur::launch_refresh_bf16(adam_args(h), h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return BTE_OK;
}

int bte_sur_get_params(bte_sur* h, float* p) {
    if (!h || !p) return fail(BTE_EINVAL, "NULL argument");
    for (int m = 0; m < h->M; ++m)
        CU(cudaMemcpyAsync(p + (long long)m * h->off.count, h->p + m * h->pstride,
                           h->off.count * 4, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return BTE_OK;
}

int bte_sur_set_data(bte_sur* h, const float* x, const float* y, int64_t n) {
    if (!h || !x || !y || n < 1 || n > (1ll << 31)) return fail(BTE_EINVAL, "bad training set");
    if (h->xd) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->xd);
        h->xd = h->yd = nullptr;
        h->nd = 0;
    }
    unsigned char* d = nullptr;
    const size_t bx = align_up((size_t)n * kIn * 4, 256), by = (size_t)n * kOut * 4;
    if (cudaMalloc(&d, bx + by) != cudaSuccess) {
        cudaGetLastError();
        return fail(BTE_ENOMEM, "training set of %lld points", (long long)n);
    }
    h->xd = (float*)d;
    h->yd = (float*)(d + bx);
    h->nd = n;
    CU(cudaMemcpyAsync(h->xd, x, (size_t)n * kIn * 4, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->yd, y, (size_t)n * kOut * 4, cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return BTE_OK;
}

int bte_sur_train(bte_sur* h, const int32_t* order, int32_t steps, int32_t batch, const float* lr,
                  double* loss) {
    if (!h || !order || !lr || steps < 0) return fail(BTE_EINVAL, "bad argument");
    if (!h->xd) return fail(BTE_ESTATE, "no training set uploaded");
    if (batch < 1 || batch > h->cap) return fail(BTE_EINVAL, "batch must be 1..%d", h->cap);
    const long long per = (long long)h->M * batch;
    for (long long i = 0; i < per * steps; ++i)
        if (order[i] < 0 || order[i] >= h->nd) return fail(BTE_EINVAL, "order[%lld] out of range", i);
    for (int s = 0; s < steps; ++s)
        if (!(lr[s] >= 0) || !std::isfinite(lr[s])) return fail(BTE_EINVAL, "bad learning rate");
    const int Bp = round128(batch);
    std::vector<int> idx((size_t)h->M * Bp, 0);
    std::vector<double> lh(h->M);
    for (int s = 0; s < steps; ++s) {
        for (int m = 0; m < h->M; ++m)
            std::memcpy(&idx[(size_t)m * Bp], order + (s * per + (long long)m * batch), batch * 4);
        /* the copy reads `idx` before the next iteration rewrites it: the
         * stream is synchronised at the end of every step below */
        CU(cudaMemcpyAsync(h->idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, h->stream));
        CU(cudaMemsetAsync(h->loss, 0, h->M * 8, h->stream));
        int rc = forward(h, h->xd, h->idx, 0, batch, Bp, true);
        if (!rc) rc = backward(h, h->xd, h->yd, h->idx, 0, batch, Bp);
        if (rc) return rc;
        h->t += 1;
        bte::sur::AdamArgs a = adam_args(h);
        a.lr = lr[s];
        a.c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)h->t)));
        a.c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)h->t)));
        KL(bte::sur::launch_adam(a, h->stream));
        if (loss) CU(cudaMemcpyAsync(lh.data(), h->loss, h->M * 8, cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        if (loss)
            for (int m = 0; m < h->M; ++m) loss[(long long)s * h->M + m] = lh[m];
    }
    int err = 0;
    CU(cudaMemcpy(&err, h->err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) return fail(BTE_ETIMEOUT, "a bounded wait in a training GEMM gave up");
    return BTE_OK;
}

int bte_sur_grad(bte_sur* h, const float* x, const float* t, int32_t n, float* grad, double* loss) {
    if (!h || !x || !t || n < 1 || n > h->cap) return fail(BTE_EINVAL, "bad argument");
    const int Bp = round128(n);
    /* the inputs go through a temporary device copy */
    unsigned char* d = nullptr;
    const size_t bx = align_up((size_t)n * kIn * 4, 256);
    if (cudaMalloc(&d, bx + (size_t)n * kOut * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(BTE_ENOMEM, "device copy of %d points", n);
    }
    float* xd = (float*)d;
    float* td = (float*)(d + bx);
    int rc = BTE_OK;
    if (cudaMemcpyAsync(xd, x, (size_t)n * kIn * 4, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(td, t, (size_t)n * kOut * 4, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->loss, 0, h->M * 8, h->stream) != cudaSuccess)
        rc = fail(BTE_ECUDA, "upload failed");
    if (!rc) rc = forward(h, xd, nullptr, 0, n, Bp, true);
    if (!rc) rc = backward(h, xd, td, nullptr, 0, n, Bp);
    if (!rc && grad)
        for (int m = 0; m < h->M && !rc; ++m)
            if (cudaMemcpyAsync(grad + (long long)m * h->off.count, h->g + m * h->pstride,
                                h->off.count * 4, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
                rc = fail(BTE_ECUDA, "gradient copy failed");
    if (!rc && loss &&
        cudaMemcpyAsync(loss, h->loss, h->M * 8, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        rc = fail(BTE_ECUDA, "loss copy failed");
    if (cudaStreamSynchronize(h->stream) != cudaSuccess && !rc) rc = fail(BTE_ECUDA, "sync failed");
    cudaFree(d);
    int err = 0;
    if (!rc && cudaMemcpy(&err, h->err, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = fail(BTE_ECUDA, "error word read failed");
    if (!rc && err) rc = fail(BTE_ETIMEOUT, "a bounded wait in a training GEMM gave up");
    return rc;
}

int bte_sur_predict_device(bte_sur* h, const float* x, int64_t n, float* mean, float* stdv,
                           uint8_t* mask, double threshold) {
    if (!h || !x || !mean || !stdv || n < 0) return fail(BTE_EINVAL, "bad argument");
    return predict_chunks(h, x, n, mean, stdv, mask, threshold);
}

int bte_sur_predict(bte_sur* h, const float* x, int64_t n, float* mean, float* stdv, uint8_t* mask,
                    double threshold) {
    if (!h || !x || !mean || !stdv || n < 0) return fail(BTE_EINVAL, "bad argument");
    if (n == 0) return BTE_OK;
    if (!h->pipe_ready) {
        int rc = make_pipe(h);
        if (rc) return rc;
    }
    /* chunk i uses buffer set i & 1: its input copy waits until the
     * inference of chunk i-2 has read that set, its inference waits for its
     * input and for the output copies of chunk i-2, its output copies wait
     * for its inference (stream order does the rest) */
    long long i = 0;
    for (long long r0 = 0; r0 < n; r0 += h->cap, ++i) {
        const int s = (int)(i & 1);
        const long long rows = std::min<long long>(h->cap, n - r0);
        if (i >= 2) CU(cudaStreamWaitEvent(h->cs_in, h->ev_comp[s], 0));
        CU(cudaMemcpyAsync(h->xin[s], x + r0 * kIn, rows * kIn * 4, cudaMemcpyHostToDevice, h->cs_in));
        CU(cudaEventRecord(h->ev_in[s], h->cs_in));
        CU(cudaStreamWaitEvent(h->stream, h->ev_in[s], 0));
        if (i >= 2) CU(cudaStreamWaitEvent(h->stream, h->ev_out[s], 0));
        int rc = predict_chunks(h, h->xin[s], rows, h->mean_d[s], h->std_d[s],
                                mask ? h->mask_d[s] : nullptr, threshold);
        if (rc) {
            cudaStreamSynchronize(h->cs_in);
            cudaStreamSynchronize(h->stream);
            cudaStreamSynchronize(h->cs_out);
            return rc;
        }
        CU(cudaEventRecord(h->ev_comp[s], h->stream));
        CU(cudaStreamWaitEvent(h->cs_out, h->ev_comp[s], 0));
        CU(cudaMemcpyAsync(mean + r0 * kOut, h->mean_d[s], rows * kOut * 4, cudaMemcpyDeviceToHost, h->cs_out));
        CU(cudaMemcpyAsync(stdv + r0 * kOut, h->std_d[s], rows * kOut * 4, cudaMemcpyDeviceToHost, h->cs_out));
        if (mask) CU(cudaMemcpyAsync(mask + r0, h->mask_d[s], rows, cudaMemcpyDeviceToHost, h->cs_out));
        CU(cudaEventRecord(h->ev_out[s], h->cs_out));
    }
    CU(cudaStreamSynchronize(h->cs_out));
    CU(cudaStreamSynchronize(h->stream));
    int err = 0;
    CU(cudaMemcpy(&err, h->err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) return fail(BTE_ETIMEOUT, "a bounded wait in the inference kernel gave up");
    return BTE_OK;
}

int bte_sur_protocol(const double* x, int32_t precision, bte_params* out) {
    if (!x || !out) return fail(BTE_EINVAL, "NULL argument");
    const double E_dc = x[0], E_omega = x[1], omega = x[2], B = x[3], mu = x[4];
    for (int i = 0; i < kIn; ++i)
        if (!std::isfinite(x[i])) return fail(BTE_EINVAL, "non-finite input");
    if (!(omega > 0) || !(mu > 0)) return fail(BTE_EINVAL, "omega and mu must be > 0");
    const double L = 7.0 / std::sqrt(mu) + 1.5 * B;
    if (!(L > 0)) return fail(BTE_EINVAL, "empty phi_y range");
    const double mp = 2.0 * std::ceil(L / 0.02) + 1.0;
    const double nm = std::ceil(12.0 + 3.0 * mu + 10.0 * B);
    std::memset(out, 0, sizeof *out);
    out->E_dc = E_dc;
    out->E_omega = E_omega;
    out->omega = omega;
    out->B = B;
    out->mu = mu;
    out->alpha = 1.0;
    out->phiy_min = -L;
    out->phiy_max = L;
    out->dt = 1e-3;
    out->periods = std::ceil(16.0 * omega / kTwoPi) + 1.0;
    out->t_max = 0.0;
    out->avg_window = 1.0;
    out->n_max = (int32_t)std::min(std::max(nm, 20.0), 200.0);
    out->m_points = (int32_t)std::min(std::max(mp, 201.0), 2001.0);
    out->precision = precision;
    out->reserved = 0;
    return BTE_OK;
}

int bte_sur_hybrid(bte_sur* h, const double* x, int64_t n, double threshold, int32_t precision,
                   const bte_batch_opts* opts, double* y, uint8_t* solved, int32_t* status) {
    if (!h || !x || !y || n < 0) return fail(BTE_EINVAL, "bad argument");
    if (n == 0) return BTE_OK;
    std::vector<float> xf((size_t)n * kIn), mean((size_t)n * kOut), sd((size_t)n * kOut);
    std::vector<uint8_t> mask(n);
    for (long long i = 0; i < n * kIn; ++i) xf[i] = (float)x[i];
    int rc = bte_sur_predict(h, xf.data(), n, mean.data(), sd.data(), mask.data(), threshold);
    if (rc) return rc;
    std::vector<bte_params> pts;
    std::vector<long long> where;
    for (long long i = 0; i < n; ++i) {
        y[i * kOut] = mean[i * kOut];
        y[i * kOut + 1] = mean[i * kOut + 1];
        if (solved) solved[i] = mask[i];
        if (status) status[i] = BTE_OK;
        if (mask[i]) {
            bte_params p;
            rc = bte_sur_protocol(x + i * kIn, precision, &p);
            if (rc) return fail(rc, "point %lld: %s", i, bte_last_error());
            pts.push_back(p);
            where.push_back(i);
        }
    }
    if (pts.empty()) return BTE_OK;
    std::vector<bte_obs> res(pts.size());
    rc = bte_batch_run(pts.data(), (int32_t)pts.size(), res.data(), opts);
    if (rc == BTE_EINVAL || rc == BTE_ENOMEM || rc == BTE_ECUDA) return rc;
    for (size_t k = 0; k < pts.size(); ++k) {
        const long long i = where[k];
        y[i * kOut] = res[k].absorption;
        y[i * kOut + 1] = res[k].v_dc_avg;
        if (status) status[i] = res[k].status;
    }
    return rc;
}

void bte_sur_destroy(bte_sur* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (cudaStream_t* cs : {&h->cs_in, &h->cs_out})
        if (*cs) {
            cudaStreamSynchronize(*cs);
            cudaStreamDestroy(*cs);
        }
    for (int s = 0; s < 2; ++s)
        for (cudaEvent_t ev : {h->ev_in[s], h->ev_comp[s], h->ev_out[s]})
            if (ev) cudaEventDestroy(ev);
    if (h->xd) cudaFree(h->xd);
    if (h->mem) cudaFree(h->mem);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
