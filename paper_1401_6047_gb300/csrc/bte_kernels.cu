/*
 * bte_kernels.cu -- the library's auxiliary kernels: initial state f = f0
 * (Sec. 2), the start-up half step z^{1/2} = T_{dt/2}(z^0; S(z^0)) (Sec. 3),
 * a plain reduction of rows 0 and 1 for one sample of the drift velocity and
 * norm, the step counter, and the FP64 window averages of Eq. absorption_def.
 * The per-step kernel lives in bte_step.cu.
 */
#include <cuda_runtime.h>

#include <cstdint>

#include "bte_device.cuh"
#include "bte_internal.h"

namespace bte {

namespace {

using namespace dev;

/* ---------------------------------------------------------------------- */
/* initial state, start-up half step, plain observables                  */
/* ---------------------------------------------------------------------- */
template <typename T>
__global__ void init_kernel(T* a_w, T* b_w, const T* row_a0, const T* col_g, int N, int M,
                            int pitch) {
    constexpr int G = Cols<T>::G;
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
    constexpr int G = Cols<T>::G;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (m > A.M || n > A.N) return;
    const int c = G + m;
    using O = Rn<T>;
    const T chi = (n == 1) ? (T)2 : (T)1;
    const T ph = A.col_phi[c];
    const T nf = (T)n;
    const T th = O::mul(nf, rot_factor<T>((T)A.E_start, (T)A.B_start, ph, A.hh));
    const T th1 = O::mul(nf, rot_factor<T>((T)A.E_end, (T)A.B_end, ph, A.hh));
    const int N = A.N, P = A.pitch;
    const T bu = ld_or0(A.bs, n + 1, c + 1, N, P) - ld_or0(A.bs, n + 1, c - 1, N, P);
    const T bd = (n - 1 >= 1) ? ld_or0(A.bs, n - 1, c + 1, N, P) - ld_or0(A.bs, n - 1, c - 1, N, P)
                              : (T)0;
    const T ad = ld_or0(A.as, n - 1, c + 1, N, P) - ld_or0(A.as, n - 1, c - 1, N, P);
    const T au = ld_or0(A.as, n + 1, c + 1, N, P) - ld_or0(A.as, n + 1, c - 1, N, P);
    const T Sa = stencil_a<T>(A.c, bu, bd);
    const T Sb = stencil_b<T>(A.c, chi, ad, au);
    const size_t g = (size_t)n * P + c;
    T an, bn;
    cn_cell<T>(A.a[g], A.b[g], Sa, Sb, O::mul(A.h, A.row_a0[n]), A.col_g[c], th, th1,
               cn_constants<T>(A.h, A.nu, A.xi), an, bn);
    if (n == 0) bn = (T)0;
    A.an[g] = an;
    A.bn[g] = bn;
}

template <typename T>
__global__ void observe_kernel(const T* a_w, const T* b_w, int M, int pitch, double vscale,
                               double nscale, double* trace_v, double* trace_n, long long slot) {
    constexpr int G = Cols<T>::G;
    __shared__ double red[32];
    double sn = 0, sv = 0;
    for (int m = threadIdx.x; m <= M; m += blockDim.x) {
        sn += (double)a_w[G + m];
        sv += (double)b_w[(size_t)pitch + G + m];
    }
    const double tn = block_sum(sn, red);
    const double tv = block_sum(sv, red);
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

/* f(phi_x_i, phi_y_m) = sum_n a_n(m) cos(n phi_x_i) + b_n(m) sin(n phi_x_i)
 * (Eq. f_fourier), phi_x_i = -pi + 2 pi i / nphix; one thread per (i, m),
 * cos / sin of n phi_x by the rotation recurrence, FP64 sums. */
template <typename T>
__global__ void pdf_kernel(const T* a, const T* b, int N, int M, int pitch, int nphix,
                           double* out) {
    constexpr int G = Cols<T>::G;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (m > M || i >= nphix) return;
    const double x = -3.14159265358979323846 + 6.28318530717958647692 * (double)i / (double)nphix;
    double s1, c1;
    sincos(x, &s1, &c1);
    double c = 1.0, s = 0.0, f = 0.0;
    for (int n = 0; n <= N; ++n) {
        const size_t q = (size_t)n * pitch + G + m;
        f += (double)a[q] * c + (double)b[q] * s;
        const double cn = c * c1 - s * s1;
        s = s * c1 + c * s1;
        c = cn;
    }
    out[(size_t)i * (M + 1) + m] = f;
}

/* The failure-detection path of the bounded waits, exercised without a
 * fault: one thread waits on a fresh mbarrier that no thread arrives on and
 * no copy completes, for limit_ns of %globaltimer, then records the timeout
 * in the error word as the solver kernels do.  Nothing is in flight when it
 * returns. */
__global__ void wait_probe_kernel(int* err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    if (!mbar_wait(b, 0u, limit_ns)) atomicExch(err, kErrTimeout);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b) : "memory");
}

}  // namespace

/* ---------------------------------------------------------------------- */
/* launchers                                                               */
/* ---------------------------------------------------------------------- */
static int ok_or(cudaError_t e) { return e == cudaSuccess ? 0 : (int)e; }

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

int launch_wait_probe(int* err, unsigned long long limit_ns, void* stream) {
    wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(err, limit_ns);
    return ok_or(cudaGetLastError());
}

int launch_finalize(const FinalArgs& a, void* stream) {
    finalize_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(a);
    return ok_or(cudaGetLastError());
}

template <typename T>
int launch_pdf(const T* a, const T* b, int N, int M, int pitch, int nphix, double* out,
               void* stream) {
    const dim3 grid((M + 1 + 127) / 128, nphix);
    pdf_kernel<T><<<grid, 128, 0, (cudaStream_t)stream>>>(a, b, N, M, pitch, nphix, out);
    return ok_or(cudaGetLastError());
}

#define BTE_INSTANTIATE(T)                                                                     \
    template int launch_init<T>(T*, T*, const T*, const T*, int, int, int, void*);             \
    template int launch_apply<T>(const ApplyArgs<T>&, void*);                                  \
    template int launch_observe<T>(const T*, const T*, int, int, double, double, double*,      \
                                   double*, long long, void*);                                 \
    template int launch_pdf<T>(const T*, const T*, int, int, int, int, double*, void*);
BTE_INSTANTIATE(float)
BTE_INSTANTIATE(double)

}  // namespace bte
