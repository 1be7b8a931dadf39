/*
 * bte_wide.cu -- single-instance solver on chip over several thread-block
 * clusters.
 *
 * The on-chip mode of bte_resident.cu holds a grid in one cluster: at most
 * 16 CTAs, so at most 16 SMs, and a small grid such as 31 x 201 leaves the
 * rest of the GPU idle (in FP64 the arithmetic of those 16 SMs is then the
 * limit).  Here the grid (harmonics n = 0..N by phi_y columns m = 0..M) is
 * cut into G column blocks of Wc columns and, inside each, C row blocks of
 * R rows: CTA r of cluster g keeps rows [r R, (r+1) R) of columns
 * [g Wc, (g+1) Wc) of the four arrays (a and b of the whole and of the
 * fractional grid, Sec. 3) in its shared memory for a whole bte_step /
 * bte_run call, with one halo row above and below and one halo column left
 * and right.  Each half-step of the leap-frog scheme (Eqs. leap_frog_1,
 * leap_frog_2) updates one grid in place from the other: the update of cell
 * (n, m) reads the other grid's rows n-1 and n+1 at columns m-1 and m+1 and
 * the cell's own values only.  As it makes them, a CTA writes
 *   - its first and last rows into the halo rows of the CTAs above and
 *     below it in its cluster (distributed shared memory, made visible by
 *     the split cluster barrier), and
 *   - its first and last columns into exchange words in global memory:
 *     8-byte words, each written and read as a whole, holding 32 bits of
 *     a value (FP64: two words) under the number of the half-step that
 *     made it, from which the CTAs of the neighbouring clusters fill their
 *     halo columns, polling each word until it carries the tag they expect.
 *     A value and its tag travel together, so the exchange needs no fence,
 *     no separate flag and no second load.
 * A CTA reads the columns of up to three CTAs on each side (the rows above
 * and below its own included: the corners of the stencil).  The words come
 * in two buffers (by the parity of the producing grid's update count), so
 * a word is rewritten four half-steps after it was written; by then the
 * writer has used columns that its readers made after reading it (the
 * readers of a CTA's columns are the CTAs whose columns it reads).
 *
 * Polls are bounded by %globaltimer and stop early when another CTA has
 * recorded an error; a CTA that gives up records kErrTimeout, and every
 * CTA then skips its remaining work while still passing each cluster
 * barrier (all CTAs pass the same number).  The host checks before the
 * launch that all G clusters fit the GPU at once (a plain cluster launch:
 * a cooperative launch with clusters faulted under the profiler, whose
 * replay did not keep the cluster shape), and the kernel checks its
 * cluster shape before it addresses another CTA's shared memory.
 *
 * The per-cell operations are those of the streaming kernel (dev::cn_row,
 * one column per thread): FP64 cells get the same bits as there, FP32 ones
 * agree to rounding (that kernel's FP32 arithmetic runs in column pairs and
 * is compiled to differently rounded code); the
 * per-step sums of rows 0 and 1 (Eqs. v_dr_generic, norm_in_phi) are taken
 * per cluster (FP64 states in FP64, FP32 states in error-free FP32 pairs)
 * and added over the clusters, in cluster order, by a second kernel that
 * writes the trace.
 */
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "bte_device.cuh"
#include "bte_internal.h"

namespace cg = cooperative_groups;

namespace bte {
namespace {

using namespace dev;

/* global array a: 0 a_w, 1 b_w, 2 a_f, 3 b_f */
template <typename T>
__device__ __forceinline__ T* wsel(const WideArgs<T>& A, int a) {
    return a == 0 ? A.a_w : a == 1 ? A.b_w : a == 2 ? A.a_f : A.b_f;
}

/* exchange word of row n: buffer (the parity of the producing grid's
 * update count), grid (0 whole, 1 fractional), side (0 first column of
 * block g, 1 last), array (0 a, 1 b), part (FP64: 0 high, 1 low half) */
template <typename T>
__device__ __forceinline__ size_t xword(int buf, int grid, int side, int ab, int part, int g, int n,
                                        int G, int N1) {
    constexpr int W = sizeof(T) / 4;
    return ((((((size_t)buf * 2 + grid) * 2 + side) * 2 + ab) * W + part) * G + g) * N1 + n;
}

/* One 8-byte word, written and read as a whole (single-copy atomic): the
 * tag in the high half, 32 bits of the value in the low half, so a reader
 * that sees the tag it expects holds the value written with it. */
__device__ __forceinline__ void st_word(unsigned long long* p, unsigned tag, unsigned bits) {
    const unsigned long long w = ((unsigned long long)tag << 32) | bits;
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

/* 32-bit part `part` of a value: FP32 its bits; FP64 part 0 the high half,
 * part 1 the low half */
__device__ __forceinline__ unsigned val_part(float v, int) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned val_part(double v, int part) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return part == 0 ? (unsigned)(b >> 32) : (unsigned)b;
}

/* A thread's part of a row sum: FP64 for FP64 states, an error-free pair
 * of FP32 numbers for FP32 states; warp() adds the warp's parts. */
template <typename T>
struct RowSum;
template <>
struct RowSum<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ double warp() const { return warp_sum(v); }
};
template <>
struct RowSum<float> {
    F2 v{0.0f, 0.0f};
    __device__ __forceinline__ void add(float x) { v = f2_add1(v, x); }
    __device__ __forceinline__ double warp() const { return warp_sum_f2(v); }
};

template <typename T>
__global__ void __launch_bounds__(kWideMaxThreads) wide_kernel(WideArgs<T> A) {
    constexpr int GG = Cols<T>::G; /* global ghost columns before m = 0 */
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = A.C, G = A.G, Wc = A.Wc, rp = A.rows_per;
    /* the halo-row pushes address the CTAs of this cluster by rank, and
     * every cell needs its thread: a launch in any other shape returns at
     * once (every CTA alike, before any barrier or access) */
    if ((int)cl.num_blocks() != C || (int)gridDim.x != G * C || gridDim.y != 1 || gridDim.z != 1 ||
        (int)blockDim.x < rp * Wc + 32) {
        if (threadIdx.x == 0) atomicExch(A.err, kErrLaunch);
        return;
    }
    const int rank = (int)cl.block_rank();
    const int g = (int)blockIdx.x / C;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = (nthr + 31) >> 5;
    const int N = A.N, M = A.M, N1 = N + 1;
    const size_t gp = (size_t)A.pitch;
    const int r0 = min(N1, rank * rp), r1 = min(N1, r0 + rp), R = r1 - r0;
    const int c0 = g * Wc;
    const int Wp = Wc + 2; /* local columns: halo, Wc own, halo */
    const size_t arr = (size_t)(rp + 2) * Wp;
    T* s = reinterpret_cast<T*>(smem); /* [4][rp + 2][Wp]: a_w, b_w, a_f, b_f */
    T* sG = s + 4 * arr;               /* [Wp] column factor of a0 */
    T* sPh = sG + Wp;                  /* [Wp] phi_m */
    T* sR = sPh + Wp;                  /* [rp + 2] row factor of a0, rows r0-1 .. r0+rp */

    /* ---- load: zero everything, then rows r0-1 .. r1 and columns
     * c0-1 .. c0+Wc that exist (halo rows and columns included) ---- */
    for (size_t q = tid; q < 4 * arr + 2 * (size_t)Wp + rp + 2; q += nthr) s[q] = (T)0;
    __syncthreads();
    if (R > 0) {
        const int rows = R + 2;
        for (int q = tid; q < 4 * rows * Wp; q += nthr) {
            const int a = q / (rows * Wp);
            const int rem = q - a * rows * Wp;
            const int li = rem / Wp, lc = rem - li * Wp;
            const int n = r0 - 1 + li, m = c0 - 1 + lc;
            if (n < 0 || n > N || m < 0 || m > M) continue;
            s[a * arr + (size_t)li * Wp + lc] = wsel(A, a)[(size_t)n * gp + GG + m];
        }
        for (int q = tid; q < Wp; q += nthr) {
            const int m = c0 - 1 + q;
            if (m < 0 || m > M) continue;
            sG[q] = A.col_g[GG + m];
            sPh[q] = A.col_phi[GG + m];
        }
        for (int q = tid; q < rows; q += nthr) {
            const int n = r0 - 1 + q;
            sR[q] = (n >= 0 && n <= N) ? A.row_a0[n] : (T)0;
        }
    }
    __syncthreads();

    /* a CTA's first own row is the halo row below the last own row of
     * rank-1 (its shared row rp + 1), its last own row the halo row above
     * rank+1's first (its shared row 0) */
    const bool have_up = R > 0 && r0 >= 1, have_dn = R > 0 && r1 <= N;
    T* halo_up = have_up ? cl.map_shared_rank(s, rank - 1) + (size_t)(rp + 1) * Wp : nullptr;
    T* halo_dn = have_dn ? cl.map_shared_rank(s, rank + 1) : nullptr;
    const int rank_lo = have_up ? rank - 1 : rank, rank_hi = have_dn ? rank + 1 : rank;
    const CnK<T> cn = cn_constants<T>(A.h, A.nu, A.xi);

    /* one cell per thread: thread tid < R Wc updates row r0 + il, column
     * c0 + j of each grid (the host keeps rows_per x Wc within the block);
     * the last warp holds no cell and, in rank 0, adds the row sums */
    const bool has = tid < R * Wc;
    const int il = has ? tid / Wc : 0, j = has ? tid - il * Wc : 0;
    const int n = r0 + il, m = c0 + j, lc = j + 1;
    const size_t c_up = (size_t)il * Wp + lc, c_own = c_up + Wp, c_dn = c_own + Wp;
    const T chi = (n == 1) ? (T)2 : (T)1;
    const T hr = Rn<T>::mul(A.h, sR[il + 1]);
    const T gcol = sG[lc], phc = sPh[lc];
    const bool col_ok = m <= M;
    const bool obs_warp = rank == 0 && warp == nwarp - 1;

    /* the drive of half-step hf at phase kq, and the part of this thread's
     * update that depends on it but not on the state */
    auto drive = [&](int hf, int kq) { return half_drive<T>(hf ? A.e_frac : A.e_whole, A.dstride, kq); };
    auto coef = [&](const Half<T>& D) {
        const T nf = (T)n;
        return cn_coef<T>(Rn<T>::mul(nf, rot_factor<T>(D.E0, D.B0, phc, A.hh)),
                          Rn<T>::mul(nf, rot_factor<T>(D.E1, D.B1, phc, A.hh)), cn);
    };
    int kk = A.P > 0 ? (int)(A.k0 % A.P) : 0; /* drive phase (k0 + k) mod P */
    Half<T> D = drive(0, kk);
    CnCoef<T> cf = coef(D);
    bool dead = false; /* a wait gave up (same on every thread) */
    cluster_arrive();  /* initial state loaded */
    for (long long k = 0; k < A.K; ++k) {
        for (int hf = 0; hf < 2; ++hf) {
            /* hf 0: whole grid z_w^{k+1} = T(z_w^k; S(z_f^{k+1/2}));
             * hf 1: fractional grid z_f^{k+3/2} = T(z_f^{k+1/2}; S(z_w^{k+1})) */
            const int o = hf ? 2 : 0, x = hf ? 0 : 2;
            const unsigned hs = (unsigned)(2 * k + hf);
            if (hf == 1 && obs_warp && !dead) {
                /* row 0 (a) and row 1 (b) of the new whole grid, which this
                 * half-step leaves unchanged, while the other warps wait
                 * and update: the step's partial sums of this cluster */
                RowSum<T> pn, pv;
                for (int q = lane; q < Wc; q += 32) {
                    pn.add(s[(size_t)Wp + 1 + q]);            /* a_w, shared row 1 */
                    pv.add(s[arr + (size_t)2 * Wp + 1 + q]);  /* b_w, shared row 2 */
                }
                const double sn = pn.warp(), sv = pv.warp();
                if (lane == 0) {
                    A.part[((size_t)k * G + g) * 2] = sn;
                    A.part[((size_t)k * G + g) * 2 + 1] = sv;
                }
            }
            cluster_wait(); /* halo rows of grid x pushed by the cluster's CTAs */
            if (G > 1 && hs > 0) {
                /* warp 0 fills the halo columns of grid x (shared rows
                 * 0 .. R+1; the left one is block g-1's last column, the
                 * right one block g+1's first) from the exchange words
                 * that the neighbouring clusters wrote in half-step hs-1,
                 * polling each until it carries tag hs (bounded by
                 * %globaltimer; given up at once once an error is recorded) */
                bool ok = !dead;
                if (warp == 0 && ok) {
                    constexpr int W = sizeof(T) / 4;
                    const int buf = ((hs - 1) >> 1) & 1;
                    const uint64_t t0 = global_timer();
                    for (int q = lane; q < 4 * W * (R + 2) && ok; q += 32) {
                        const int side = q & 1, ab = (q >> 1) & 1, part = (q >> 2) % W;
                        const int li = q / (4 * W);
                        const int nq = r0 - 1 + li, gg = side ? g + 1 : g - 1;
                        if (nq < 0 || nq > N || gg < 0 || gg >= G) continue;
                        const unsigned long long* p =
                            A.xw + xword<T>(buf, x >> 1, side ? 0 : 1, ab, part, gg, nq, G, N1);
                        unsigned long long w = ld_word(p);
                        while ((unsigned)(w >> 32) != hs) {
                            if (*reinterpret_cast<const volatile int*>(A.err) != 0 ||
                                global_timer() - t0 > kWaitLimitNs) {
                                ok = false;
                                break;
                            }
                            w = ld_word(p);
                        }
                        /* the value's 32-bit part into its place in the halo
                         * cell (FP64: the high half at the higher address) */
                        T* cellp = s + (size_t)(x + ab) * arr + (size_t)li * Wp + (side ? Wc + 1 : 0);
                        reinterpret_cast<unsigned*>(cellp)[W == 2 && part == 0 ? 1 : 0] = (unsigned)w;
                    }
                    ok = __all_sync(0xffffffffu, ok);
                }
                if (__syncthreads_or(!ok)) {
                    if (!dead && tid == 0) atomicExch(A.err, kErrTimeout);
                    dead = true;
                }
            }
            /* ---- the update of this thread's cell of grid o from grid x,
             * stored in place and written where other CTAs read it next ---- */
            if (has && !dead) {
                const T* xa = s + (size_t)x * arr;
                const T* xb = xa + arr;
                const T da_u = xa[c_up + 1] - xa[c_up - 1];
                const T da_d = xa[c_dn + 1] - xa[c_dn - 1];
                const T db_u = xb[c_up + 1] - xb[c_up - 1];
                const T db_d = xb[c_dn + 1] - xb[c_dn - 1];
                T* pa = s + (size_t)o * arr + c_own;
                T* pb = pa + arr;
                T an, bn;
                cn_update<T>(*pa, *pb, stencil_a<T>(D.cc, db_d, db_u), stencil_b<T>(D.cc, chi, da_u, da_d),
                             hr, gcol, cf, cn, an, bn);
                const T na = col_ok ? an : (T)0;
                const T nb = (col_ok && n > 0) ? bn : (T)0;
                *pa = na;
                *pb = nb;
                if (il == 0 && halo_up) {
                    halo_up[(size_t)o * arr + lc] = na;
                    halo_up[(size_t)(o + 1) * arr + lc] = nb;
                }
                if (il == R - 1 && halo_dn) {
                    halo_dn[(size_t)o * arr + lc] = na;
                    halo_dn[(size_t)(o + 1) * arr + lc] = nb;
                }
                /* a first (side 0) or last (side 1) column that a
                 * neighbouring cluster reads: tagged words, tag hs + 1 */
                const bool w_first = j == 0 && g > 0, w_last = j == Wc - 1 && g + 1 < G;
                if (w_first || w_last) {
                    constexpr int W = sizeof(T) / 4;
                    const int buf = (hs >> 1) & 1;
#pragma unroll
                    for (int sd = 0; sd < 2; ++sd) {
                        if (!(sd == 0 ? w_first : w_last)) continue;
#pragma unroll
                        for (int part = 0; part < W; ++part) {
                            st_word(A.xw + xword<T>(buf, o >> 1, sd, 0, part, g, n, G, N1), hs + 1,
                                    val_part(na, part));
                            st_word(A.xw + xword<T>(buf, o >> 1, sd, 1, part, g, n, G, N1), hs + 1,
                                    val_part(nb, part));
                        }
                    }
                }
            }
            /* the next half-step's drive and coefficients, computed while
             * this one's stores drain and the neighbours catch up */
            const int kn = hf == 0 ? kk : (A.P > 0 ? (kk + 1 == A.P ? 0 : kk + 1) : 0);
            D = drive(hf ^ 1, kn);
            cf = coef(D);
            __syncthreads();
            cluster_arrive();
        }
        if (A.P > 0 && ++kk == A.P) kk = 0; /* P = 0 (omega = 0): row 0 every step */
    }
    cluster_wait(); /* pairs the last arrive: no CTA writes this one's shared memory after it */

    /* ---- final state of the own rows and columns ---- */
    if (!dead && R > 0) {
        for (int u = tid; u < 4 * R * Wc; u += nthr) {
            const int a = u / (R * Wc);
            const int rem = u - a * R * Wc;
            const int il = rem / Wc, j = rem - il * Wc;
            const int m = c0 + j;
            if (m > M) continue;
            wsel(A, a)[(size_t)(r0 + il) * gp + GG + m] = s[a * arr + (size_t)(il + 1) * Wp + j + 1];
        }
    }
}

/* Trace of steps k0+1 .. k0+K from the per-cluster sums, added in cluster
 * order (the same order whatever the launch's timing). */
__global__ void wide_fold_kernel(const double* part, int G, long long K, long long k0,
                                 double vscale, double nscale, double* trace_v, double* trace_n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < K;
         k += (long long)gridDim.x * blockDim.x) {
        double sn = 0, sv = 0;
        for (int g = 0; g < G; ++g) {
            sn += part[((size_t)k * G + g) * 2];
            sv += part[((size_t)k * G + g) * 2 + 1];
        }
        trace_n[k0 + k + 1] = nscale * sn;
        trace_v[k0 + k + 1] = vscale * sv;
    }
}

}  // namespace

template <typename T>
size_t wide_smem_bytes(int rows_per, int Wc) {
    const size_t Wp = (size_t)Wc + 2;
    const size_t arr = (size_t)(rows_per + 2) * Wp;
    const size_t b = (4 * arr + 2 * Wp + rows_per + 2) * sizeof(T);
    return (b + 15) / 16 * 16;
}

template <typename T>
int wide_max_clusters(int C, size_t smem, int threads, int* clusters) {
    auto fn = wide_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return (int)cudaOccupancyMaxActiveClusters(clusters, fn, &cfg);
}

template <typename T>
int launch_wide(const WideArgs<T>& a, int threads, size_t smem, void* stream) {
    int fit = 0;
    int rc = wide_max_clusters<T>(a.C, smem, threads, &fit); /* attributes are per function */
    if (rc) return rc;
    if (fit < a.G) return (int)cudaErrorLaunchOutOfResources; /* the G clusters do not fit at once */
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.G * a.C, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = a.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, wide_kernel<T>, a);
    return e == cudaSuccess ? 0 : (int)e;
}

int launch_wide_fold(const double* part, int G, long long K, long long k0, double vscale,
                     double nscale, double* trace_v, double* trace_n, void* stream) {
    if (K <= 0) return 0;
    const int threads = 256;
    const long long blocks = (K + threads - 1) / threads;
    wide_fold_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), threads, 0, (cudaStream_t)stream>>>(
        part, G, K, k0, vscale, nscale, trace_v, trace_n);
    return (int)cudaGetLastError();
}

template size_t wide_smem_bytes<float>(int, int);
template size_t wide_smem_bytes<double>(int, int);
template int wide_max_clusters<float>(int, size_t, int, int*);
template int wide_max_clusters<double>(int, size_t, int, int*);
template int launch_wide<float>(const WideArgs<float>&, int, size_t, void*);
template int launch_wide<double>(const WideArgs<double>&, int, size_t, void*);

}  // namespace bte
