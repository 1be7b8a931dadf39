/*
 * bte_internal.h -- structures shared by the library's host code and its
 * CUDA kernels.  Not part of the public ABI.
 *
 * Device layout of one grid array (a or b, whole or fractional grid):
 *   rows n = 0..N (N = n_max), row pitch `pitch` elements, column m of the
 *   phi_y grid at physical index G + m with G = 128 / sizeof(T) zero ghost
 *   columns on the left (so tiles start on 128-byte lines); columns
 *   G+M+1 .. pitch-1 are zero ghosts too.
 *   Ghost columns are written once (zero) and never again, so the stencil
 *   at m = 0 and m = M reads the boundary value 0 of Eqs. a_boundary and
 *   b_boundary without a branch.  Rows outside 0..N are never stored; the
 *   kernels substitute 0 for them.
 */
#pragma once
#include <cstddef>
#include <cstdint>

namespace bte {

/* value stored in the device error word when a bounded wait gives up */
constexpr int kErrTimeout = 1;
/* ... and when a kernel finds itself launched in another shape than the
 * one its arguments describe (it then returns before any access) */
constexpr int kErrLaunch = 2;

/* Column layout constants: G zero ghost columns before m = 0 (128 bytes),
 * H halo columns streamed on each side of a tile (16 bytes, the TMA
 * granule; the row pitch leaves room for 32). */
template <typename T>
struct Cols {
    static constexpr int G = 128 / (int)sizeof(T);
    static constexpr int H = 16 / (int)sizeof(T);
};

/* Ping-pong state above this many bytes does not stay in L2 (129 MB on a
 * GB300) from one step to the next: the step kernel then alternates the
 * direction of its row walks, so that each step starts with the rows the
 * step before wrote last. */
constexpr size_t kAltStateBytes = 96ull << 20;

/* Arguments of the fused step kernel (one leap-frog step). */
template <typename T>
struct StepArgs {
    T* a_w[2];            /* ping-pong sets: set (k & 1) holds step k           */
    T* b_w[2];
    T* a_f[2];
    T* b_f[2];
    const T* row_a0;      /* [N+1]   sigma_n I_n/I_0 / pi                        */
    const T* col_g;       /* [pitch] sqrt(mu/(2 pi alpha)) exp(-mu phi^2/2), 0 in ghosts */
    const T* col_phi;     /* [pitch] phi_y(m), 0 in ghosts                      */
    const T* e_whole;     /* [3][dstride] at t = i dt_eff: E(t), B(t), and the
                             stencil coefficient B(t + dt/2) dt/(4 dphi) of the
                             whole-grid half-step from t (i = 0..P+1); FP64
                             values rounded to T once on the host             */
    const T* e_frac;      /* [3][dstride] at t = (i + 1/2) dt_eff: E(t), B(t),
                             and B(t + dt/2) dt/(4 dphi) of the fractional
                             half-step from t                                   */
    const long long* base;/* device step counter: the launch advances step base+i */
    double* trace_v;      /* [K+1] whole-grid v_dr samples                       */
    double* trace_n;      /* [K+1] whole-grid norm samples                       */
    double* part;         /* [dring][2][ntx] per-tile partial sums of row 0 / row 1 */
    unsigned* ticket;     /* [dring] arrival counters of the row-0 CTAs          */
    int dring;            /* slots of part / ticket: step k uses slot k % dring  */
    int* err;             /* device error word (timeouts)                        */
    unsigned* done;       /* [ntx * nty] steps each item has completed in a
                             persistent launch (zero at its start)             */
    int nsteps;           /* steps of a persistent launch                        */
    int N, M, pitch, P;
    int dstride;          /* row stride of the drive tables (>= P + 2)          */
    int tile_m, chunk_n, ntx, nty;
    int vec;              /* phi_y columns per compute thread (2 or 4)         */
    int grid;             /* persistent CTAs; items are ntx * nty              */
    int alt;              /* 1: one-step launches alternate the row-walk
                             direction (a state larger than L2)              */
    T h, hh, nu, xi;      /* dt, dt/2, 1 + dt/2, 1 - dt/2                        */
    double vscale, nscale;/* pi sqrt(alpha) dphi, 2 pi sqrt(alpha) dphi          */
};

/* One instance of a batched launch (device array, one record per instance).
 * All instances of a batch share tile_m / chunk_n / vec and advance in
 * lock-step (step base + i); an instance whose K steps are done is skipped.
 * Instead of a trace, the instance accumulates the window sums in FP64. */
template <typename T>
struct BatchInst {
    T* a_w[2];
    T* b_w[2];
    T* a_f[2];
    T* b_f[2];
    const T* row_a0;
    const T* col_g;
    const T* col_phi;
    const T* e_whole;     /* drive tables as in StepArgs                         */
    const T* e_frac;
    double* part;         /* [2][ntx] per-tile partial sums                      */
    unsigned* ticket;     /* arrival counter of the row-0 items                  */
    double* acc;          /* [8]: sum v cos(omega t) and sum v over the window,
                             max |norm-1|, non-finite flag, v and norm of the
                             latest step, v and norm of step 0               */
    long long K, Kw;      /* steps of the run, window samples                    */
    long long k0;         /* step index of the state the run starts from (the
                             on-chip kernel continues a single instance's run) */
    double *trace_v, *trace_n; /* [k0 + K + 1] per-step samples, or NULL         */
    int N, M, pitch, P, ntx, nty;
    int dstride;
    int item0;            /* index of the instance's first work item            */
    T h, hh, nu, xi;
    double vscale, nscale;
    double omega, dt_eff;
};

/* Arguments of a batched launch. */
template <typename T>
struct BatchArgs {
    const BatchInst<T>* inst;
    const int* item_inst; /* [items] instance of each work item                  */
    int ninst, items;     /* instances; total work items                         */
    const long long* base;/* common step counter                                 */
    int* err;
    int tile_m, chunk_n, vec, grid;
    int alt;              /* as StepArgs::alt, for the batch's total state     */
};

/* Arguments of the on-chip batched kernel (bte_resident.cu): clusters of C
 * CTAs take points order[0..count) from the queue counter; each CTA holds
 * ceil((N+1)/C) harmonic rows of its point in shared memory; the per-warp
 * partial sums start at byte red_off, after the largest point's arrays. */
template <typename T>
struct ResArgs {
    const BatchInst<T>* inst;
    const int* order;
    int count;
    unsigned* queue;
    int C;
    size_t red_off;
};

/* threads per CTA of the on-chip kernel over several clusters, at most */
constexpr int kWideMaxThreads = 512;

/* Arguments of the single-instance on-chip kernel over several clusters
 * (bte_wide.cu): G clusters of C CTAs.  Cluster g holds phi_y columns
 * [g Wc, (g+1) Wc) of every harmonic row; CTA r of it rows [r R, (r+1) R),
 * R = rows_per.  The state is advanced in place (one ping-pong set). */
template <typename T>
struct WideArgs {
    T* a_w; T* b_w; T* a_f; T* b_f;   /* state, rows `pitch` elements apart      */
    const T* row_a0; const T* col_g; const T* col_phi;
    const T* e_whole; const T* e_frac; /* drive tables as in StepArgs           */
    unsigned long long* xw; /* [2 buffers][2 grids][2 sides][2 arrays][W][G][N+1]
                         exchange words: each block's first (side 0) and last
                         (side 1) column, the value's 32-bit part(s) (W = 1
                         for FP32; 2 for FP64: high, low) under the number of
                         the half-step that made it, plus one (zeroed by the
                         caller before the launch)                           */
    double* part;     /* [K][G][2]: per-step row sums of row 0 (a) and row 1
                         (b) of the whole grid over each cluster's columns  */
    int* err;         /* error word: kErrTimeout when a wait gave up, kErrLaunch
                         when the launch shape is not G clusters of C CTAs */
    long long K;      /* steps of this launch                                */
    long long k0;     /* step index the launch starts from                   */
    int N, M, pitch, P, dstride;
    int C, G, Wc, rows_per;
    T h, hh, nu, xi;
};

/* One plain application of T (start-up half step), unfused. */
template <typename T>
struct ApplyArgs {
    const T* a;  const T* b;     /* state at t0                                */
    const T* as; const T* bs;    /* stencil source                             */
    T* an; T* bn;                /* output (may not alias the inputs)          */
    const T* row_a0; const T* col_g; const T* col_phi;
    int N, M, pitch;
    double E_start, E_end, B_start, B_end;
    T h, hh, nu, xi, c;   /* c: stencil coefficient at the source's time        */
};

struct FinalArgs {
    const double* trace_v;
    const double* trace_n;
    long long k;          /* current step: samples 0..k are valid */
    long long K, Kw, P;
    double omega, dt_eff, inv_r1;
    double* out;          /* [4]: A, vbar, max|norm-1|, nonfinite flag */
};

/* Kernel launchers (bte_kernels.cu). */
template <typename T>
int launch_init(T* a_w, T* b_w, const T* row_a0, const T* col_g, int N, int M, int pitch,
                void* stream);
template <typename T>
int launch_apply(const ApplyArgs<T>& a, void* stream);
/* Launches step base + i, reading ping-pong set (parity + i) & 1 and writing
 * the other one (the host knows the set, so no device read is needed to
 * choose it).  `pdl` enables programmatic dependent launch (the prologue
 * overlaps the previous launch). */
template <typename T>
int launch_step(const StepArgs<T>& a, int i, int parity, bool pdl, void* stream);
/* Persistent form: one cooperative launch of a.grid = ntx * nty CTAs, one
 * work item each, advances a.nsteps steps from base (set `parity` holds
 * step base).  Before step s > 0 an item waits until the items around it
 * (its tile and chunk neighbours, whose step s - 1 output it reads and whose
 * step s - 1 input it overwrites) have completed s steps in a.done (zeroed
 * by the caller before the launch); a.dring > ntx slots of the row-0
 * partial sums keep the steps that may be in flight at once apart. */
template <typename T>
int launch_step_persist(const StepArgs<T>& a, int parity, void* stream);
template <typename T>
int step_kernel_configure_persist(int tile_m, int chunk_n, int vec, int* blocks_per_sm);
/* Batched form: every active instance of the batch advances one step. */
template <typename T>
int launch_step_batch(const BatchArgs<T>& a, int i, int parity, bool pdl, void* stream);
template <typename T>
int step_kernel_configure_batch(int tile_m, int chunk_n, int vec, int* blocks_per_sm);
template <typename T>
int launch_observe(const T* a_w, const T* b_w, int M, int pitch, double vscale,
                   double nscale, double* trace_v, double* trace_n, long long slot,
                   void* stream);
int launch_advance_base(long long* base, long long by, void* stream);
/* one bounded wait that nothing completes; records kErrTimeout in *err */
int launch_wait_probe(int* err, unsigned long long limit_ns, void* stream);
int launch_finalize(const FinalArgs& a, void* stream);
/* f on an nphix x (M+1) grid from the harmonics of one grid: out [nphix][M+1] (device) */
template <typename T>
int launch_pdf(const T* a, const T* b, int N, int M, int pitch, int nphix, double* out,
               void* stream);
/* On-chip batched kernel: shared memory a CTA needs for a point of N+1
 * harmonics and M+1 columns split over C CTAs (*arrays_bytes: the part
 * before the warp partials), clusters that fit the GPU at once, launch. */
template <typename T>
size_t resident_smem_bytes(int N, int M, int C, size_t* arrays_bytes);
template <typename T>
int resident_max_clusters(int C, size_t smem, int threads, int* clusters);
template <typename T>
int launch_resident(const ResArgs<T>& a, int clusters, int threads, size_t smem, void* stream);
/* On-chip kernel over several clusters: shared memory of one CTA, clusters
 * of C CTAs that fit the GPU at once (sets
 * the kernel's attributes), launch of G clusters (cooperative where the
 * driver accepts it with clusters), and the fold of the per-cluster row
 * sums of K steps into the trace. */
template <typename T>
size_t wide_smem_bytes(int rows_per, int Wc);
template <typename T>
int wide_max_clusters(int C, size_t smem, int threads, int* clusters);
template <typename T>
int launch_wide(const WideArgs<T>& a, int threads, size_t smem, void* stream);
int launch_wide_fold(const double* part, int G, long long K, long long k0, double vscale,
                     double nscale, double* trace_v, double* trace_n, void* stream);
/* Sets the calling thread's bte_last_error() message; returns code. */
int report_error(int code, const char* msg);
template <typename T>
size_t step_smem_bytes(int tile_m, int chunk_n, int vec);
template <typename T>
int step_block_threads(int tile_m, int vec);
template <typename T>
int step_max_tile(int vec);
template <typename T>
int step_kernel_configure(int tile_m, int chunk_n, int vec, int* blocks_per_sm);

}  // namespace bte
