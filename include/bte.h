/*
 * bte.h -- C ABI of the GB300 solver for the two-dimensional, spatially
 * homogeneous superlattice Boltzmann transport equation
 *     df/dt + (E + B phi_y) df/dphi_x - B sin(phi_x) df/dphi_y = f0 - f
 * (Priimak, arXiv:1401.6047, Sec. 2, Eq. boltzmann_final), with the drive
 * E(t) = E_dc + E_omega cos(omega t) and a constant B (the paper's runs) or
 * B(t) = B + B_omega cos(omega t + B_phase) (bte_params.B_omega, B_phase).
 *
 * f is held as Fourier harmonics a_n(phi_y), b_n(phi_y), n = 0..n_max
 * (Sec. 2, Eq. f_fourier) on a uniform phi_y grid, and advanced by the
 * paper's Crank-Nicolson / staggered leap-frog scheme (Sec. 3, Eqs.
 * a_t_plus_1, b_t_plus_1, leap_frog_1, leap_frog_2).  One time step advances
 * the whole grid z^t -> z^{t+1} and the fractional grid z^{t+1/2} ->
 * z^{t+3/2}; both run in one fused CUDA kernel.
 *
 * Conventions for every entry point:
 *   - Functions return a bte_status (0 = BTE_OK).  No exception crosses the
 *     ABI.  bte_last_error() gives a message for the last failure on the
 *     calling thread.
 *   - Pointers to parameters and outputs are HOST pointers owned by the
 *     caller, unless a comment says "device".
 *   - A handle owns every device allocation it made; bte_destroy frees them.
 *   - Work is queued on the handle's CUDA stream; bte_step returns before the
 *     GPU finishes, bte_observables / bte_trace / bte_get_state synchronise.
 *   - A handle may be used by one host thread at a time.
 *
 * Readings of the paper implemented here (the same ones as the test oracle):
 *   sigma(0) = 1/2 (Eq. Bolzmann_initial_pdf); b^{t+1} = (g mu' + h nu)/D
 *   (Eq. b_t_plus_1 with the sign that solves the 2x2 system); stencil
 *   coefficient B dt/(4 dphi) without alpha; b_0 = 0 (Eq. b_boundary);
 *   theta at the step start, theta' at its end; start-up half step with
 *   dt/2; dt adjusted to a whole number of steps per drive period; window
 *   averages over whole periods; observables from the whole grid; a
 *   time-dependent B sampled where E is, and in the stencil coefficient at
 *   the time of the grid that supplies the stencil.
 */
#ifndef BTE_H
#define BTE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BTE_API __attribute__((visibility("default")))
#else
#define BTE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BTE_OK = 0,
    BTE_EINVAL = -1,    /* invalid argument or parameter                     */
    BTE_ENOMEM = -2,    /* device allocation failed / workspace too small     */
    BTE_ECUDA = -3,     /* a CUDA runtime call failed                         */
    BTE_EUNSTABLE = -4, /* NaN/Inf seen, or |norm - 1| above the threshold    */
    BTE_ETIMEOUT = -5,  /* a bounded in-kernel wait gave up                   */
    BTE_ESTATE = -6     /* call not valid in the handle's state               */
} bte_status;

typedef enum {
    BTE_FP64 = 0,       /* state, stencil and 2x2 solve in FP64               */
    BTE_FP32_MIXED = 1  /* FP32 state and stencil in increment form; drive
                           table, coefficients (rounded once), reductions,
                           norm and time averages in FP64                     */
} bte_precision;

/* Problem parameters (dimensionless units of Sec. 2, Eqs. substitutions). */
typedef struct {
    double E_dc, E_omega, omega; /* drive E(t) = E_dc + E_omega cos(omega t)   */
    double B;                    /* magnetic field: its constant part          */
    double mu;                   /* Delta_1 / (2 k_B T), > 0                   */
    double alpha;                /* m / m_x, > 0 (observables do not depend on it) */
    double phiy_min, phiy_max;   /* phi_y grid, both ends included             */
    double dt;                   /* requested step; dt_eff = 2 pi/(omega P),
                                    P = round(2 pi/(omega dt)) when omega > 0  */
    double periods;              /* run length in drive periods (omega > 0)   */
    double t_max;                /* run length in time units (omega == 0)     */
    double avg_window;           /* averaging window at the end of the run:
                                    periods (omega > 0) or time (omega == 0)  */
    int32_t n_max;               /* harmonics n = 0..n_max, >= 1               */
    int32_t m_points;            /* phi_y points M+1, >= 3                      */
    int32_t precision;           /* bte_precision                               */
    int32_t reserved;            /* must be 0                                   */
    /* Time-dependent field B(t) = B + B_omega cos(omega t + B_phase), at the
     * drive's frequency (constant B + B_omega cos(B_phase) when omega == 0).
     * Eqs. a_n_dot and b_n_dot hold for any B(t) (Sec. 2); the scheme samples
     * B where it samples E: the rotation n (E + B phi_y) of a half-step at
     * its start and its end, the stencil coefficient B dt/(4 dphi) at the
     * time of the other grid that supplies the stencil (the middle of the
     * half-step; t = 0 for the start-up half step).  Zero for the paper's
     * constant field. */
    double B_omega, B_phase;
} bte_params;

/* Observables (Sec. 2, Eqs. v_dr_generic, norm_in_phi, absorption_def). */
typedef struct {
    double t;                /* time of the current whole-grid state          */
    int64_t step;            /* its step index k (t = k dt_eff)               */
    double v_dr;             /* pi sqrt(alpha) int b_1 dphi_y at step k        */
    double norm;             /* 2 pi sqrt(alpha) int a_0 dphi_y at step k      */
    double v_dc_avg;         /* window mean of v_dr (NaN before the window ends) */
    double absorption;       /* (2 I_0/I_1) <v_dr cos(omega t)> over the window;
                                NaN when omega == 0 or the window is not done  */
    double norm_max_abs_err; /* max over steps 0..k of |norm - 1|              */
    double dt_eff;           /* time step actually used                        */
    int64_t steps_total;     /* K, steps of the full run                       */
    int64_t steps_per_period;/* P (0 when omega == 0)                          */
    int64_t window_steps;    /* Kw, samples in the averaging window            */
    int32_t status;          /* bte_status of the run so far                   */
    int32_t reserved;
} bte_obs;

/* Optional launch shape of the fused step kernel; 0 fields = automatic. */
typedef struct {
    int32_t tile_m;      /* phi_y columns per work item (multiple of 4, 32..1024) */
    int32_t chunk_n;     /* harmonic rows per work item (>= 4)               */
    int32_t graph_steps; /* steps captured per CUDA graph replay (0 = auto)  */
    int32_t vec;         /* phi_y columns per thread: 2 or 4 (FP64: 2)      */
    int32_t resident;    /* 1: keep the grid on chip -- all four arrays in the
                            shared memory of one thread-block cluster of C
                            CTAs (the largest C in 16, 8, 4, 2, 1 that leaves
                            every CTA at least two harmonic rows and fits
                            232,448 bytes per CTA), each bte_step/bte_run call
                            one persistent launch that advances the state in
                            place (the kernel of the batched run's on-chip
                            tier); BTE_EINVAL when the grid does not fit.
                            2: persistent -- the state stays in global
                            memory (held in L2 across steps when it fits
                            there) and each bte_step/bte_run call is one
                            cooperative launch per 8192 steps with one CTA
                            per work item (all resident at once; BTE_EINVAL
                            when the grid has more items than co-resident
                            CTAs); an item starts step k once the 3 x 3
                            items around it have finished step k-1 (a
                            release/acquire completion counter per item,
                            polled with a %globaltimer bound: BTE_ETIMEOUT
                            when it gives up).  Same per-cell arithmetic
                            and reduction order as mode 0: bit-identical.
                            On a GB300 it is slower than mode 0 on the
                            grids measured (401 x 4001 FP32: 20.9 against
                            17.4 us per step).
                            3: on chip over several clusters -- the grid
                            cut into G column blocks (one cluster of C CTAs
                            each, C as for 1) whose CTAs keep their part of
                            the four arrays in shared memory; each
                            bte_step/bte_run call is one launch per 8192
                            steps of G x C CTAs, all resident at once
                            (checked before the launch), that exchange their edge
                            columns through global memory as words tagged
                            with their half-step, polled with a
                            %globaltimer bound (BTE_ETIMEOUT when a wait
                            gives up).  Per-cell arithmetic as in mode
                            0; the per-step sums of rows 0 and 1 are added
                            per cluster, then over clusters in order.
                            One thread per cell: BTE_EINVAL when a CTA's
                            block has more than 480 cells or does not fit
                            232,448 bytes, or the G clusters do not fit the
                            GPU at once (small grids: 31 x 201 FP64 runs
                            5.5 instead of 16.1 us per step on a GB300).
                            0: one fused step kernel launch per step.      */
    int32_t walk;        /* order in which one-step launches walk the
                            harmonic rows of a work item: 0 automatic
                            (alternate when the ping-pong state exceeds 96
                            MB, so that each step starts with the rows the
                            step before wrote last, which L2 still holds;
                            upward otherwise), 1 upward every step, 2
                            alternate every step.  The results are the same
                            bits in every order.                           */
    int32_t wide_cols;   /* resident = 3: phi_y columns per cluster, 1..4096,
                            at most 32 clusters (0: automatic -- about 32
                            columns per cluster in FP64, 128 in FP32, at
                            most 128 CTAs in all and no more clusters than
                            fit the GPU at once)                           */
} bte_tuning;

typedef struct bte_handle bte_handle;

/* Device bytes a handle needs for these parameters and launch shape
 * (state ping-pong, tables, trace, reduction scratch). */
BTE_API int bte_workspace_size(const bte_params* p, const bte_tuning* tune, size_t* bytes);

/* Creates a solver, initialises f = f0 (a_n = a0_n, b_n = 0; Sec. 2) and
 * runs the start-up half step (Sec. 3: z^{1/2} = T with dt/2).
 *   stream : cudaStream_t to queue work on, or NULL for a stream the handle
 *            creates.
 * On success *out owns its device memory. */
BTE_API int bte_create(const bte_params* p, void* stream, bte_handle** out);

/* As bte_create with an explicit launch shape and, when workspace != NULL,
 * caller-owned DEVICE memory of workspace_bytes >= bte_workspace_size()
 * bytes (256-byte aligned) used instead of cudaMalloc.  The caller keeps the
 * workspace alive until bte_destroy. */
BTE_API int bte_create_ex(const bte_params* p, void* stream, const bte_tuning* tune,
                  void* workspace, size_t workspace_bytes, bte_handle** out);

/* Queues a return to the initial state of bte_create (f = f0, start-up half
 * step, step index 0, trace and error word cleared) without reallocating. */
BTE_API int bte_reset(bte_handle* h);

/* Queues nsteps leap-frog steps (Eqs. leap_frog_1, leap_frog_2) after the
 * current one.  BTE_ESTATE if that would pass steps_total. */
BTE_API int bte_step(bte_handle* h, int64_t nsteps);

/* Queues the remaining steps of the run (to steps_total). */
BTE_API int bte_run(bte_handle* h);

/* Waits for queued work and fills *out; the window results are final once
 * step == steps_total.  Returns the run status (BTE_EUNSTABLE when a NaN,
 * an Inf or |norm - 1| > 0.05 was seen; BTE_ETIMEOUT after a bounded wait in
 * a kernel gave up). */
BTE_API int bte_observables(bte_handle* h, bte_obs* out);

/* Exercises the failure detection of the bounded in-kernel waits without a
 * fault (the paper has no counterpart; failure handling is the library's
 * own).  Queues one kernel whose single thread waits on a shared-memory
 * mbarrier that nothing completes, bounded by limit_ns nanoseconds of the
 * GPU's %globaltimer (1 <= limit_ns <= 2e9; the solver kernels' own waits
 * give up after 2e9), and then records the timeout in the handle's error
 * word exactly as a solver kernel whose wait gave up does: bte_observables
 * returns BTE_ETIMEOUT (status BTE_ETIMEOUT) until bte_reset clears the
 * word.  No copy or other asynchronous work is in flight when the wait
 * gives up, and the context stays usable.  BTE_EINVAL for a NULL handle or
 * a limit out of range. */
BTE_API int bte_wait_probe(bte_handle* h, int64_t limit_ns);

/* Copies whole-grid samples k0..k0+count-1 of v_dr and norm (HOST arrays,
 * either may be NULL).  Samples beyond the current step are BTE_EINVAL. */
BTE_API int bte_trace(bte_handle* h, int64_t k0, int64_t count, double* v, double* norm);

/* State of one grid (0 = whole grid at step k, 1 = fractional grid at
 * k + 1/2) as HOST FP64 arrays a[n_max+1][m_points], b[n_max+1][m_points]
 * (row n, column m, row-major).  FP32 state is widened exactly. */
BTE_API int bte_get_state(bte_handle* h, int grid, double* a, double* b);

/* Overwrites one grid from HOST FP64 arrays laid out as in bte_get_state
 * (FP32 state rounds to nearest).  b[0][*] must be 0. */
BTE_API int bte_set_state(bte_handle* h, int grid, const double* a, const double* b);

/* Sets the current step index to k (0 <= k <= steps_total) and restores the
 * whole-grid samples 0..k (HOST arrays of length k+1) that the window
 * averages and norm error are computed from.  Used with bte_set_state to
 * resume from a checkpoint. */
BTE_API int bte_set_step(bte_handle* h, int64_t k, const double* v, const double* norm);

/* The distribution itself, f(phi_x, phi_y) = sum_{n=0}^{n_max} a_n(phi_y)
 * cos(n phi_x) + b_n(phi_y) sin(n phi_x) (Sec. 2, Eq. f_fourier; a_0 holds
 * the sigma_0 = 1/2 factor), of one grid (0 = whole grid at step k, 1 =
 * fractional grid) on nphix phi_x points -pi + 2 pi i / nphix (i = 0 ..
 * nphix-1) times the m_points phi_y grid, evaluated on the GPU in FP64:
 * HOST out [nphix][m_points].  1 <= nphix <= 65535; synchronises. */
BTE_API int bte_pdf(bte_handle* h, int grid, int32_t nphix, double* out);

/* Frees the handle and everything it allocated.  NULL is ignored. */
BTE_API void bte_destroy(bte_handle* h);

/* Message of the last failing call on this thread ("" if none). */
BTE_API const char* bte_last_error(void);

/* I_n(mu)/I_0(mu), n = 0..nmax, into HOST array r (Miller's backward
 * recurrence); the library's own equilibrium coefficients (Sec. 2,
 * Eq. Bolzmann_initial_pdf) come from it.  Host-only, needs no GPU. */
BTE_API int bte_bessel_ratio(double mu, int32_t nmax, double* r);

/* Time grid of a parameter set: dt_eff, steps per period P, total steps K,
 * window samples Kw (any pointer may be NULL).  Host-only. */
BTE_API int bte_time_grid(const bte_params* p, double* dt_eff, int64_t* P, int64_t* K,
                  int64_t* Kw);

/* Launch shape of the fused step kernel and row pitch (elements) of the
 * device arrays that bte_create_ex would choose for p and tune (any output
 * pointer may be NULL).  Host-only. */
BTE_API int bte_launch_shape(const bte_params* p, const bte_tuning* tune, int32_t* tile_m,
                             int32_t* chunk_n, int32_t* pitch, int32_t* grid_x,
                             int32_t* grid_y);

/* Drift velocity and norm (out[0] = pi sqrt(alpha) dphi sum_m b1_row[m],
 * out[1] = 2 pi sqrt(alpha) dphi sum_m a0_row[m]) of caller-owned DEVICE
 * rows a0_row (harmonic n = 0 of a) and b1_row (n = 1 of b), m_points
 * contiguous values each, FP64 when p->precision is BTE_FP64, else FP32;
 * out is a DEVICE array of 2 doubles.  Queued on `stream`; returns without
 * waiting.  The paper has no counterpart to this entry point: it exists for
 * callers that cannot allocate device memory (applications whose device
 * memory all belongs to their own pool allocator, host paths that cannot
 * afford the synchronisation an allocation may cause).  It allocates
 * nothing: its partial sums and arrival ticket live in one fixed array of
 * the library (16.6 KB per GPU, held until the process exits), so m_points
 * may be at most 1,048,576 (BTE_EINVAL beyond that, below 3, or for bad
 * parameters).  Its first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, with the device current); make that first
 * call before any stream capture.  Later calls outside capture look the
 * address up again (a device reset by the caller moves the array); calls
 * while `stream` is capturing reuse the address found by the device's last
 * call outside capture, so after a cudaDeviceReset make one call outside
 * capture before capturing again.  Every call shares the array and clears
 * the ticket before use; calls that overlap on the GPU race. */
BTE_API int bte_observe_noalloc(const bte_params* p, const void* a0_row, const void* b1_row,
                                double* out, void* stream);

/* Options of bte_batch_run (zero fields take the defaults given). */
typedef struct bte_batch_opts {
    int32_t tile_m;          /* phi_y columns per work item (0: 64 * vec)             */
    int32_t chunk_n;         /* harmonics per work item (0: 16)                       */
    int32_t vec;             /* columns per thread, 2 or 4 (0: 4 FP32, 2 FP64)        */
    int32_t graph_steps;     /* steps per captured CUDA graph (0: 1024)               */
    int32_t max_batch;       /* parameter points advanced together (0: 1024)          */
    int32_t resident;        /* 0: on chip where a point fits, 1: never, 2: only      */
    int64_t max_batch_bytes; /* device bytes one batch may hold (0: 4 GiB)            */
    void* stream;            /* cudaStream_t to queue on (NULL: a private stream)     */
    int32_t resident_smem;   /* shared memory per CTA for on-chip points, bytes
                                (0: 232,448, the most a CTA may have)                */
    int32_t walk;            /* row-walk order of the streamed tier, as
                                bte_tuning.walk (for the batch's total state)        */
} bte_batch_opts;

/* Full solve (Sec. 3 scheme from the Sec. 2 initial state, window averages
 * of Eq. absorption_def) of n independent parameter points p[0..n-1], as a
 * parameter sweep of the kind behind the paper's absorption and drift maps
 * (Sec. 4).  All points must share one precision; each keeps its own grid,
 * time step and run length.  Two tiers:
 *   on chip: a point whose four grid arrays fit the shared memory of a
 *     cluster of C = 1, 2, 4, 8 or 16 CTAs (resident_smem bytes each) is
 *     run start to end by one cluster with the state held in shared
 *     memory; clusters take points from a queue, longest first;
 *   streamed: the other points are grouped into batches (longest runs
 *     first, at most max_batch points and about max_batch_bytes of device
 *     memory each) that advance in lock-step, one fused launch per time
 *     step covering every point's tiles; a point whose run is over is
 *     skipped by later launches of its batch.
 * Both give the same per-cell arithmetic; the per-step sums over phi_y are
 * added in different orders.  out[i] receives the
 * final observables of p[i] exactly as bte_observables reports them after
 * bte_run (absorption NaN when omega == 0), with a per-point status
 * (BTE_OK, BTE_EUNSTABLE, BTE_ETIMEOUT).  Returns BTE_OK when every point
 * is OK, else the worst status; BTE_EINVAL (nothing run) for a bad point or
 * option, BTE_ENOMEM / BTE_ECUDA when device work fails (later points are
 * not run).  Blocks until done; allocates and frees its device memory. */
BTE_API int bte_batch_run(const bte_params* p, int32_t n, bte_obs* out,
                          const bte_batch_opts* opts);

/* The tier bte_batch_run would give each point (same validation, no GPU
 * work): tier[i] = CTAs per cluster of the on-chip tier (1..16) or 0 when
 * p[i] is streamed.  HOST arrays; BTE_EINVAL as bte_batch_run. */
BTE_API int bte_batch_plan(const bte_params* p, int32_t n, const bte_batch_opts* opts,
                           int32_t* tier);

/* Autotuner of bte_batch_run's options for a set of points.  Takes
 * `sample` of the points (evenly spaced in cost order, cost = cells x
 * steps), shortens their runs so that the longest has about `steps` time
 * steps (relative run lengths kept), and times bte_batch_run on them for 12
 * candidate option sets (each run once untimed, then timed): on-chip tier
 * with 232,448 / 160,000 / 113,664 bytes of shared memory per CTA, then the
 * streamed tier alone with tile_m = {32, 64, 128} x vec and chunk_n = {8, 16,
 * 32}.  *best receives the fastest (fields not tuned copied from *base,
 * which may be NULL); seconds (HOST, 12 values, may be NULL) the time of each
 * candidate in that order (1e300 where a candidate does not apply).
 * Synchronous; uses the GPU. */
BTE_API int bte_batch_tune(const bte_params* p, int32_t n, const bte_batch_opts* base,
                           int32_t sample, int32_t steps, bte_batch_opts* best, double* seconds);

/* Library version string. */
BTE_API const char* bte_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BTE_H */
