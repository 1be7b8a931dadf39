/*
 * bte_host.cpp -- host side of the C ABI declared in include/bte.h.
 *
 * Responsibilities: parameter validation, the time grid, the equilibrium
 * coefficients (Miller's backward recurrence for I_n(mu)/I_0(mu)), the drive
 * table, the device layout, kernel launch shapes, CUDA-graph capture of runs
 * of steps, state and trace transfers.  All arithmetic of a time step runs
 * in the kernels of bte_kernels.cu.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/bte.h"
#include "bte_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(BTE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

const double kTwoPi = 6.283185307179586476925286766559;
const double kPi = 3.14159265358979323846264338328;

struct TimeGrid {
    double dt_eff;
    long long P, K, Kw;
};

int validate(const bte_params* p) {
    if (!p) return fail(BTE_EINVAL, "params is NULL");
    const double v[] = {p->E_dc, p->E_omega, p->omega, p->B, p->mu, p->alpha,
                        p->phiy_min, p->phiy_max, p->dt, p->periods, p->t_max, p->avg_window,
                        p->B_omega, p->B_phase};
    for (double x : v)
        if (!std::isfinite(x)) return fail(BTE_EINVAL, "non-finite parameter");
    if (p->n_max < 1) return fail(BTE_EINVAL, "n_max must be >= 1");
    if (p->m_points < 3) return fail(BTE_EINVAL, "m_points must be >= 3");
    if (p->mu <= 0) return fail(BTE_EINVAL, "mu must be > 0");
    if (p->alpha <= 0) return fail(BTE_EINVAL, "alpha must be > 0");
    if (p->dt <= 0) return fail(BTE_EINVAL, "dt must be > 0");
    if (p->omega < 0) return fail(BTE_EINVAL, "omega must be >= 0");
    if (!(p->phiy_max > p->phiy_min)) return fail(BTE_EINVAL, "phiy_max must exceed phiy_min");
    if (p->avg_window < 0) return fail(BTE_EINVAL, "avg_window must be >= 0");
    if (p->precision != BTE_FP64 && p->precision != BTE_FP32_MIXED)
        return fail(BTE_EINVAL, "unknown precision %d", p->precision);
    if (p->reserved != 0) return fail(BTE_EINVAL, "reserved field must be 0");
    if (p->omega > 0) {
        if (p->periods <= 0) return fail(BTE_EINVAL, "periods must be > 0 when omega > 0");
        if (p->avg_window > p->periods) return fail(BTE_EINVAL, "avg_window exceeds the run");
    } else {
        if (p->t_max <= 0) return fail(BTE_EINVAL, "t_max must be > 0 when omega == 0");
        if (p->avg_window > p->t_max) return fail(BTE_EINVAL, "avg_window exceeds the run");
    }
    if ((long long)(p->n_max + 1) * (long long)p->m_points > (1ll << 31))
        return fail(BTE_EINVAL, "grid too large");
    return BTE_OK;
}

int time_grid(const bte_params* p, TimeGrid& g) {
    if (p->omega > 0) {
        const double Pd = std::nearbyint(kTwoPi / (p->omega * p->dt));
        if (!(Pd >= 1.0) || Pd > 1e9) return fail(BTE_EINVAL, "steps per period out of range");
        g.P = (long long)Pd;
        g.dt_eff = kTwoPi / (p->omega * (double)g.P);
        g.K = std::llround(p->periods * (double)g.P);
        g.Kw = std::llround(p->avg_window * (double)g.P);
    } else {
        g.P = 0;
        g.dt_eff = p->dt;
        g.K = std::llround(p->t_max / p->dt);
        g.Kw = std::llround(p->avg_window / p->dt);
    }
    if (g.K < 1 || g.K > (1ll << 40)) return fail(BTE_EINVAL, "run length out of range");
    if (g.Kw > g.K) g.Kw = g.K;
    if (g.Kw < 1) g.Kw = 1;
    return BTE_OK;
}

/* Miller's backward recurrence (J.C.P. Miller, 1952) for the minimal
 * solution of I_{n-1}(x) = (2n/x) I_n(x) + I_{n+1}(x): start far above the
 * highest order needed with (I_{s+1}, I_s) = (0, 1), recur downward and
 * divide by the I_0 obtained.  Values are rescaled when they grow large;
 * orders above nmax are not kept. */
void miller_ratio(double x, int nmax, double* r) {
    const int s = nmax + 32 + (int)std::ceil(x) + (int)std::ceil(8.0 * std::sqrt(x + nmax + 16.0));
    std::vector<double> I(nmax + 1, 0.0);
    double ip1 = 0.0, in = 1.0; /* I_{n+1}, I_n at n = s */
    for (int n = s; n >= 1; --n) {
        double im1 = (2.0 * n / x) * in + ip1;
        ip1 = in;
        in = im1;
        if (n - 1 <= nmax) I[n - 1] = im1;
        if (n <= nmax) I[n] = ip1;
        if (std::fabs(in) > 1e250) {
            in *= 1e-250;
            ip1 *= 1e-250;
            for (int q = std::max(n - 1, 0); q <= nmax; ++q) I[q] *= 1e-250;
        }
    }
    for (int n = 0; n <= nmax; ++n) r[n] = I[n] / I[0];
}

int pick_tile(const bte_params* p, const bte_tuning* t, int& tile_m, int& chunk_n, int& vec) {
    const int M1 = p->m_points, N1 = p->n_max + 1;
    const bool fp64 = p->precision == BTE_FP64;
    tile_m = (t && t->tile_m) ? t->tile_m : 0;
    chunk_n = (t && t->chunk_n) ? t->chunk_n : 0;
    vec = (t && t->vec) ? t->vec : (fp64 ? 2 : 4);
    if (vec != 2 && vec != 4) return fail(BTE_EINVAL, "vec must be 2 or 4");
    if (fp64 && vec != 2) return fail(BTE_EINVAL, "FP64 runs with vec = 2");
    if (tile_m) {
        if (tile_m % 4 || tile_m < 32 || tile_m > 1024)
            return fail(BTE_EINVAL, "tile_m must be a multiple of 4 in 32..1024");
    } else {
        /* whole warps of compute threads per item: w warps cover 32*vec*w
         * columns; pick w in 2..6 with the fewest warps over the grid's
         * width (the producer warp of each item counted as half a warp).
         * Grids of at most 512 columns use one-warp items so that several
         * SMs share them. */
        const int per_warp = 32 * vec;
        if (M1 <= 512) {
            tile_m = per_warp;
        } else {
            double best = 1e30;
            for (int w = 2; w <= 6; ++w) {
                const int t = per_warp * w;
                if (fp64 && t > 512) break;
                const int ntx = (M1 + t - 1) / t;
                const double cost = ntx * (w + 0.5);
                if (cost < best - 1e-9) {
                    best = cost;
                    tile_m = t;
                }
            }
        }
    }
    if (chunk_n) {
        if (chunk_n < 4) return fail(BTE_EINVAL, "chunk_n must be >= 4");
    } else {
        /* about one item per resident CTA (persistent launch): ~2 CTAs per
         * SM; at least 4 rows (8 when rows are plenty) */
        const int ntx = (M1 + tile_m - 1) / tile_m;
        const int slots = 304;
        const int rows_per = std::max(1, slots / ntx);
        chunk_n = (N1 + rows_per - 1) / rows_per;
        chunk_n = std::max(chunk_n, N1 >= 64 ? 8 : 4);
    }
    return BTE_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    int G, H, pitch, tile_m, chunk_n, vec, ts, ntx, nty;
    int resC;                 /* on-chip mode: CTAs of the cluster, 0 = streamed */
    bool persist;             /* persistent mode: one launch per call, grid barriers */
    int walk;                 /* tuning.walk: 0 automatic, 1 upward, 2 alternate */
    size_t res_smem, res_arrays; /* its shared memory per CTA, and the arrays' part */
    size_t elem;
    size_t off_state[8];
    size_t off_row_a0, off_col_g, off_col_phi, off_ew, off_ef, off_tv, off_tn, off_part,
        off_ticket, off_err, off_base, off_fin, off_res, off_done, total;
    int dring;                /* slots of the row-0 partial sums (persistent: ntx + 1) */
    /* on chip over several clusters (resident = 3; wideG = 0 otherwise):
     * G clusters of C CTAs, Wc columns per cluster, rp rows per CTA */
    int wideG, wideC, wideWc, wide_rp, wide_threads;
    size_t wide_smem;
    size_t off_wx, off_wpart;  /* tagged edge-column words, per-cluster sums */
    size_t wide_words;         /* bytes of the tagged words */
};

/* steps of one persistent launch at most (a bte_step/bte_run call of more
 * steps queues several launches) */
constexpr long long kPersistMaxSteps = 8192;

/* on chip over several clusters: shared memory per CTA at most, clusters
 * at most, and the automatic choice: about 32 (FP64) or 128 (FP32) columns
 * per cluster -- the FP64 arithmetic wants the most SMs, the FP32 steps the
 * fewest cross-cluster exchanges (31 x 201 on a GB300: FP64 6.8-7.5 us per
 * step with 7 clusters against 7.1-8.6 with 4; FP32 3.4-3.5 with 2 against
 * 3.5-3.9 with 4) -- with at most 128 CTAs in all, and at create time no
 * more clusters than fit the GPU at once */
constexpr size_t kWideSmemMax = 232448;
constexpr int kWideMaxClusters = 32;
constexpr int kWideAutoCtas = 128;
constexpr int kWideMaxCells = bte::kWideMaxThreads - 32; /* a block's cells: one thread each, plus a warp */
int wide_auto_cols(size_t elem) { return elem == 8 ? 32 : 128; }
size_t wide_need(size_t elem, int rp, int Wc) {
    return elem == 8 ? bte::wide_smem_bytes<double>(rp, Wc) : bte::wide_smem_bytes<float>(rp, Wc);
}
/* one thread per cell of the block, and one more warp (the row sums) */
int wide_threads(int rp, int Wc) { return (rp * Wc + 31) / 32 * 32 + 32; }

/* bytes of the on-chip mode's device record: the point's BatchInst, its
 * order entry and queue counter, and the kernel's window-sum scratch */
constexpr size_t kResBytes = 1024;
constexpr int kResThreads = 512; /* threads per CTA of the on-chip kernel */

int plan(const bte_params* p, const bte_tuning* t, const TimeGrid& tg, Layout& L) {
    if (t && (t->walk < 0 || t->walk > 2)) return fail(BTE_EINVAL, "tuning.walk must be 0, 1 or 2");
    if (t && (t->resident < 0 || t->resident > 3))
        return fail(BTE_EINVAL, "tuning.resident must be 0, 1, 2 or 3");
    if (t && (t->wide_cols < 0 || t->wide_cols > 4096))
        return fail(BTE_EINVAL, "tuning.wide_cols must be in 0..4096");
    int rc = pick_tile(p, t, L.tile_m, L.chunk_n, L.vec);
    if (rc) return rc;
    L.elem = p->precision == BTE_FP64 ? 8 : 4;
    /* on-chip mode: the largest cluster that leaves every CTA two rows and fits */
    L.resC = 0;
    L.res_smem = L.res_arrays = 0;
    L.persist = t && t->resident == 2;
    L.walk = t ? t->walk : 0;
    if (t && t->resident == 1) {
        const int N1 = p->n_max + 1;
        for (int C = 16; C >= 1; C /= 2) {
            if (C > 1 && (N1 + C - 1) / C < 2) continue;
            size_t arrays = 0;
            const size_t need = L.elem == 8
                                    ? bte::resident_smem_bytes<double>(p->n_max, p->m_points - 1, C, &arrays)
                                    : bte::resident_smem_bytes<float>(p->n_max, p->m_points - 1, C, &arrays);
            if (need <= 232448) {
                L.resC = C;
                L.res_smem = need;
                L.res_arrays = arrays;
                break;
            }
        }
        if (!L.resC)
            return fail(BTE_EINVAL, "grid %dx%d does not fit the shared memory of a 16-CTA cluster",
                        p->n_max + 1, p->m_points);
    }
    /* on chip over several clusters: C as for the on-chip mode (at least
     * two rows per CTA), then Wc columns per cluster (given, or about 32
     * with at most 128 CTAs, fewer columns while a block does not fit) */
    L.wideG = L.wideC = L.wideWc = L.wide_rp = L.wide_threads = 0;
    L.wide_smem = 0;
    if (t && t->resident == 3) {
        const int N1 = p->n_max + 1, M1 = p->m_points;
        const int auto_cols = wide_auto_cols(L.elem);
        auto need = [&](int rp, int Wc) { return wide_need(L.elem, rp, Wc); };
        for (int C = 16; C >= 1 && !L.wideG; C /= 2) {
            if (C > 1 && (N1 + C - 1) / C < 2) continue;
            const int rp = (N1 + C - 1) / C;
            int Wc = t->wide_cols;
            if (!Wc) {
                int G = std::min((M1 + auto_cols - 1) / auto_cols, std::max(1, kWideAutoCtas / C));
                G = std::max(G, 1);
                Wc = (M1 + G - 1) / G;
                while ((need(rp, Wc) > kWideSmemMax || rp * Wc > kWideMaxCells) &&
                       (M1 + Wc - 1) / Wc < kWideMaxClusters)
                    Wc = (M1 + (M1 + Wc - 1) / Wc) / ((M1 + Wc - 1) / Wc + 1);
            }
            const int G = (M1 + Wc - 1) / Wc;
            const size_t bytes = need(rp, Wc);
            /* one cell per thread: a block of at most kWideMaxCells cells */
            if (G > kWideMaxClusters || bytes > kWideSmemMax || rp * Wc > kWideMaxCells) continue;
            L.wideG = G;
            L.wideC = C;
            L.wideWc = Wc;
            L.wide_rp = rp;
            L.wide_smem = bytes;
            L.wide_threads = wide_threads(rp, Wc);
        }
        if (!L.wideG)
            return fail(BTE_EINVAL,
                        "grid %dx%d does not fit %d clusters of 16 CTAs (%zu bytes and %d cells each)",
                        N1, M1, kWideMaxClusters, kWideSmemMax, kWideMaxCells);
    }
    L.G = (int)(128 / L.elem);
    L.H = (int)(32 / L.elem); /* halo columns the step kernel streams per side */
    const int max_tile = L.elem == 8 ? bte::step_max_tile<double>(L.vec)
                                     : bte::step_max_tile<float>(L.vec);
    if (L.tile_m > max_tile) {
        if (t && t->tile_m) return fail(BTE_EINVAL, "tile_m %d above %d for this precision", L.tile_m, max_tile);
        L.tile_m = max_tile;
    }
    L.ts = 1; /* steps per launch */
    const size_t smem = L.elem == 8 ? bte::step_smem_bytes<double>(L.tile_m, L.chunk_n, L.vec)
                                    : bte::step_smem_bytes<float>(L.tile_m, L.chunk_n, L.vec);
    if (smem > 227 * 1024)
        return fail(BTE_EINVAL, "tile_m %d needs %zu bytes of shared memory", L.tile_m, smem);
    const int M1 = p->m_points, N1 = p->n_max + 1;
    L.ntx = (M1 + L.tile_m - 1) / L.tile_m;
    L.nty = (N1 + L.chunk_n - 1) / L.chunk_n;
    /* the last tile reads up to column G + ntx*tile_m + H - 1 */
    L.pitch = (int)align_up((size_t)(L.G + L.ntx * L.tile_m + L.H), 32);
    size_t o = 0;
    const size_t arr = align_up((size_t)N1 * L.pitch * L.elem, 256);
    for (int q = 0; q < 8; ++q) {
        L.off_state[q] = o;
        o += arr;
    }
    L.off_row_a0 = o;
    o += align_up((size_t)N1 * L.elem, 256);
    L.off_col_g = o;
    o += align_up((size_t)L.pitch * L.elem, 256);
    L.off_col_phi = o;
    o += align_up((size_t)L.pitch * L.elem, 256);
    const long long Pt = tg.P > 0 ? tg.P : 1;
    L.off_ew = o;
    o += align_up((size_t)3 * (Pt + 2) * L.elem, 256);
    L.off_ef = o;
    o += align_up((size_t)3 * (Pt + 2) * L.elem, 256);
    L.off_tv = o;
    o += align_up((size_t)(tg.K + 1) * 8, 256);
    L.off_tn = o;
    o += align_up((size_t)(tg.K + 1) * 8, 256);
    /* a persistent launch may have steps k .. k + ntx in flight at once (an
     * item's dependencies spread by one tile per step): that many slots */
    L.dring = L.persist ? L.ntx + 1 : 1;
    L.off_part = o;
    o += align_up((size_t)2 * L.dring * L.ntx * 8, 256);
    L.off_ticket = o;
    o += align_up((size_t)L.dring * sizeof(unsigned), 256);
    L.off_err = o;
    o += 256;
    L.off_base = o;
    o += 256;
    L.off_fin = o;
    o += 256;
    L.off_res = o;
    o += kResBytes;
    L.off_done = o;
    o += align_up((size_t)L.ntx * L.nty * sizeof(unsigned), 256);
    L.off_wx = L.off_wpart = o;
    L.wide_words = 0;
    if (L.wideG) {
        /* 2 buffers x 2 grids x 2 sides x 2 arrays x (elem / 4) words of 8
         * bytes per cluster and row */
        L.wide_words = (size_t)16 * (L.elem / 4) * L.wideG * N1 * 8;
        L.off_wx = o;
        o += align_up(L.wide_words, 256);
        L.off_wpart = o;
        o += align_up((size_t)kPersistMaxSteps * L.wideG * 2 * sizeof(double), 256);
    }
    L.total = o;
    return BTE_OK;
}

}  // namespace

struct bte_handle {
    bte_params p;
    TimeGrid tg;
    Layout L;
    bool fp64;
    bool own_mem;
    bool own_stream;
    unsigned char* mem;
    cudaStream_t stream;
    cudaStream_t cap_stream;
    long long k;   /* steps queued so far */
    long long base_host;
    int graph_len; /* steps per captured graph (a multiple of the fused step count) */
    int grid[3];   /* persistent CTAs of the step kernel fusing 1 / 2 steps */
    int grid_persist; /* CTAs of a persistent (multi-step) launch, all co-resident */
    int set;       /* ping-pong set holding the current state (flips per launch) */
    cudaGraphExec_t graph[2]; /* one graph per starting set */
    double r1;     /* I_1/I_0 */
    double dphi;
    template <typename T>
    T* ptr(size_t off) const {
        return reinterpret_cast<T*>(mem + off);
    }
};

namespace {

template <typename T>
bte::StepArgs<T> step_args(const bte_handle* h) {
    bte::StepArgs<T> a;
    const Layout& L = h->L;
    for (int s = 0; s < 2; ++s) {
        a.a_w[s] = h->ptr<T>(L.off_state[4 * s + 0]);
        a.b_w[s] = h->ptr<T>(L.off_state[4 * s + 1]);
        a.a_f[s] = h->ptr<T>(L.off_state[4 * s + 2]);
        a.b_f[s] = h->ptr<T>(L.off_state[4 * s + 3]);
    }
    a.row_a0 = h->ptr<T>(L.off_row_a0);
    a.col_g = h->ptr<T>(L.off_col_g);
    a.col_phi = h->ptr<T>(L.off_col_phi);
    a.e_whole = h->ptr<T>(L.off_ew);
    a.e_frac = h->ptr<T>(L.off_ef);
    a.base = h->ptr<long long>(L.off_base);
    a.trace_v = h->ptr<double>(L.off_tv);
    a.trace_n = h->ptr<double>(L.off_tn);
    a.part = h->ptr<double>(L.off_part);
    a.ticket = h->ptr<unsigned>(L.off_ticket);
    a.err = h->ptr<int>(L.off_err);
    a.done = h->ptr<unsigned>(L.off_done);
    a.dring = L.dring;
    a.nsteps = 0;
    a.N = h->p.n_max;
    a.M = h->p.m_points - 1;
    a.pitch = L.pitch;
    a.P = h->tg.P > 0 ? (int)h->tg.P : 1;
    a.dstride = a.P + 2;
    a.tile_m = L.tile_m;
    a.chunk_n = L.chunk_n;
    a.ntx = L.ntx;
    a.nty = L.nty;
    a.vec = L.vec;
    a.grid = h->grid[L.ts];
    a.alt = L.walk == 2 ||
            (L.walk == 0 && 8 * L.elem * (size_t)(h->p.n_max + 1) * (size_t)L.pitch > bte::kAltStateBytes);
    const double dt = h->tg.dt_eff;
    a.h = (T)dt;
    a.hh = (T)(0.5 * dt);
    a.nu = (T)(1.0 + 0.5 * dt);
    a.xi = (T)(1.0 - 0.5 * dt);
    const double sq = std::sqrt(h->p.alpha);
    a.vscale = kPi * sq * h->dphi;
    a.nscale = 2.0 * kPi * sq * h->dphi;
    return a;
}

/* Host tables of one instance (Sec. 2): row factors sigma_n I_n/(pi I_0),
 * column factors sqrt(mu/(2 pi alpha)) exp(-mu phi^2/2) and phi_m laid out
 * with G ghost columns, and the drive (FP64, rounded to T once) over one
 * period plus two entries
 * in two [3][P+2] tables: at the whole-grid times i dt (ew) and the
 * fractional-grid times (i + 1/2) dt (ef), E(t) (Sec. 2, E(t) = E_dc +
 * E_omega cos(omega t)), B(t) = B + B_omega cos(omega t + B_phase), and the
 * stencil coefficient B dt/(4 dphi) of the half-step starting at t, with B
 * taken at the time of the other grid, t + dt/2. */
template <typename T>
void build_tables(const bte_params& p, const TimeGrid& tg, int G, int pitch, double dphi,
                  std::vector<T>& row, std::vector<T>& colg, std::vector<T>& colp,
                  std::vector<T>& ew, std::vector<T>& ef, double& r1) {
    const int N1 = p.n_max + 1, M1 = p.m_points;
    std::vector<double> r(N1);
    miller_ratio(p.mu, p.n_max, r.data());
    r1 = r[1];
    row.assign(N1, (T)0);
    colg.assign(pitch, (T)0);
    colp.assign(pitch, (T)0);
    for (int n = 0; n < N1; ++n) row[n] = (T)((n == 0 ? 0.5 : 1.0) * r[n] / kPi);
    const double pref = std::sqrt(p.mu / (2.0 * kPi * p.alpha));
    for (int m = 0; m < M1; ++m) {
        const double phi = p.phiy_min + m * dphi;
        colg[G + m] = (T)(pref * std::exp(-0.5 * p.mu * phi * phi));
        colp[G + m] = (T)phi;
    }
    const long long Pt = tg.P > 0 ? tg.P : 1;
    const long long S = Pt + 2;
    ew.assign(3 * S, (T)0);
    ef.assign(3 * S, (T)0);
    const double dt = tg.dt_eff;
    /* drive phase of time (q + s/2) dt: 2 pi (q + s/2)/P, or 0 when omega == 0 */
    auto ph = [&](long long q, int s) {
        return tg.P > 0 ? kTwoPi * ((double)q + 0.5 * s) / (double)Pt : 0.0;
    };
    auto Bt = [&](double x) { return p.B + p.B_omega * std::cos(x + p.B_phase); };
    for (long long q = 0; q < S; ++q) {
        ew[q] = (T)(p.E_dc + p.E_omega * std::cos(ph(q, 0)));
        ef[q] = (T)(p.E_dc + p.E_omega * std::cos(ph(q, 1)));
        ew[S + q] = (T)Bt(ph(q, 0));
        ef[S + q] = (T)Bt(ph(q, 1));
        ew[2 * S + q] = (T)(Bt(ph(q, 1)) * dt / (4.0 * dphi));
        ef[2 * S + q] = (T)(Bt(ph(q, 2)) * dt / (4.0 * dphi));
    }
}

/* Start-up half step (Sec. 3, reading R6): T with dt/2 from t = 0, the
 * initial state as its own stencil source, so the stencil coefficient takes
 * B(0); the rotation takes E and B at 0 and dt/2. */
template <typename T>
void startup_drive(const bte_params& p, double dt_eff, double dphi, bte::ApplyArgs<T>& a) {
    const double hs = 0.5 * dt_eff;
    a.E_start = p.E_dc + p.E_omega;
    a.E_end = p.E_dc + p.E_omega * std::cos(p.omega * hs);
    a.B_start = p.B + p.B_omega * std::cos(p.B_phase);
    a.B_end = p.B + p.B_omega * std::cos(p.omega * hs + p.B_phase);
    a.h = (T)hs;
    a.hh = (T)(0.5 * hs);
    a.nu = (T)(1.0 + 0.5 * hs);
    a.xi = (T)(1.0 - 0.5 * hs);
    a.c = (T)(a.B_start * hs / (4.0 * dphi));
}

template <typename T>
int upload_tables(bte_handle* h) {
    const Layout& L = h->L;
    const int N1 = h->p.n_max + 1;
    std::vector<T> row, colg, colp, ew, ef;
    build_tables<T>(h->p, h->tg, L.G, L.pitch, h->dphi, row, colg, colp, ew, ef, h->r1);
    const long long Pt = h->tg.P > 0 ? h->tg.P : 1;
    CU(cudaMemcpyAsync(h->ptr<T>(L.off_row_a0), row.data(), N1 * sizeof(T), cudaMemcpyHostToDevice,
                       h->stream));
    CU(cudaMemcpyAsync(h->ptr<T>(L.off_col_g), colg.data(), L.pitch * sizeof(T),
                       cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->ptr<T>(L.off_col_phi), colp.data(), L.pitch * sizeof(T),
                       cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->ptr<T>(L.off_ew), ew.data(), 3 * (Pt + 2) * sizeof(T), cudaMemcpyHostToDevice,
                       h->stream));
    CU(cudaMemcpyAsync(h->ptr<T>(L.off_ef), ef.data(), 3 * (Pt + 2) * sizeof(T), cudaMemcpyHostToDevice,
                       h->stream));
    CU(cudaStreamSynchronize(h->stream)); /* host vectors go out of scope */
    return BTE_OK;
}

/* f = f0 on the whole grid, then z^{1/2} = T_{dt/2}(z^0; S(z^0)) (Sec. 3).
 * `full` clears every buffer (creation); otherwise only the counters and the
 * error word are cleared, since the kernels rewrite every interior cell and
 * never write ghost cells. */
template <typename T>
int initialise(bte_handle* h, bool full, bool sync) {
    const Layout& L = h->L;
    const bte_params& p = h->p;
    if (full) {
        CU(cudaMemsetAsync(h->mem, 0, L.off_row_a0, h->stream));
        CU(cudaMemsetAsync(h->mem + L.off_tv, 0, L.off_fin + 256 - L.off_tv, h->stream));
    } else {
        CU(cudaMemsetAsync(h->mem + L.off_ticket, 0, L.off_fin - L.off_ticket, h->stream));
    }
    T* aw = h->ptr<T>(L.off_state[0]);
    T* bw = h->ptr<T>(L.off_state[1]);
    int rc = bte::launch_init<T>(aw, bw, h->ptr<T>(L.off_row_a0), h->ptr<T>(L.off_col_g), p.n_max,
                                 p.m_points - 1, L.pitch, h->stream);
    if (rc) return fail(BTE_ECUDA, "init kernel: %s", cudaGetErrorString((cudaError_t)rc));
    bte::ApplyArgs<T> a;
    a.a = aw;
    a.b = bw;
    a.as = aw;
    a.bs = bw;
    a.an = h->ptr<T>(L.off_state[2]);
    a.bn = h->ptr<T>(L.off_state[3]);
    a.row_a0 = h->ptr<T>(L.off_row_a0);
    a.col_g = h->ptr<T>(L.off_col_g);
    a.col_phi = h->ptr<T>(L.off_col_phi);
    a.N = p.n_max;
    a.M = p.m_points - 1;
    a.pitch = L.pitch;
    startup_drive<T>(p, h->tg.dt_eff, h->dphi, a);
    rc = bte::launch_apply<T>(a, h->stream);
    if (rc) return fail(BTE_ECUDA, "start-up kernel: %s", cudaGetErrorString((cudaError_t)rc));
    const bte::StepArgs<T> sa = step_args<T>(h);
    rc = bte::launch_observe<T>(aw, bw, p.m_points - 1, L.pitch, sa.vscale, sa.nscale, sa.trace_v,
                                sa.trace_n, 0, h->stream);
    if (rc) return fail(BTE_ECUDA, "observe kernel: %s", cudaGetErrorString((cudaError_t)rc));
    h->k = 0;
    h->set = 0;
    h->base_host = 0;
    if (sync) CU(cudaStreamSynchronize(h->stream));
    return BTE_OK;
}

template <typename T>
int capture_graph(bte_handle* h, int set) {
    const bte::StepArgs<T> a = step_args<T>(h);
    long long* base = h->ptr<long long>(h->L.off_base);
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    for (int i = 0; i < h->graph_len && !rc; ++i)
        rc = bte::launch_step<T>(a, i, set, i > 0, h->cap_stream);
    if (!rc) rc = bte::launch_advance_base(base, h->graph_len, h->cap_stream);
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(BTE_ECUDA, "graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : (cudaError_t)rc));
    }
    e = cudaGraphInstantiate(&h->graph[set], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph[set] = nullptr;
        return fail(BTE_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    return BTE_OK;
}

/* On-chip mode: one persistent launch of the on-chip kernel (one cluster,
 * one point) advances the current ping-pong set n steps in place, writing
 * the per-step samples into the trace; the set does not change. */
template <typename T>
int enqueue_resident(bte_handle* h, long long n) {
    const Layout& L = h->L;
    const int set = h->set;
    unsigned char* res = h->mem + L.off_res;
    bte::BatchInst<T> R{};
    static_assert(sizeof(R) <= 448, "record region");
    for (int s = 0; s < 2; ++s) {
        R.a_w[s] = h->ptr<T>(L.off_state[4 * set + 0]);
        R.b_w[s] = h->ptr<T>(L.off_state[4 * set + 1]);
        R.a_f[s] = h->ptr<T>(L.off_state[4 * set + 2]);
        R.b_f[s] = h->ptr<T>(L.off_state[4 * set + 3]);
    }
    R.row_a0 = h->ptr<T>(L.off_row_a0);
    R.col_g = h->ptr<T>(L.off_col_g);
    R.col_phi = h->ptr<T>(L.off_col_phi);
    R.e_whole = h->ptr<T>(L.off_ew);
    R.e_frac = h->ptr<T>(L.off_ef);
    R.part = h->ptr<double>(L.off_part);
    R.ticket = h->ptr<unsigned>(L.off_ticket);
    R.acc = reinterpret_cast<double*>(res + 512); /* window sums: scratch here */
    R.K = n;
    R.Kw = 0;
    R.k0 = h->k;
    R.trace_v = h->ptr<double>(L.off_tv);
    R.trace_n = h->ptr<double>(L.off_tn);
    R.N = h->p.n_max;
    R.M = h->p.m_points - 1;
    R.pitch = L.pitch;
    R.P = h->tg.P > 0 ? (int)h->tg.P : 0;
    R.dstride = (h->tg.P > 0 ? (int)h->tg.P : 1) + 2;
    R.ntx = L.ntx;
    R.nty = L.nty;
    R.item0 = 0;
    const double dt = h->tg.dt_eff;
    R.h = (T)dt;
    R.hh = (T)(0.5 * dt);
    R.nu = (T)(1.0 + 0.5 * dt);
    R.xi = (T)(1.0 - 0.5 * dt);
    const double sq = std::sqrt(h->p.alpha);
    R.vscale = kPi * sq * h->dphi;
    R.nscale = 2.0 * kPi * sq * h->dphi;
    R.omega = h->p.omega;
    R.dt_eff = dt;
    /* pageable source: staged before the call returns */
    CU(cudaMemcpyAsync(res, &R, sizeof R, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemsetAsync(res + 448, 0, 64, h->stream)); /* order[0] = 0, queue = 0 */
    bte::ResArgs<T> ra{};
    ra.inst = reinterpret_cast<const bte::BatchInst<T>*>(res);
    ra.order = reinterpret_cast<const int*>(res + 448);
    ra.count = 1;
    ra.queue = reinterpret_cast<unsigned*>(res + 452);
    ra.C = L.resC;
    ra.red_off = L.res_arrays;
    /* the kernel's shared-memory attribute is per function: another handle or
     * a batched run may have set it since this handle was created */
    int clusters = 0;
    int rc = bte::resident_max_clusters<T>(L.resC, L.res_smem, kResThreads, &clusters);
    if (!rc) rc = bte::launch_resident<T>(ra, 1, kResThreads, L.res_smem, h->stream);
    if (!rc) rc = bte::launch_advance_base(h->ptr<long long>(L.off_base), n, h->stream);
    if (rc) return fail(BTE_ECUDA, "on-chip step kernel: %s", cudaGetErrorString((cudaError_t)rc));
    h->k += n;
    return BTE_OK;
}

/* On chip over several clusters: launches of at most kPersistMaxSteps
 * steps, each one launch of G clusters that advances the current ping-pong
 * set in place (counters zeroed before it), then the fold of the
 * per-cluster row sums into the trace. */
template <typename T>
int enqueue_wide(bte_handle* h, long long n) {
    const Layout& L = h->L;
    const int set = h->set;
    bte::WideArgs<T> w{};
    w.a_w = h->ptr<T>(L.off_state[4 * set + 0]);
    w.b_w = h->ptr<T>(L.off_state[4 * set + 1]);
    w.a_f = h->ptr<T>(L.off_state[4 * set + 2]);
    w.b_f = h->ptr<T>(L.off_state[4 * set + 3]);
    w.row_a0 = h->ptr<T>(L.off_row_a0);
    w.col_g = h->ptr<T>(L.off_col_g);
    w.col_phi = h->ptr<T>(L.off_col_phi);
    w.e_whole = h->ptr<T>(L.off_ew);
    w.e_frac = h->ptr<T>(L.off_ef);
    w.xw = h->ptr<unsigned long long>(L.off_wx);
    w.part = h->ptr<double>(L.off_wpart);
    w.err = h->ptr<int>(L.off_err);
    w.N = h->p.n_max;
    w.M = h->p.m_points - 1;
    w.pitch = L.pitch;
    w.P = h->tg.P > 0 ? (int)h->tg.P : 0;
    w.dstride = (h->tg.P > 0 ? (int)h->tg.P : 1) + 2;
    w.C = L.wideC;
    w.G = L.wideG;
    w.Wc = L.wideWc;
    w.rows_per = L.wide_rp;
    const double dt = h->tg.dt_eff;
    w.h = (T)dt;
    w.hh = (T)(0.5 * dt);
    w.nu = (T)(1.0 + 0.5 * dt);
    w.xi = (T)(1.0 - 0.5 * dt);
    const double sq = std::sqrt(h->p.alpha);
    const double vscale = kPi * sq * h->dphi, nscale = 2.0 * kPi * sq * h->dphi;
    while (n > 0) {
        const long long c = n < kPersistMaxSteps ? n : kPersistMaxSteps;
        w.K = c;
        w.k0 = h->k;
        CU(cudaMemsetAsync(w.xw, 0, L.wide_words, h->stream)); /* no tag left from an earlier launch */
        int rc = bte::launch_wide<T>(w, L.wide_threads, L.wide_smem, h->stream);
        if (!rc)
            rc = bte::launch_wide_fold(w.part, L.wideG, c, h->k, vscale, nscale,
                                       h->ptr<double>(L.off_tv), h->ptr<double>(L.off_tn), h->stream);
        if (!rc) rc = bte::launch_advance_base(h->ptr<long long>(L.off_base), c, h->stream);
        if (rc) return fail(BTE_ECUDA, "on-chip kernel over clusters: %s", cudaGetErrorString((cudaError_t)rc));
        h->k += c;
        n -= c;
    }
    return BTE_OK;
}

/* Queues n steps: whole graphs of graph_len steps (one graph per starting
 * ping-pong set, captured on first use), then single launches.  Every launch
 * advances one step and flips the ping-pong set; launches after the first of
 * a run use programmatic dependent launch. */
/* Persistent mode: launches of at most kPersistMaxSteps steps, each one
 * cooperative launch of one CTA per work item that advances every step,
 * an item starting a step once its neighbours have finished the step
 * before (their completion counters zeroed before the launch). */
template <typename T>
int enqueue_persist(bte_handle* h, long long n) {
    bte::StepArgs<T> a = step_args<T>(h);
    a.grid = h->grid_persist;
    while (n > 0) {
        const long long c = n < kPersistMaxSteps ? n : kPersistMaxSteps;
        a.nsteps = (int)c;
        CU(cudaMemsetAsync(a.done, 0, (size_t)h->L.ntx * h->L.nty * sizeof(unsigned), h->stream));
        int rc = bte::launch_step_persist<T>(a, h->set, h->stream);
        if (!rc) rc = bte::launch_advance_base(h->ptr<long long>(h->L.off_base), c, h->stream);
        if (rc) return fail(BTE_ECUDA, "persistent step kernel: %s", cudaGetErrorString((cudaError_t)rc));
        h->k += c;
        h->set ^= (int)(c & 1);
        n -= c;
    }
    return BTE_OK;
}

template <typename T>
int enqueue_steps(bte_handle* h, long long n) {
    if (h->L.resC) return n > 0 ? enqueue_resident<T>(h, n) : BTE_OK;
    if (h->L.wideG) return n > 0 ? enqueue_wide<T>(h, n) : BTE_OK;
    if (h->L.persist) return enqueue_persist<T>(h, n);
    while (h->graph_len >= 2 && n >= h->graph_len) {
        const int set = h->set;
        if (!h->graph[set]) {
            int rc = capture_graph<T>(h, set);
            if (rc) return rc;
        }
        CU(cudaGraphLaunch(h->graph[set], h->stream));
        n -= h->graph_len;
        h->k += h->graph_len;
        h->set ^= h->graph_len & 1;
    }
    if (n > 0) {
        const bte::StepArgs<T> a = step_args<T>(h);
        const int set = h->set;
        int rc = 0;
        for (long long i = 0; i < n && !rc; ++i)
            rc = bte::launch_step<T>(a, (int)i, set, i > 0, h->stream);
        if (!rc) rc = bte::launch_advance_base(h->ptr<long long>(h->L.off_base), n, h->stream);
        if (rc) return fail(BTE_ECUDA, "step kernel: %s", cudaGetErrorString((cudaError_t)rc));
        h->k += n;
        h->set ^= (int)(n & 1);
    }
    return BTE_OK;
}

template <typename T>
int get_grid(bte_handle* h, int grid, double* a, double* b) {
    const Layout& L = h->L;
    const int set = h->set;
    const int N1 = h->p.n_max + 1, M1 = h->p.m_points;
    const T* da = h->ptr<T>(L.off_state[4 * set + 2 * grid + 0]);
    const T* db = h->ptr<T>(L.off_state[4 * set + 2 * grid + 1]);
    std::vector<T> buf((size_t)N1 * M1);
    for (int which = 0; which < 2; ++which) {
        const T* src = which ? db : da;
        double* dst = which ? b : a;
        if (!dst) continue;
        CU(cudaMemcpy2DAsync(buf.data(), M1 * sizeof(T), src + L.G, L.pitch * sizeof(T),
                             M1 * sizeof(T), N1, cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        for (size_t q = 0; q < buf.size(); ++q) dst[q] = (double)buf[q];
    }
    return BTE_OK;
}

template <typename T>
int set_grid(bte_handle* h, int grid, const double* a, const double* b) {
    const Layout& L = h->L;
    const int set = h->set;
    const int N1 = h->p.n_max + 1, M1 = h->p.m_points;
    for (int m = 0; m < M1; ++m)
        if (b[m] != 0.0) return fail(BTE_EINVAL, "b[0][*] must be 0 (Eq. b_boundary)");
    std::vector<T> buf((size_t)N1 * M1);
    for (int which = 0; which < 2; ++which) {
        const double* src = which ? b : a;
        T* dst = h->ptr<T>(L.off_state[4 * set + 2 * grid + which]);
        for (size_t q = 0; q < buf.size(); ++q) buf[q] = (T)src[q];
        CU(cudaMemcpy2DAsync(dst + L.G, L.pitch * sizeof(T), buf.data(), M1 * sizeof(T),
                             M1 * sizeof(T), N1, cudaMemcpyHostToDevice, h->stream));
        CU(cudaStreamSynchronize(h->stream));
    }
    return BTE_OK;
}

}  // namespace

/* ---------------------------------------------------------------------- */
/* batched sweep                                                           */
/* ---------------------------------------------------------------------- */
namespace {

struct BatchPoint {
    int idx; /* position in the caller's array */
    int resC; /* CTAs per cluster of the on-chip tier, 0: streamed */
    TimeGrid tg;
    int N1, M1, ntx, nty, pitch, items;
    double dphi;
    size_t state_off, state_bytes, tab_off; /* within the batch workspace */
    size_t o_row, o_colg, o_colp, o_ew, o_ef, o_part, o_ticket, o_acc; /* within the tables */
    size_t tab_bytes;
    double r1;
};

constexpr int kAcc = 8; /* per-instance accumulators, see BatchInst::acc */

/* Runs points [first, last) of `pts` as one batch: advancing in lock-step,
 * or (resident) on chip, one cluster of pts[i].resC CTAs per point. */
template <typename T>
int run_batch(const bte_params* p, std::vector<BatchPoint>& pts, size_t first, size_t last,
              int tile, int chunk, int vec, int graph_len, bool resident, int walk, cudaStream_t st,
              cudaStream_t cap, bte_obs* out) {
    const int elem = (int)sizeof(T);
    const int G = 128 / elem, Hp = 32 / elem;
    /* layout: [all states][all tables, accumulators][records][counter, error] */
    size_t o = 0;
    int items = 0;
    long long Kmax = 0;
    for (size_t i = first; i < last; ++i) {
        BatchPoint& b = pts[i];
        b.pitch = (int)align_up((size_t)(G + b.ntx * tile + Hp), 32);
        b.state_bytes = align_up((size_t)b.N1 * b.pitch * elem, 256);
        b.state_off = o;
        o += (resident ? 4 : 8) * b.state_bytes; /* on chip: no ping-pong set */
        b.items = b.ntx * b.nty;
        items += b.items;
        Kmax = std::max(Kmax, b.tg.K);
    }
    const size_t states_end = o;
    for (size_t i = first; i < last; ++i) {
        BatchPoint& b = pts[i];
        const long long Pt = b.tg.P > 0 ? b.tg.P : 1;
        size_t t = 0;
        b.o_row = t;
        t += align_up((size_t)b.N1 * elem, 256);
        b.o_colg = t;
        t += align_up((size_t)b.pitch * elem, 256);
        b.o_colp = t;
        t += align_up((size_t)b.pitch * elem, 256);
        b.o_ew = t;
        t += align_up((size_t)3 * (Pt + 2) * elem, 256);
        b.o_ef = t;
        t += align_up((size_t)3 * (Pt + 2) * elem, 256);
        b.o_part = t;
        t += align_up((size_t)2 * b.ntx * 8, 256);
        b.o_ticket = t;
        t += 256;
        b.o_acc = t;
        t += 256;
        b.tab_bytes = t;
        b.tab_off = o;
        o += t;
    }
    const size_t tables_begin = states_end, tables_end = o;
    const size_t n = last - first;
    const size_t rec_off = align_up(o, 256);
    o = rec_off + align_up(n * sizeof(bte::BatchInst<T>), 256);
    const size_t map_off = o;
    o += align_up((size_t)items * sizeof(int), 256);
    const size_t base_off = o;
    o += 256;
    const size_t err_off = o;
    o += 256;
    const size_t total = o;

    unsigned char* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BTE_ENOMEM, "batch workspace of %zu bytes: %s", total, cudaGetErrorString(e));
    }
    std::vector<unsigned char> host(tables_end - tables_begin, 0);
    std::vector<bte::BatchInst<T>> rec(n);
    std::vector<int> item_inst;
    item_inst.reserve(items);
    int rc = BTE_OK;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        for (auto& g : graph)
            if (g) cudaGraphExecDestroy(g);
        cudaStreamSynchronize(st);
        cudaFree(mem);
    };
    int item0 = 0;
    for (size_t i = first; i < last; ++i) {
        BatchPoint& b = pts[i];
        const bte_params& pp = p[b.idx];
        std::vector<T> row, colg, colp, ew, ef;
        build_tables<T>(pp, b.tg, G, b.pitch, b.dphi, row, colg, colp, ew, ef, b.r1);
        unsigned char* hb = host.data() + (b.tab_off - tables_begin);
        std::memcpy(hb + b.o_row, row.data(), row.size() * elem);
        std::memcpy(hb + b.o_colg, colg.data(), colg.size() * elem);
        std::memcpy(hb + b.o_colp, colp.data(), colp.size() * elem);
        std::memcpy(hb + b.o_ew, ew.data(), ew.size() * elem);
        std::memcpy(hb + b.o_ef, ef.data(), ef.size() * elem);
        unsigned char* tb = mem + b.tab_off;
        bte::BatchInst<T>& R = rec[i - first];
        for (int s = 0; s < 2; ++s) {
            const int ss = resident ? 0 : s;
            R.a_w[s] = reinterpret_cast<T*>(mem + b.state_off + (4 * ss + 0) * b.state_bytes);
            R.b_w[s] = reinterpret_cast<T*>(mem + b.state_off + (4 * ss + 1) * b.state_bytes);
            R.a_f[s] = reinterpret_cast<T*>(mem + b.state_off + (4 * ss + 2) * b.state_bytes);
            R.b_f[s] = reinterpret_cast<T*>(mem + b.state_off + (4 * ss + 3) * b.state_bytes);
        }
        R.row_a0 = reinterpret_cast<const T*>(tb + b.o_row);
        R.col_g = reinterpret_cast<const T*>(tb + b.o_colg);
        R.col_phi = reinterpret_cast<const T*>(tb + b.o_colp);
        R.e_whole = reinterpret_cast<const T*>(tb + b.o_ew);
        R.e_frac = reinterpret_cast<const T*>(tb + b.o_ef);
        R.part = reinterpret_cast<double*>(tb + b.o_part);
        R.ticket = reinterpret_cast<unsigned*>(tb + b.o_ticket);
        R.acc = reinterpret_cast<double*>(tb + b.o_acc);
        R.K = b.tg.K;
        R.Kw = b.tg.Kw;
        R.N = b.N1 - 1;
        R.M = b.M1 - 1;
        R.pitch = b.pitch;
        R.P = b.tg.P > 0 ? (int)b.tg.P : 1;
        R.dstride = R.P + 2;
        R.ntx = b.ntx;
        R.nty = b.nty;
        R.item0 = item0;
        item0 += b.items;
        item_inst.insert(item_inst.end(), (size_t)b.items, (int)(i - first));
        const double dt = b.tg.dt_eff;
        R.h = (T)dt;
        R.hh = (T)(0.5 * dt);
        R.nu = (T)(1.0 + 0.5 * dt);
        R.xi = (T)(1.0 - 0.5 * dt);
        const double sq = std::sqrt(pp.alpha);
        R.vscale = kPi * sq * b.dphi;
        R.nscale = 2.0 * kPi * sq * b.dphi;
        R.omega = pp.omega;
        R.dt_eff = dt;
        /* window angle: P > 0 uses 2 pi (k mod P)/P; omega == 0 has no window angle */
        if (b.tg.P == 0) R.P = 0;
    }
#define BCU(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            rc = fail(BTE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));          \
            cleanup();                                                                     \
            return rc;                                                                     \
        }                                                                                  \
    } while (0)
    BCU(cudaMemsetAsync(mem, 0, states_end, st));
    BCU(cudaMemcpyAsync(mem + tables_begin, host.data(), host.size(), cudaMemcpyHostToDevice, st));
    BCU(cudaMemcpyAsync(mem + rec_off, rec.data(), n * sizeof(bte::BatchInst<T>),
                        cudaMemcpyHostToDevice, st));
    BCU(cudaMemcpyAsync(mem + map_off, item_inst.data(), (size_t)items * sizeof(int),
                        cudaMemcpyHostToDevice, st));
    BCU(cudaMemsetAsync(mem + base_off, 0, 512, st));
    /* initial state and start-up half step of every instance (Sec. 2, Sec. 3) */
    for (size_t i = first; i < last; ++i) {
        const BatchPoint& b = pts[i];
        const bte_params& pp = p[b.idx];
        const bte::BatchInst<T>& R = rec[i - first];
        int r = bte::launch_init<T>(R.a_w[0], R.b_w[0], R.row_a0, R.col_g, R.N, R.M, R.pitch, st);
        bte::ApplyArgs<T> a;
        a.a = R.a_w[0];
        a.b = R.b_w[0];
        a.as = R.a_w[0];
        a.bs = R.b_w[0];
        a.an = R.a_f[0];
        a.bn = R.b_f[0];
        a.row_a0 = R.row_a0;
        a.col_g = R.col_g;
        a.col_phi = R.col_phi;
        a.N = R.N;
        a.M = R.M;
        a.pitch = R.pitch;
        startup_drive<T>(pp, b.tg.dt_eff, b.dphi, a);
        if (!r) r = bte::launch_apply<T>(a, st);
        if (!r)
            r = bte::launch_observe<T>(R.a_w[0], R.b_w[0], R.M, R.pitch, R.vscale, R.nscale,
                                       R.acc + 6, R.acc + 7, 0, st);
        if (r) {
            rc = fail(BTE_ECUDA, "batch initialisation: %s", cudaGetErrorString((cudaError_t)r));
            cleanup();
            return rc;
        }
    }
    /* lock-step advance: graphs of graph_len launches, then single launches */
    bte::BatchArgs<T> ba;
    ba.inst = reinterpret_cast<const bte::BatchInst<T>*>(mem + rec_off);
    ba.item_inst = reinterpret_cast<const int*>(mem + map_off);
    ba.ninst = (int)n;
    ba.items = items;
    ba.base = reinterpret_cast<const long long*>(mem + base_off);
    ba.err = reinterpret_cast<int*>(mem + err_off);
    ba.tile_m = tile;
    ba.chunk_n = chunk;
    ba.vec = vec;
    ba.alt = walk == 2 || (walk == 0 && states_end > bte::kAltStateBytes);
    if (resident) {
        /* on chip: one persistent launch per cluster size, all launches
         * concurrent (each on its own stream, so the CTAs that one launch
         * frees at its end go to the others); within a launch, clusters take
         * points from a queue, costliest first (cells x steps) */
        std::vector<int> order(n);
        for (size_t i = 0; i < n; ++i) order[i] = (int)i;
        std::sort(order.begin(), order.end(), [&](int x, int y) {
            const BatchPoint& a = pts[first + x];
            const BatchPoint& b = pts[first + y];
            if (a.resC != b.resC) return a.resC > b.resC;
            const double ca = (double)a.N1 * a.M1 * a.tg.K, cb = (double)b.N1 * b.M1 * b.tg.K;
            return ca != cb ? ca > cb : x < y;
        });
        /* the item table is not used on this path: its space holds the order */
        if (items < (int)n) {
            rc = fail(BTE_ECUDA, "internal: order table too small");
            cleanup();
            return rc;
        }
        BCU(cudaMemcpyAsync(mem + map_off, order.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
        struct Launch {
            int C, begin, count;
            size_t smem, arrays;
            double longest;
        };
        std::vector<Launch> launches;
        for (size_t q = 0; q < n;) {
            Launch L{pts[first + order[q]].resC, (int)q, 0, 0, 0, 0.0};
            while (q < n && pts[first + order[q]].resC == L.C) {
                const BatchPoint& b = pts[first + order[q]];
                size_t ab = 0;
                L.smem = std::max(L.smem, bte::resident_smem_bytes<T>(b.N1 - 1, b.M1 - 1, L.C, &ab));
                L.arrays = std::max(L.arrays, ab);
                L.longest = std::max(L.longest, (double)b.tg.K * b.N1 * b.M1 / L.C);
                ++L.count;
                ++q;
            }
            launches.push_back(L);
        }
        /* the launch holding the longest point first */
        std::sort(launches.begin(), launches.end(),
                  [](const Launch& a, const Launch& b) { return a.longest > b.longest; });
        constexpr int kThreads = kResThreads;
        cudaEvent_t ready = nullptr;
        BCU(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        BCU(cudaEventRecord(ready, st));
        std::vector<cudaStream_t> side(launches.size(), nullptr);
        std::vector<cudaEvent_t> done(launches.size(), nullptr);
        int r = 0;
        for (size_t c = 0; c < launches.size() && !r; ++c) {
            const Launch& L = launches[c];
            bte::ResArgs<T> ra;
            ra.inst = ba.inst;
            ra.order = reinterpret_cast<const int*>(mem + map_off) + L.begin;
            ra.count = L.count;
            ra.queue = reinterpret_cast<unsigned*>(mem + base_off) + c;
            ra.C = L.C;
            ra.red_off = L.arrays;
            int clusters = 0;
            r = bte::resident_max_clusters<T>(L.C, L.smem, kThreads, &clusters);
            if (r || clusters < 1) {
                rc = fail(BTE_ECUDA, "on-chip kernel: no cluster of %d CTAs with %zu bytes fits (%s)",
                          L.C, L.smem, cudaGetErrorString((cudaError_t)r));
                r = -1;
                break;
            }
            clusters = std::min(clusters, L.count);
            if (cudaStreamCreateWithFlags(&side[c], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&done[c], cudaEventDisableTiming) != cudaSuccess ||
                cudaStreamWaitEvent(side[c], ready, 0) != cudaSuccess) {
                rc = fail(BTE_ECUDA, "on-chip launch: stream setup failed");
                r = -1;
                break;
            }
            r = bte::launch_resident<T>(ra, clusters, kThreads, L.smem, side[c]);
            if (r) {
                rc = fail(BTE_ECUDA, "on-chip kernel launch: %s", cudaGetErrorString((cudaError_t)r));
                break;
            }
            if (cudaEventRecord(done[c], side[c]) != cudaSuccess ||
                cudaStreamWaitEvent(st, done[c], 0) != cudaSuccess) {
                rc = fail(BTE_ECUDA, "on-chip launch: join failed");
                r = -1;
                break;
            }
        }
        for (size_t c = 0; c < side.size(); ++c) {
            if (side[c]) {
                cudaStreamSynchronize(side[c]);
                cudaStreamDestroy(side[c]);
            }
            if (done[c]) cudaEventDestroy(done[c]);
        }
        cudaEventDestroy(ready);
        if (r) {
            cleanup();
            return rc;
        }
    } else {
    {
        int bps = 0, dev = 0, sms = 0;
        BCU(cudaGetDevice(&dev));
        BCU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int r = bte::step_kernel_configure_batch<T>(tile, chunk, vec, &bps);
        if (r || bps < 1) {
            rc = fail(BTE_ECUDA, "batch kernel configure failed");
            cleanup();
            return rc;
        }
        ba.grid = std::min(items, bps * sms);
    }
    long long* base = reinterpret_cast<long long*>(mem + base_off);
    int set = 0;
    long long left = Kmax;
    const int L = (int)std::min<long long>(graph_len, Kmax);
    while (L >= 2 && left >= L) {
        if (!graph[set]) {
            cudaGraph_t g = nullptr;
            BCU(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            int r = 0;
            for (int i = 0; i < L && !r; ++i) r = bte::launch_step_batch<T>(ba, i, set, i > 0, cap);
            if (!r) r = bte::launch_advance_base(base, L, cap);
            cudaError_t ee = cudaStreamEndCapture(cap, &g);
            if (r || ee != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                rc = fail(BTE_ECUDA, "batch graph capture failed");
                cleanup();
                return rc;
            }
            ee = cudaGraphInstantiate(&graph[set], g, 0);
            cudaGraphDestroy(g);
            if (ee != cudaSuccess) {
                graph[set] = nullptr;
                rc = fail(BTE_ECUDA, "batch graph instantiate failed");
                cleanup();
                return rc;
            }
        }
        BCU(cudaGraphLaunch(graph[set], st));
        left -= L;
        set ^= L & 1;
    }
    if (left > 0) {
        int r = 0;
        for (long long i = 0; i < left && !r; ++i)
            r = bte::launch_step_batch<T>(ba, (int)i, set, i > 0, st);
        if (!r) r = bte::launch_advance_base(base, left, st);
        if (r) {
            rc = fail(BTE_ECUDA, "batch step: %s", cudaGetErrorString((cudaError_t)r));
            cleanup();
            return rc;
        }
    }
    }  // streamed tier
    /* window averages and status of every instance */
    std::vector<unsigned char> acc_host(tables_end - tables_begin);
    int err = 0;
    BCU(cudaMemcpyAsync(acc_host.data(), mem + tables_begin, acc_host.size(),
                        cudaMemcpyDeviceToHost, st));
    BCU(cudaMemcpyAsync(&err, mem + err_off, sizeof err, cudaMemcpyDeviceToHost, st));
    BCU(cudaStreamSynchronize(st));
#undef BCU
    int worst = BTE_OK;
    for (size_t i = first; i < last; ++i) {
        const BatchPoint& b = pts[i];
        const bte_params& pp = p[b.idx];
        double acc[kAcc];
        std::memcpy(acc, acc_host.data() + (b.tab_off - tables_begin) + b.o_acc, sizeof acc);
        bte_obs& ob = out[b.idx];
        std::memset(&ob, 0, sizeof ob);
        ob.t = b.tg.K * b.tg.dt_eff;
        ob.step = b.tg.K;
        ob.v_dr = acc[4];
        ob.norm = acc[5];
        ob.v_dc_avg = acc[1] / (double)b.tg.Kw;
        ob.absorption = pp.omega > 0 ? 2.0 / b.r1 * acc[0] / (double)b.tg.Kw : NAN;
        ob.norm_max_abs_err = std::fmax(acc[2], std::fabs(acc[7] - 1.0));
        ob.dt_eff = b.tg.dt_eff;
        ob.steps_total = b.tg.K;
        ob.steps_per_period = b.tg.P;
        ob.window_steps = b.tg.Kw;
        int s = BTE_OK;
        if (err) s = BTE_ETIMEOUT;
        else if (acc[3] != 0.0 || !std::isfinite(acc[6]) || !std::isfinite(acc[7]) ||
                 !(ob.norm_max_abs_err <= 0.05))
            s = BTE_EUNSTABLE;
        ob.status = s;
        if (s != BTE_OK && (worst == BTE_OK || s == BTE_ETIMEOUT)) worst = s;
    }
    cleanup();
    return worst;
}

struct BatchCfg {
    bool fp64;
    int vec, tile, chunk, graph_len, max_batch;
    long long max_bytes;
};

/* Validates the points and options of a batched run and assigns each point
 * its tier (BatchPoint::resC: on-chip cluster size, 0 for streamed). */
int batch_prepare(const bte_params* p, int32_t n, const bte_batch_opts* opts,
                  std::vector<BatchPoint>& pts, BatchCfg& cfg) {
    const int prec = p[0].precision;
    pts.assign(n, BatchPoint{});
    for (int i = 0; i < n; ++i) {
        int rc = validate(&p[i]);
        if (rc) return fail(rc, "point %d: %s", i, g_err.c_str());
        if (p[i].precision != prec) return fail(BTE_EINVAL, "all points must share one precision");
        BatchPoint& b = pts[i];
        b.idx = i;
        rc = time_grid(&p[i], b.tg);
        if (rc) return fail(rc, "point %d: %s", i, g_err.c_str());
        b.N1 = p[i].n_max + 1;
        b.M1 = p[i].m_points;
        b.dphi = (p[i].phiy_max - p[i].phiy_min) / (p[i].m_points - 1);
    }
    const bool fp64 = prec == BTE_FP64;
    int vec = (opts && opts->vec) ? opts->vec : (fp64 ? 2 : 4);
    if (vec != 2 && vec != 4) return fail(BTE_EINVAL, "vec must be 2 or 4");
    if (fp64 && vec != 2) return fail(BTE_EINVAL, "FP64 runs with vec = 2");
    /* two compute warps per item (measured best on the 4096-point sweep sample) */
    const int tile = (opts && opts->tile_m) ? opts->tile_m : 64 * vec;
    const int chunk = (opts && opts->chunk_n) ? opts->chunk_n : 16;
    const int max_tile = fp64 ? bte::step_max_tile<double>(vec) : bte::step_max_tile<float>(vec);
    if (tile % 4 || tile < 32 || tile > max_tile)
        return fail(BTE_EINVAL, "tile_m must be a multiple of 4 in 32..%d", max_tile);
    if (chunk < 4) return fail(BTE_EINVAL, "chunk_n must be >= 4");
    const size_t smem = fp64 ? bte::step_smem_bytes<double>(tile, chunk, vec)
                             : bte::step_smem_bytes<float>(tile, chunk, vec);
    if (smem > 227 * 1024)
        return fail(BTE_EINVAL, "tile_m %d needs %zu bytes of shared memory", tile, smem);
    const int graph_len = (opts && opts->graph_steps > 0) ? opts->graph_steps : 1024;
    const int max_batch = (opts && opts->max_batch > 0) ? opts->max_batch : 1024;
    const long long max_bytes =
        (opts && opts->max_batch_bytes > 0) ? opts->max_batch_bytes : (4ll << 30);
    const int mode = opts ? opts->resident : 0;
    if (mode < 0 || mode > 2) return fail(BTE_EINVAL, "resident must be 0, 1 or 2");
    const long long budget = (opts && opts->resident_smem > 0) ? opts->resident_smem : 232448;
    if (budget > 232448) return fail(BTE_EINVAL, "resident_smem above 232,448 bytes");
    if (opts && (opts->walk < 0 || opts->walk > 2)) return fail(BTE_EINVAL, "walk must be 0, 1 or 2");
    for (auto& b : pts) {
        b.ntx = (b.M1 + tile - 1) / tile;
        b.nty = (b.N1 + chunk - 1) / chunk;
        /* smallest cluster whose CTAs hold the point in `budget` bytes each,
         * with at least two rows per CTA (rows 0 and 1 in the first CTA) */
        b.resC = 0;
        if (mode != 1)
            for (int C = 1; C <= 16; C *= 2) {
                if (C > 1 && (b.N1 + C - 1) / C < 2) break;
                const size_t need = fp64 ? bte::resident_smem_bytes<double>(b.N1 - 1, b.M1 - 1, C, nullptr)
                                         : bte::resident_smem_bytes<float>(b.N1 - 1, b.M1 - 1, C, nullptr);
                if ((long long)need <= budget) {
                    b.resC = C;
                    break;
                }
            }
        if (mode == 2 && !b.resC)
            return fail(BTE_EINVAL, "point %d does not fit on chip in %lld bytes per CTA", b.idx, budget);
    }
    cfg.fp64 = fp64;
    cfg.vec = vec;
    cfg.tile = tile;
    cfg.chunk = chunk;
    cfg.graph_len = graph_len;
    cfg.max_batch = max_batch;
    cfg.max_bytes = max_bytes;
    return BTE_OK;
}

}  // namespace

namespace bte {
/* Sets the thread's last-error message for other translation units. */
int report_error(int code, const char* msg) {
    g_err = msg ? msg : "";
    return code;
}
}  // namespace bte

extern "C" {

const char* bte_last_error(void) { return g_err.c_str(); }

int bte_batch_run(const bte_params* p, int32_t n, bte_obs* out, const bte_batch_opts* opts) {
    if (!p || !out || n < 0) return fail(BTE_EINVAL, "bte_batch_run: bad argument");
    if (n == 0) return BTE_OK;
    std::vector<BatchPoint> pts;
    BatchCfg cfg;
    {
        const int rc = batch_prepare(p, n, opts, pts, cfg);
        if (rc) return rc;
    }
    const bool fp64 = cfg.fp64;
    const int vec = cfg.vec, tile = cfg.tile, chunk = cfg.chunk, graph_len = cfg.graph_len;
    const int max_batch = cfg.max_batch;
    const long long max_bytes = cfg.max_bytes;
    /* by tier (on-chip cluster size, then streamed), longest runs first, so a
     * streamed batch's members need similar step counts */
    std::sort(pts.begin(), pts.end(), [](const BatchPoint& x, const BatchPoint& y) {
        if (x.resC != y.resC) return x.resC > y.resC;
        return x.tg.K != y.tg.K ? x.tg.K > y.tg.K : x.idx < y.idx;
    });
    cudaStream_t st = opts && opts->stream ? (cudaStream_t)opts->stream : nullptr;
    bool own = false;
    if (!st) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return fail(BTE_ECUDA, "cudaStreamCreate failed");
        own = true;
    }
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        if (own) cudaStreamDestroy(st);
        return fail(BTE_ECUDA, "cudaStreamCreate failed");
    }
    const int elem = fp64 ? 8 : 4;
    int worst = BTE_OK;
    size_t first = 0;
    while (first < pts.size()) {
        size_t last = first;
        long long bytes = 0;
        /* on-chip points of every cluster size share a batch */
        const int resC = pts[first].resC;
        while (last < pts.size() && (pts[last].resC > 0) == (resC > 0) &&
               (resC > 0 || (int)(last - first) < max_batch)) {
            const BatchPoint& b = pts[last];
            const long long pitch = (long long)align_up((size_t)(128 / elem + b.ntx * tile + 32 / elem), 32);
            /* state arrays, the two [3][P+2] drive tables, other tables */
            const long long sb = (resC > 0 ? 4ll : 8ll) * b.N1 * pitch * elem + 6ll * (b.tg.P + 2) * elem + 4096;
            if (last > first && bytes + sb > max_bytes) break;
            bytes += sb;
            ++last;
        }
        const bool res = resC > 0;
        const int walk = opts ? opts->walk : 0;
        const int rc = fp64 ? run_batch<double>(p, pts, first, last, tile, chunk, vec, graph_len, res, walk, st, cap, out)
                            : run_batch<float>(p, pts, first, last, tile, chunk, vec, graph_len, res, walk, st, cap, out);
        if (rc == BTE_ECUDA || rc == BTE_ENOMEM) {
            worst = rc;
            break;
        }
        if (rc != BTE_OK && (worst == BTE_OK || rc == BTE_ETIMEOUT)) worst = rc;
        first = last;
    }
    cudaStreamDestroy(cap);
    if (own) cudaStreamDestroy(st);
    if (worst != BTE_OK && g_err.empty()) fail(worst, "at least one point failed");
    return worst;
}

int bte_batch_plan(const bte_params* p, int32_t n, const bte_batch_opts* opts, int32_t* tier) {
    if (!p || !tier || n < 0) return fail(BTE_EINVAL, "bte_batch_plan: bad argument");
    if (n == 0) return BTE_OK;
    std::vector<BatchPoint> pts;
    BatchCfg cfg;
    const int rc = batch_prepare(p, n, opts, pts, cfg);
    if (rc) return rc;
    for (const BatchPoint& b : pts) tier[b.idx] = b.resC;
    return BTE_OK;
}

int bte_batch_tune(const bte_params* p, int32_t n, const bte_batch_opts* base, int32_t sample,
                   int32_t steps, bte_batch_opts* best, double* seconds) {
    if (!p || !best || n < 1 || sample < 1 || steps < 2)
        return fail(BTE_EINVAL, "bte_batch_tune: bad argument");
    bte_batch_opts b0;
    if (base) b0 = *base;
    else std::memset(&b0, 0, sizeof b0);
    {
        std::vector<BatchPoint> pts;
        BatchCfg cfg;
        const int rc = batch_prepare(p, n, &b0, pts, cfg); /* validates every point */
        if (rc) return rc;
    }
    /* the sample: points evenly spaced in cost order, runs shortened to about
     * `steps` steps (relative run lengths kept) */
    std::vector<std::pair<double, int>> cost(n);
    for (int i = 0; i < n; ++i) {
        TimeGrid tg;
        time_grid(&p[i], tg);
        cost[i] = {(double)(p[i].n_max + 1) * p[i].m_points * tg.K, i};
    }
    std::sort(cost.begin(), cost.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
        return a.first != b.first ? a.first > b.first : a.second < b.second;
    });
    const int ns = std::min(sample, n);
    long long Kmax = 0;
    for (int i = 0; i < n; ++i) {
        TimeGrid tg;
        time_grid(&p[i], tg);
        Kmax = std::max(Kmax, tg.K);
    }
    const double scale = std::min(1.0, (double)steps / (double)Kmax);
    std::vector<bte_params> sp(ns);
    for (int j = 0; j < ns; ++j) {
        bte_params q = p[cost[(size_t)j * n / ns].second];
        if (q.omega > 0) {
            const double Pd = std::nearbyint(kTwoPi / (q.omega * q.dt)); /* steps per period */
            q.periods = std::max(q.periods * scale, 2.0 / Pd);
            if (q.avg_window > q.periods) q.avg_window = q.periods;
        } else {
            q.t_max = std::max(q.t_max * scale, 2.0 * q.dt);
            if (q.avg_window > q.t_max) q.avg_window = q.t_max;
        }
        sp[j] = q;
    }
    /* candidates: on-chip budgets, then streamed shapes */
    const bool fp64 = p[0].precision == BTE_FP64;
    const int v = b0.vec ? b0.vec : (fp64 ? 2 : 4);
    std::vector<bte_batch_opts> cand;
    for (int smem : {232448, 160000, 113664}) {
        bte_batch_opts o = b0;
        o.resident = 0;
        o.resident_smem = smem;
        cand.push_back(o);
    }
    for (int tw : {32, 64, 128})
        for (int ch : {8, 16, 32}) {
            bte_batch_opts o = b0;
            o.resident = 1;
            o.tile_m = tw * v;
            o.chunk_n = ch;
            cand.push_back(o);
        }
    std::vector<bte_obs> out(ns);
    double best_t = 1e300;
    int best_i = -1;
    for (size_t c = 0; c < cand.size(); ++c) {
        double t = 1e300;
        std::vector<BatchPoint> chk;
        BatchCfg cfg;
        if (batch_prepare(sp.data(), ns, &cand[c], chk, cfg) == BTE_OK) {
            /* the first run builds graphs and warms caches; the second is timed */
            int rc = bte_batch_run(sp.data(), ns, out.data(), &cand[c]);
            if (rc == BTE_OK || rc == BTE_EUNSTABLE) {
                const auto t0 = std::chrono::steady_clock::now();
                rc = bte_batch_run(sp.data(), ns, out.data(), &cand[c]);
                const auto t1 = std::chrono::steady_clock::now();
                if (rc == BTE_OK || rc == BTE_EUNSTABLE) t = std::chrono::duration<double>(t1 - t0).count();
            }
            if (rc == BTE_ECUDA || rc == BTE_ENOMEM || rc == BTE_ETIMEOUT) return rc;
        }
        if (seconds) seconds[c] = t;
        if (t < best_t) {
            best_t = t;
            best_i = (int)c;
        }
    }
    if (best_i < 0) return fail(BTE_EINVAL, "no candidate launch shape ran");
    *best = cand[best_i];
    g_err.clear();
    return BTE_OK;
}

const char* bte_version(void) { return "bte-gb300 0.1 (sm_103a)"; }

int bte_bessel_ratio(double mu, int32_t nmax, double* r) {
    if (!(mu > 0) || !std::isfinite(mu) || nmax < 0 || !r)
        return fail(BTE_EINVAL, "bte_bessel_ratio: bad argument");
    miller_ratio(mu, nmax, r);
    return BTE_OK;
}

int bte_time_grid(const bte_params* p, double* dt_eff, int64_t* P, int64_t* K, int64_t* Kw) {
    int rc = validate(p);
    if (rc) return rc;
    TimeGrid g;
    rc = time_grid(p, g);
    if (rc) return rc;
    if (dt_eff) *dt_eff = g.dt_eff;
    if (P) *P = g.P;
    if (K) *K = g.K;
    if (Kw) *Kw = g.Kw;
    return BTE_OK;
}

int bte_workspace_size(const bte_params* p, const bte_tuning* tune, size_t* bytes) {
    int rc = validate(p);
    if (rc) return rc;
    if (!bytes) return fail(BTE_EINVAL, "bytes is NULL");
    TimeGrid g;
    rc = time_grid(p, g);
    if (rc) return rc;
    Layout L;
    rc = plan(p, tune, g, L);
    if (rc) return rc;
    *bytes = L.total;
    return BTE_OK;
}

int bte_launch_shape(const bte_params* p, const bte_tuning* tune, int32_t* tile_m,
                     int32_t* chunk_n, int32_t* pitch, int32_t* grid_x, int32_t* grid_y) {
    int rc = validate(p);
    if (rc) return rc;
    TimeGrid g;
    rc = time_grid(p, g);
    if (rc) return rc;
    Layout L;
    rc = plan(p, tune, g, L);
    if (rc) return rc;
    if (tile_m) *tile_m = L.tile_m;
    if (chunk_n) *chunk_n = L.chunk_n;
    if (pitch) *pitch = L.pitch;
    if (grid_x) *grid_x = L.ntx;
    if (grid_y) *grid_y = L.nty;
    return BTE_OK;
}

int bte_create_ex(const bte_params* p, void* stream, const bte_tuning* tune, void* workspace,
                  size_t workspace_bytes, bte_handle** out) {
    if (!out) return fail(BTE_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    bte_handle* h = new (std::nothrow) bte_handle();
    if (!h) return fail(BTE_ENOMEM, "host allocation failed");
    h->p = *p;
    h->fp64 = p->precision == BTE_FP64;
    h->dphi = (p->phiy_max - p->phiy_min) / (p->m_points - 1);
    rc = time_grid(p, h->tg);
    if (!rc) rc = plan(p, tune, h->tg, h->L);
    if (rc) {
        delete h;
        return rc;
    }
    h->graph_len = (tune && tune->graph_steps > 0) ? tune->graph_steps : 1024;
    if (h->graph_len > h->tg.K) h->graph_len = (int)h->tg.K;
    auto bail = [&](int code) {
        bte_destroy(h);
        return code;
    };
    if (stream) {
        h->stream = (cudaStream_t)stream;
        h->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return fail(BTE_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        h->own_stream = true;
    }
    {
        cudaError_t e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(fail(BTE_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
    }
    if (workspace) {
        if (workspace_bytes < h->L.total)
            return bail(fail(BTE_ENOMEM, "workspace of %zu bytes, %zu needed", workspace_bytes,
                             h->L.total));
        if ((uintptr_t)workspace % 256)
            return bail(fail(BTE_EINVAL, "workspace must be 256-byte aligned"));
        h->mem = (unsigned char*)workspace;
        h->own_mem = false;
    } else {
        cudaError_t e = cudaMalloc(&h->mem, h->L.total);
        if (e != cudaSuccess) {
            h->mem = nullptr;
            cudaGetLastError();
            return bail(fail(BTE_ENOMEM, "cudaMalloc(%zu): %s", h->L.total, cudaGetErrorString(e)));
        }
        h->own_mem = true;
    }
    {
        int bps = 0, dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return bail(fail(BTE_ECUDA, "no CUDA device"));
        const long long items = (long long)h->L.ntx * h->L.nty;
        rc = h->fp64 ? bte::step_kernel_configure<double>(h->L.tile_m, h->L.chunk_n, h->L.vec, &bps)
                     : bte::step_kernel_configure<float>(h->L.tile_m, h->L.chunk_n, h->L.vec, &bps);
        if (rc)
            return bail(fail(BTE_ECUDA, "kernel configure: %s", cudaGetErrorString((cudaError_t)rc)));
        if (bps < 1) return bail(fail(BTE_EINVAL, "launch shape does not fit on an SM"));
        const long long slots = (long long)bps * sms;
        h->grid[1] = (int)(items < slots ? items : slots);
        h->grid_persist = 0;
        if (h->L.persist) {
            int pb = 0;
            rc = h->fp64 ? bte::step_kernel_configure_persist<double>(h->L.tile_m, h->L.chunk_n, h->L.vec, &pb)
                         : bte::step_kernel_configure_persist<float>(h->L.tile_m, h->L.chunk_n, h->L.vec, &pb);
            if (rc)
                return bail(fail(BTE_ECUDA, "kernel configure: %s", cudaGetErrorString((cudaError_t)rc)));
            if (pb < 1) return bail(fail(BTE_EINVAL, "launch shape does not fit on an SM"));
            /* one CTA per item, every CTA co-resident */
            const long long cap = (long long)pb * sms;
            if (items > cap)
                return bail(fail(BTE_EINVAL,
                                 "persistent mode: %lld work items but %lld co-resident CTAs; "
                                 "use larger chunk_n or tile_m",
                                 items, cap));
            h->grid_persist = (int)items;
        }
    }
    if (h->L.resC) {
        /* sets the on-chip kernel's shared-memory (and cluster-size) attributes */
        int clusters = 0;
        rc = h->fp64 ? bte::resident_max_clusters<double>(h->L.resC, h->L.res_smem, kResThreads, &clusters)
                     : bte::resident_max_clusters<float>(h->L.resC, h->L.res_smem, kResThreads, &clusters);
        if (rc) return bail(fail(BTE_ECUDA, "on-chip kernel configure: %s", cudaGetErrorString((cudaError_t)rc)));
        if (clusters < 1)
            return bail(fail(BTE_EINVAL, "a cluster of %d CTAs with %zu bytes each cannot be scheduled",
                             h->L.resC, h->L.res_smem));
    }
    if (h->L.wideG) {
        /* all G clusters must be resident at once (their waits are bounded);
         * an automatic shape takes no more clusters than fit (wider blocks:
         * the workspace planned for the first choice still covers it) */
        Layout& L = h->L;
        int clusters = 0;
        for (int attempt = 0; attempt < 4; ++attempt) {
            rc = h->fp64 ? bte::wide_max_clusters<double>(L.wideC, L.wide_smem, L.wide_threads, &clusters)
                         : bte::wide_max_clusters<float>(L.wideC, L.wide_smem, L.wide_threads, &clusters);
            if (rc)
                return bail(fail(BTE_ECUDA, "on-chip kernel configure: %s", cudaGetErrorString((cudaError_t)rc)));
            if (clusters >= L.wideG || (tune && tune->wide_cols) || clusters < 1) break;
            const int M1 = h->p.m_points;
            const int Wc = (M1 + clusters - 1) / clusters;
            const size_t bytes = wide_need(L.elem, L.wide_rp, Wc);
            if (bytes > kWideSmemMax || L.wide_rp * Wc > kWideMaxCells) break;
            L.wideWc = Wc;
            L.wideG = (M1 + Wc - 1) / Wc;
            L.wide_smem = bytes;
            L.wide_threads = wide_threads(L.wide_rp, Wc);
        }
        if (clusters < L.wideG)
            return bail(fail(BTE_EINVAL, "%d clusters of %d CTAs (%zu bytes each) do not fit the GPU at once (%d do)",
                             L.wideG, L.wideC, L.wide_smem, clusters));
    }
    rc = h->fp64 ? upload_tables<double>(h) : upload_tables<float>(h);
    if (rc) return bail(rc);
    rc = h->fp64 ? initialise<double>(h, true, true) : initialise<float>(h, true, true);
    if (rc) return bail(rc);
    *out = h;
    return BTE_OK;
}

int bte_create(const bte_params* p, void* stream, bte_handle** out) {
    return bte_create_ex(p, stream, nullptr, nullptr, 0, out);
}

int bte_reset(bte_handle* h) {
    if (!h) return fail(BTE_EINVAL, "handle is NULL");
    return h->fp64 ? initialise<double>(h, false, false) : initialise<float>(h, false, false);
}

int bte_step(bte_handle* h, int64_t nsteps) {
    if (!h) return fail(BTE_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(BTE_EINVAL, "nsteps < 0");
    if (h->k + nsteps > h->tg.K)
        return fail(BTE_ESTATE, "step %lld + %lld passes the end of the run (%lld)", h->k,
                    (long long)nsteps, h->tg.K);
    return h->fp64 ? enqueue_steps<double>(h, nsteps) : enqueue_steps<float>(h, nsteps);
}

int bte_run(bte_handle* h) {
    if (!h) return fail(BTE_EINVAL, "handle is NULL");
    return bte_step(h, h->tg.K - h->k);
}

int bte_observables(bte_handle* h, bte_obs* out) {
    if (!h || !out) return fail(BTE_EINVAL, "NULL argument");
    const Layout& L = h->L;
    bte::FinalArgs f;
    f.trace_v = h->ptr<double>(L.off_tv);
    f.trace_n = h->ptr<double>(L.off_tn);
    f.k = h->k;
    f.K = h->tg.K;
    f.Kw = h->tg.Kw;
    f.P = h->tg.P;
    f.omega = h->p.omega;
    f.dt_eff = h->tg.dt_eff;
    f.inv_r1 = 1.0 / h->r1;
    f.out = h->ptr<double>(L.off_fin);
    int rc = bte::launch_finalize(f, h->stream);
    if (rc) return fail(BTE_ECUDA, "finalize kernel: %s", cudaGetErrorString((cudaError_t)rc));
    double fin[4], vn[2];
    int err = 0;
    CU(cudaMemcpyAsync(fin, f.out, sizeof fin, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&vn[0], f.trace_v + h->k, 8, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&vn[1], f.trace_n + h->k, 8, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&err, h->ptr<int>(L.off_err), sizeof err, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    const bool done = h->k == h->tg.K;
    out->t = h->k * h->tg.dt_eff;
    out->step = h->k;
    out->v_dr = vn[0];
    out->norm = vn[1];
    out->v_dc_avg = done ? fin[1] : NAN;
    out->absorption = (done && h->p.omega > 0) ? fin[0] : NAN;
    out->norm_max_abs_err = fin[2];
    out->dt_eff = h->tg.dt_eff;
    out->steps_total = h->tg.K;
    out->steps_per_period = h->tg.P;
    out->window_steps = h->tg.Kw;
    int st = BTE_OK;
    if (err == bte::kErrLaunch) st = BTE_ECUDA;
    else if (err) st = BTE_ETIMEOUT;
    else if (fin[3] != 0.0 || !(fin[2] <= 0.05)) st = BTE_EUNSTABLE;
    out->status = st;
    out->reserved = 0;
    if (st == BTE_ECUDA) return fail(st, "a solver kernel found itself launched in the wrong shape");
    if (st == BTE_ETIMEOUT) return fail(st, "a bounded wait in a solver kernel gave up");
    if (st == BTE_EUNSTABLE)
        return fail(st, "unstable run: |norm-1| reached %g%s", fin[2],
                    fin[3] != 0.0 ? " (non-finite values)" : "");
    return BTE_OK;
}

int bte_wait_probe(bte_handle* h, int64_t limit_ns) {
    if (!h) return fail(BTE_EINVAL, "handle is NULL");
    if (limit_ns < 1 || limit_ns > 2000000000ll)
        return fail(BTE_EINVAL, "limit_ns %lld outside 1..2e9", (long long)limit_ns);
    const int rc = bte::launch_wait_probe(h->ptr<int>(h->L.off_err), (unsigned long long)limit_ns,
                                          h->stream);
    if (rc) return fail(BTE_ECUDA, "wait probe kernel: %s", cudaGetErrorString((cudaError_t)rc));
    return BTE_OK;
}

int bte_trace(bte_handle* h, int64_t k0, int64_t count, double* v, double* norm) {
    if (!h) return fail(BTE_EINVAL, "handle is NULL");
    if (k0 < 0 || count < 0 || k0 + count > h->k + 1)
        return fail(BTE_EINVAL, "trace range [%lld, %lld) outside 0..%lld", (long long)k0,
                    (long long)(k0 + count), h->k);
    if (count == 0) return BTE_OK;
    if (v)
        CU(cudaMemcpyAsync(v, h->ptr<double>(h->L.off_tv) + k0, count * 8, cudaMemcpyDeviceToHost,
                           h->stream));
    if (norm)
        CU(cudaMemcpyAsync(norm, h->ptr<double>(h->L.off_tn) + k0, count * 8,
                           cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return BTE_OK;
}

int bte_get_state(bte_handle* h, int grid, double* a, double* b) {
    if (!h || (grid != 0 && grid != 1)) return fail(BTE_EINVAL, "bad handle or grid");
    return h->fp64 ? get_grid<double>(h, grid, a, b) : get_grid<float>(h, grid, a, b);
}

int bte_set_state(bte_handle* h, int grid, const double* a, const double* b) {
    if (!h || (grid != 0 && grid != 1) || !a || !b) return fail(BTE_EINVAL, "bad argument");
    return h->fp64 ? set_grid<double>(h, grid, a, b) : set_grid<float>(h, grid, a, b);
}

int bte_set_step(bte_handle* h, int64_t k, const double* v, const double* norm) {
    if (!h || !v || !norm) return fail(BTE_EINVAL, "bad argument");
    if (k < 0 || k > h->tg.K) return fail(BTE_EINVAL, "step %lld outside 0..%lld", (long long)k, h->tg.K);
    h->base_host = k;
    CU(cudaMemcpyAsync(h->ptr<long long>(h->L.off_base), &h->base_host, 8, cudaMemcpyHostToDevice,
                       h->stream));
    CU(cudaMemcpyAsync(h->ptr<double>(h->L.off_tv), v, (k + 1) * 8, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->ptr<double>(h->L.off_tn), norm, (k + 1) * 8, cudaMemcpyHostToDevice,
                       h->stream));
    CU(cudaStreamSynchronize(h->stream));
    h->k = k;
    return BTE_OK;
}

int bte_pdf(bte_handle* h, int grid, int32_t nphix, double* out) {
    if (!h || (grid != 0 && grid != 1) || !out || nphix < 1 || nphix > 65535)
        return fail(BTE_EINVAL, "bad argument (grid 0/1, 1 <= nphix <= 65535)");
    const Layout& L = h->L;
    const int set = h->set, M1 = h->p.m_points;
    const size_t bytes = (size_t)nphix * M1 * sizeof(double);
    double* d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(BTE_ENOMEM, "pdf buffer of %zu bytes", bytes);
    }
    const size_t oa = L.off_state[4 * set + 2 * grid], ob = L.off_state[4 * set + 2 * grid + 1];
    int r = h->fp64 ? bte::launch_pdf<double>(h->ptr<double>(oa), h->ptr<double>(ob), h->p.n_max,
                                              M1 - 1, L.pitch, nphix, d, h->stream)
                    : bte::launch_pdf<float>(h->ptr<float>(oa), h->ptr<float>(ob), h->p.n_max,
                                             M1 - 1, L.pitch, nphix, d, h->stream);
    cudaError_t e = r ? (cudaError_t)r : cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(BTE_ECUDA, "pdf: %s", cudaGetErrorString(e));
    return BTE_OK;
}

void bte_destroy(bte_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int q = 0; q < 2; ++q)
        if (h->graph[q]) cudaGraphExecDestroy(h->graph[q]);
    if (h->own_mem && h->mem) cudaFree(h->mem);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  /* extern "C" */
