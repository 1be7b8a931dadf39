/*
 * bte_oracle.cpp -- FP64 CPU oracle for the superlattice Boltzmann transport
 * solver of Priimak, "Finite difference numerical method for the superlattice
 * Boltzmann transport equation ..." (arXiv:1401.6047).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * What it computes, in the paper's order:
 *   - Sec. 2, Eq. (f0_fourier) and Eq. (Bolzmann_initial_pdf): the Fourier
 *     coefficients a0_n(phi_y) of the equilibrium distribution.  I_n/I_0 is
 *     taken straight from its definition as a Fourier coefficient of
 *     exp(mu cos phi_x) (trapezoid rule on the periodic integrand).
 *   - Sec. 3, Eqs. (a_forward)..(b_backward) and (a_t_plus_1),(b_t_plus_1):
 *     the Crank-Nicolson operator T for one cell.
 *   - Sec. 3, Eqs. (leap_frog_1),(leap_frog_2): the staggered whole /
 *     fractional grids, started by a half step.
 *   - Sec. 2, Eq. (v_dr_generic), Eq. (norm_in_phi), Eq. (absorption_def):
 *     drift velocity, norm and time-averaged absorption.
 *
 * Readings of the paper taken here (each one is also listed in the design
 * notes of the repository):
 *   R1 sigma(0)=1/2, sigma(n>=1)=1   (the printed "n != 1" is a typo; only
 *      this choice normalises f0, Eq. norm_in_phi).
 *   R2 b^{t+1} = (g mu' + h nu)/D    (the printed minus sign does not solve
 *      the 2x2 Crank-Nicolson system of Eqs. a_backward, b_backward).
 *   R3 the stencil coefficient is B dt/(4 dphi) without alpha (the continuum
 *      Eqs. a_n_dot, b_n_dot carry no alpha).
 *   R4 b_0 is identically zero (boundary condition Eq. b_boundary), so the
 *      n = 0 update of b is discarded.
 *   R5 theta uses E at the start of the (half-)step, theta' at its end.
 *   R6 the start-up half step is T with dt replaced by dt/2 everywhere and
 *      the initial state as its own stencil source.
 *   R7 dt is adjusted to dt_eff = 2 pi/(omega P), P = round(2 pi/(omega dt)),
 *      so a drive period is a whole number of steps; time averages are the
 *      equal-weight mean of whole-grid samples over the last avg_periods
 *      periods (rectangle rule on a periodic signal).
 *   R8 integrals over phi_y are dphi * sum over the M+1 grid points.
 *   R9 observables are taken from the whole grid at integer steps.
 *   R13 a time-dependent field B(t) (Sec. 2 notes that Eqs. a_n_dot, b_n_dot
 *      allow one; here B(t) = B + B_omega cos(omega t + B_phase)) is sampled
 *      like E: the rotation mu, mu' takes B at the start and the end of the
 *      (half-)step, the stencil coefficient B dt/(4 dphi) takes B at the time
 *      of the grid that supplies the stencil (the middle of the half-step; 0
 *      for the start-up half step, whose source is the initial state).
 *
 * Parity pins: every function here is pinned by tests that do not use this
 * file's arithmetic (closed forms at B = 0, Esaki-Tsu, Tucker, relaxation,
 * stationarity of f0 at E = 0, symmetries, sublattice decoupling, order of
 * convergence, the method of characteristics at B != 0, scipy's Bessel
 * functions).
 *
 * Planted-mistake switches (oracle_params.flags) exist only so that the test
 * suite can show each pin fails on a plausible error; flags = 0 is the method.
 */
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

/* Problem parameters, dimensionless units of Eqs. (substitutions). */
typedef struct {
    double E_dc, E_omega, omega, B, mu, alpha;
    double phiy_min, phiy_max;
    double dt;          /* requested time step (R7 adjusts it)                */
    double periods;     /* run length in drive periods (omega > 0)            */
    double t_max;       /* run length in time units (omega == 0)              */
    double avg_window;  /* averaging window: periods (omega>0) or time (=0)   */
    int32_t n_max;      /* harmonics n = 0..n_max                             */
    int32_t m_points;   /* phi_y grid points M+1                              */
    int32_t flags;      /* planted mistakes, 0 = the method                   */
    int32_t reserved;
    double B_omega, B_phase; /* B(t) = B + B_omega cos(omega t + B_phase)     */
} oracle_params;

enum {
    ORACLE_MUT_PAPER_B_SIGN = 1,      /* use the printed sign of b^{t+1}       */
    ORACLE_MUT_ALPHA_STENCIL = 2,     /* keep the printed alpha in the stencil */
    ORACLE_MUT_SIGMA0_ONE = 4,        /* sigma(0) = 1                          */
    ORACLE_MUT_NO_CHI = 8,            /* chi(1) = 1                            */
    ORACLE_MUT_STALE_SOURCE = 16,     /* fractional step reads the old whole grid */
    ORACLE_MUT_THETA_START_ONLY = 32, /* theta' evaluated at the step start    */
    ORACLE_MUT_STENCIL_INDEX = 64,    /* off-by-one column in one S^a term     */
    ORACLE_MUT_NO_B0_RESET = 128,     /* keep the n = 0 b update               */
    ORACLE_MUT_B_STENCIL_START = 256  /* stencil coefficient from B at t0      */
};

} /* extern "C" */

namespace {

const double kPi = 3.14159265358979323846;

struct Grid {
    int N, M;           /* n = 0..N, m = 0..M */
    double dphi;
    double dt_eff;
    long long P;        /* steps per drive period (0 when omega == 0) */
    long long K;        /* total steps */
    long long Kw;       /* samples in the averaging window */
    std::vector<double> phi;  /* phi_y(m) */
    std::vector<double> a0;   /* [N+1][M+1] */
    std::vector<double> r;    /* I_n(mu)/I_0(mu) */
};

int check_params(const oracle_params* p) {
    if (!p) return -1;
    const double v[] = {p->E_dc, p->E_omega, p->omega, p->B, p->mu, p->alpha,
                        p->phiy_min, p->phiy_max, p->dt, p->periods, p->t_max,
                        p->avg_window, p->B_omega, p->B_phase};
    for (double x : v)
        if (!std::isfinite(x)) return -1;
    if (p->n_max < 1 || p->m_points < 3) return -1;
    if (p->mu <= 0 || p->alpha <= 0 || p->dt <= 0 || p->omega < 0) return -1;
    if (!(p->phiy_max > p->phiy_min)) return -1;
    if (p->avg_window < 0) return -1;
    if (p->omega > 0) {
        if (p->periods <= 0 || p->avg_window > p->periods) return -1;
    } else {
        if (p->t_max <= 0 || p->avg_window > p->t_max) return -1;
    }
    return 0;
}

/* I_n(mu)/I_0(mu), n = 0..nmax, from the definition of I_n as the n-th
 * cosine coefficient of exp(mu cos x):  I_n(mu) = (1/2pi) int_0^{2pi}
 * exp(mu cos x) cos(n x) dx.  The trapezoid rule on a periodic analytic
 * integrand converges geometrically; the number of nodes keeps the first
 * aliased coefficient (order Q - n) below double precision. */
void bessel_ratio(double mu, int nmax, double* r) {
    int Q = 2 * (nmax + 1) + 64 + 16 * (int)std::ceil(std::sqrt(mu) + 1.0);
    Q = (Q + 3) / 4 * 4;
    std::vector<double> w(Q), c(Q);
    double s0 = 0;
    for (int j = 0; j < Q; ++j) {
        double x = 2.0 * kPi * j / Q;
        c[j] = std::cos(x);
        w[j] = std::exp(mu * (c[j] - 1.0));
        s0 += w[j];
    }
    for (int n = 0; n <= nmax; ++n) {
        double s = 0;
        for (int j = 0; j < Q; ++j) {
            long long idx = ((long long)n * j) % Q; /* cos(n x_j) = cos(x_{n j mod Q}) */
            s += w[j] * c[idx];
        }
        r[n] = s / s0;
    }
}

int make_grid(const oracle_params* p, Grid& g) {
    if (check_params(p)) return -1;
    g.N = p->n_max;
    g.M = p->m_points - 1;
    g.dphi = (p->phiy_max - p->phiy_min) / g.M;
    if (p->omega > 0) {
        /* R7 */
        g.P = std::llround(2.0 * kPi / (p->omega * p->dt));
        if (g.P < 1) g.P = 1;
        g.dt_eff = 2.0 * kPi / (p->omega * (double)g.P);
        g.K = std::llround(p->periods * (double)g.P);
        g.Kw = std::llround(p->avg_window * (double)g.P);
    } else {
        g.P = 0;
        g.dt_eff = p->dt;
        g.K = std::llround(p->t_max / p->dt);
        g.Kw = std::llround(p->avg_window / p->dt);
    }
    if (g.K < 1) return -1;
    if (g.Kw > g.K) g.Kw = g.K;
    g.phi.resize(g.M + 1);
    for (int m = 0; m <= g.M; ++m) g.phi[m] = p->phiy_min + m * g.dphi;
    g.r.resize(g.N + 1);
    bessel_ratio(p->mu, g.N, g.r.data());
    /* Eq. (Bolzmann_initial_pdf): a0_n = sigma(n) I_n/(pi I_0) sqrt(mu/(2 pi alpha))
     * exp(-mu phi_y^2/2), sigma(0)=1/2 (R1). */
    g.a0.assign((size_t)(g.N + 1) * (g.M + 1), 0.0);
    const double pref = std::sqrt(p->mu / (2.0 * kPi * p->alpha));
    for (int n = 0; n <= g.N; ++n) {
        double sigma = (n == 0 && !(p->flags & ORACLE_MUT_SIGMA0_ONE)) ? 0.5 : 1.0;
        for (int m = 0; m <= g.M; ++m)
            g.a0[(size_t)n * (g.M + 1) + m] =
                sigma * g.r[n] / kPi * pref * std::exp(-0.5 * p->mu * g.phi[m] * g.phi[m]);
    }
    return 0;
}

double E_at(const oracle_params* p, double t) {
    /* Sec. 2: E(t) = E_dc + E_omega cos(omega t). */
    return p->E_dc + p->E_omega * std::cos(p->omega * t);
}

double B_at(const oracle_params* p, double t) {
    /* reading R13: B(t) = B + B_omega cos(omega t + B_phase); B for the paper */
    return p->B + p->B_omega * std::cos(p->omega * t + p->B_phase);
}

/* Value of a grid array at (n, m); zero outside the computed region
 * (boundary conditions Eqs. a_boundary and b_boundary). */
inline double at(const double* x, const Grid& g, int n, int m) {
    if (n < 0 || n > g.N || m < 0 || m > g.M) return 0.0;
    return x[(size_t)n * (g.M + 1) + m];
}
inline double at_b(const double* x, const Grid& g, int n, int m) {
    if (n < 1) return 0.0; /* b_n = 0 for n outside 1..N */
    return at(x, g, n, m);
}

/* One application of the operator T of Eq. (time_shift):
 *   (a, b) at time t0, step h, stencil source (as, bs) at time ts
 *   ->  (an, bn) at t0 + h.
 * Forward / backward differences Eqs. (a_forward)..(b_backward), combined
 * Crank-Nicolson style, solved in closed form Eqs. (a_t_plus_1), (b_t_plus_1)
 * with readings R2..R5.  The output arrays must not alias the inputs. */
void apply_T(const oracle_params* p, const Grid& g, double t0, double h, double ts,
             const double* a, const double* b, const double* as, const double* bs,
             double* an, double* bn) {
    const double nu = 1.0 + h / 2.0;
    const double xi = 1.0 - h / 2.0;
    double c = B_at(p, (p->flags & ORACLE_MUT_B_STENCIL_START) ? t0 : ts) * h / (4.0 * g.dphi);
    if (p->flags & ORACLE_MUT_ALPHA_STENCIL) c *= p->alpha;
    const double Es = E_at(p, t0);
    const double Ee = (p->flags & ORACLE_MUT_THETA_START_ONLY) ? Es : E_at(p, t0 + h);
    const double Bs = B_at(p, t0);
    const double Be = (p->flags & ORACLE_MUT_THETA_START_ONLY) ? Bs : B_at(p, t0 + h);
    const int N = g.N, M = g.M;
#pragma omp parallel for schedule(static)
    for (int n = 0; n <= N; ++n) {
        const double chi = (n == 1 && !(p->flags & ORACLE_MUT_NO_CHI)) ? 2.0 : 1.0;
        for (int m = 0; m <= M; ++m) {
            const size_t i = (size_t)n * (M + 1) + m;
            /* mu^t_{n,m} = n beta^t_m dt/2, beta^t_m = E^t + B^t phi_y(m) */
            const double th = n * (Es + Bs * g.phi[m]) * h / 2.0;
            const double th1 = n * (Ee + Be * g.phi[m]) * h / 2.0;
            /* the paper's B^t_{n,m} (acts on a) and A^t_{n,m} (acts on b) */
            double Sa;
            if (p->flags & ORACLE_MUT_STENCIL_INDEX)
                Sa = c * (at_b(bs, g, n + 1, m + 1) - at_b(bs, g, n + 1, m - 1) -
                          at_b(bs, g, n - 1, m + 1) + at_b(bs, g, n - 1, m));
            else
                Sa = c * (at_b(bs, g, n + 1, m + 1) - at_b(bs, g, n + 1, m - 1) -
                          at_b(bs, g, n - 1, m + 1) + at_b(bs, g, n - 1, m - 1));
            const double Sb = c * (chi * (at(as, g, n - 1, m + 1) - at(as, g, n - 1, m - 1)) -
                                   at(as, g, n + 1, m + 1) + at(as, g, n + 1, m - 1));
            const double gg = a[i] * xi - b[i] * th + Sa + g.a0[i] * h;
            const double qq = b[i] * xi + a[i] * th + Sb;
            const double D = nu * nu + th1 * th1;
            an[i] = (gg * nu - qq * th1) / D;
            if (p->flags & ORACLE_MUT_PAPER_B_SIGN)
                bn[i] = (gg * th1 - qq * nu) / D;
            else
                bn[i] = (gg * th1 + qq * nu) / D;
            if (n == 0 && !(p->flags & ORACLE_MUT_NO_B0_RESET)) bn[i] = 0.0; /* R4 */
        }
    }
}

/* v_dr = pi sqrt(alpha) int b_1 dphi_y ; norm = 2 pi sqrt(alpha) int a_0 dphi_y
 * (Eq. v_dr_generic in Fourier form, Eq. norm_in_phi, reading R8). */
void observe(const oracle_params* p, const Grid& g, const double* a, const double* b,
             double* v, double* norm) {
    double sb = 0, sa = 0;
    for (int m = 0; m <= g.M; ++m) {
        sb += b[(size_t)1 * (g.M + 1) + m];
        sa += a[m];
    }
    const double sq = std::sqrt(p->alpha);
    *v = kPi * sq * g.dphi * sb;
    *norm = 2.0 * kPi * sq * g.dphi * sa;
}

} /* namespace */

extern "C" {

/* Number of threads the oracle's loops use. */
int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Time grid of reading R7.  Returns 0, or -1 on invalid parameters. */
int oracle_time_grid(const oracle_params* p, double* dt_eff, long long* P, long long* K,
                     long long* Kw) {
    if (check_params(p)) return -1;
    Grid g;
    /* avoid the Bessel work: replicate only the time part */
    if (p->omega > 0) {
        g.P = std::llround(2.0 * kPi / (p->omega * p->dt));
        if (g.P < 1) g.P = 1;
        g.dt_eff = 2.0 * kPi / (p->omega * (double)g.P);
        g.K = std::llround(p->periods * (double)g.P);
        g.Kw = std::llround(p->avg_window * (double)g.P);
    } else {
        g.P = 0;
        g.dt_eff = p->dt;
        g.K = std::llround(p->t_max / p->dt);
        g.Kw = std::llround(p->avg_window / p->dt);
    }
    if (g.K < 1) return -1;
    if (g.Kw > g.K) g.Kw = g.K;
    if (dt_eff) *dt_eff = g.dt_eff;
    if (P) *P = g.P;
    if (K) *K = g.K;
    if (Kw) *Kw = g.Kw;
    return 0;
}

/* I_n(mu)/I_0(mu) for n = 0..nmax. */
int oracle_bessel_ratio(double mu, int nmax, double* r) {
    if (!(mu > 0) || nmax < 0 || !r) return -1;
    bessel_ratio(mu, nmax, r);
    return 0;
}

/* a0_{n,m}, host array [n_max+1][m_points]. */
int oracle_equilibrium(const oracle_params* p, double* a0) {
    Grid g;
    if (make_grid(p, g)) return -1;
    std::memcpy(a0, g.a0.data(), g.a0.size() * sizeof(double));
    return 0;
}

/* Initial state (Sec. 2: a_n = a0_n, b_n = 0 at t = 0) and start-up half step
 * (Sec. 3, reading R6): whole grid (aw,bw) at t=0, fractional grid (af,bf) at
 * t = dt_eff/2.  Arrays are [n_max+1][m_points]. */
int oracle_init(const oracle_params* p, double* aw, double* bw, double* af, double* bf) {
    Grid g;
    if (make_grid(p, g)) return -1;
    const size_t sz = g.a0.size();
    std::memcpy(aw, g.a0.data(), sz * sizeof(double));
    std::memset(bw, 0, sz * sizeof(double));
    apply_T(p, g, 0.0, g.dt_eff / 2.0, 0.0, aw, bw, aw, bw, af, bf);
    return 0;
}

/* Advance both grids nsteps leap-frog steps (Eqs. leap_frog_1, leap_frog_2),
 * starting with the whole grid at step k0 (t = k0 dt_eff) and the fractional
 * grid at t = (k0 + 1/2) dt_eff.  The arrays are updated in place.  After step
 * k (1-based within this call) v_out[k-1], norm_out[k-1] receive the
 * observables of the whole grid (either may be NULL). */
int oracle_advance(const oracle_params* p, long long k0, long long nsteps, double* aw,
                   double* bw, double* af, double* bf, double* v_out, double* norm_out) {
    Grid g;
    if (make_grid(p, g)) return -1;
    if (nsteps < 0 || k0 < 0) return -1;
    const size_t sz = g.a0.size();
    std::vector<double> an(sz), bn(sz), afn(sz), bfn(sz);
    const double h = g.dt_eff;
    for (long long s = 0; s < nsteps; ++s) {
        const long long k = k0 + s;
        const double t = k * h;
        /* z^{t+1} = T(z^t; S(z^{t+1/2})) */
        apply_T(p, g, t, h, t + 0.5 * h, aw, bw, af, bf, an.data(), bn.data());
        /* z^{t+3/2} = T(z^{t+1/2}; S(z^{t+1})) -- source is the NEW whole grid */
        if (p->flags & ORACLE_MUT_STALE_SOURCE)
            apply_T(p, g, t + 0.5 * h, h, t + h, af, bf, aw, bw, afn.data(), bfn.data());
        else
            apply_T(p, g, t + 0.5 * h, h, t + h, af, bf, an.data(), bn.data(), afn.data(),
                    bfn.data());
        std::memcpy(aw, an.data(), sz * sizeof(double));
        std::memcpy(bw, bn.data(), sz * sizeof(double));
        std::memcpy(af, afn.data(), sz * sizeof(double));
        std::memcpy(bf, bfn.data(), sz * sizeof(double));
        double v, nr;
        observe(p, g, aw, bw, &v, &nr);
        if (v_out) v_out[s] = v;
        if (norm_out) norm_out[s] = nr;
    }
    return 0;
}

/* Observables of one grid state. */
int oracle_observe(const oracle_params* p, const double* a, const double* b, double* v,
                   double* norm) {
    Grid g;
    if (check_params(p)) return -1;
    g.N = p->n_max;
    g.M = p->m_points - 1;
    g.dphi = (p->phiy_max - p->phiy_min) / g.M;
    observe(p, g, a, b, v, norm);
    return 0;
}

/* Window averages of Eq. (absorption_def) from a trace v[0..K] of whole-grid
 * samples (v[k] at t = k dt_eff):  A = (2 I_0/I_1) <v cos(omega t)>,
 * vbar = <v>, both over the last Kw samples k = K-Kw+1..K (reading R7).
 * A is NaN when omega == 0. */
int oracle_window(const oracle_params* p, const double* v, long long K, double* A,
                  double* vbar) {
    double dt_eff;
    long long P, Kt, Kw;
    if (oracle_time_grid(p, &dt_eff, &P, &Kt, &Kw)) return -1;
    if (K < Kw || Kw < 1) return -1;
    double r[2];
    bessel_ratio(p->mu, 1, r);
    double sc = 0, s = 0;
    for (long long k = K - Kw + 1; k <= K; ++k) {
        sc += v[k] * std::cos(p->omega * (double)k * dt_eff);
        s += v[k];
    }
    *vbar = s / (double)Kw;
    *A = (p->omega > 0) ? 2.0 / r[1] * sc / (double)Kw : NAN;
    return 0;
}

/* Complete run of the paper's protocol: equilibrium start, start-up half
 * step, K leap-frog steps, window averages.  v_trace / norm_trace (length
 * K+1, may be NULL) receive the whole-grid samples k = 0..K.
 * out[0] = A, out[1] = vbar_dc, out[2] = max_k |norm_k - 1|, out[3] = dt_eff,
 * out[4] = K, out[5] = Kw.  The final state is returned when the four state
 * pointers are non-NULL. */
int oracle_solve(const oracle_params* p, double* v_trace, double* norm_trace, double* out,
                 double* aw_out, double* bw_out, double* af_out, double* bf_out) {
    Grid g;
    if (make_grid(p, g)) return -1;
    const size_t sz = g.a0.size();
    std::vector<double> aw(sz), bw(sz), af(sz), bf(sz);
    oracle_init(p, aw.data(), bw.data(), af.data(), bf.data());
    std::vector<double> v(g.K + 1), nr(g.K + 1);
    observe(p, g, aw.data(), bw.data(), &v[0], &nr[0]);
    oracle_advance(p, 0, g.K, aw.data(), bw.data(), af.data(), bf.data(), &v[1], &nr[1]);
    double A, vbar;
    oracle_window(p, v.data(), g.K, &A, &vbar);
    double err = 0;
    for (long long k = 0; k <= g.K; ++k) err = std::fmax(err, std::fabs(nr[k] - 1.0));
    out[0] = A;
    out[1] = vbar;
    out[2] = err;
    out[3] = g.dt_eff;
    out[4] = (double)g.K;
    out[5] = (double)g.Kw;
    if (v_trace) std::memcpy(v_trace, v.data(), v.size() * sizeof(double));
    if (norm_trace) std::memcpy(norm_trace, nr.data(), nr.size() * sizeof(double));
    if (aw_out && bw_out && af_out && bf_out) {
        std::memcpy(aw_out, aw.data(), sz * sizeof(double));
        std::memcpy(bw_out, bw.data(), sz * sizeof(double));
        std::memcpy(af_out, af.data(), sz * sizeof(double));
        std::memcpy(bf_out, bf.data(), sz * sizeof(double));
    }
    return 0;
}

} /* extern "C" */
