/*
 * FP64 CPU oracle for voxelwise ABC rejection (vPET-ABC, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * used by the test-suite, by the smoke check and by the CPU-baseline leg of
 * the benchmark.  The product (the CUDA library) neither links nor calls it,
 * and it shares no code, header, table or helper with the CUDA sources.
 *
 * Every function is a plain, slow restatement of the paper's definitions:
 *   - prior draws: Philox4x32-10 counter RNG (Salmon et al., SC'11), uniform
 *     boxes (Algorithm 1, steps 1-2; Sec. III-A priors);
 *   - 2TCM: Eq. 1-2, closed-form impulse response convolved with a
 *     poly-exponential input term by term (textbook partial fractions, series
 *     where the two rates nearly coincide), frame means by adaptive
 *     Gauss-Legendre quadrature of the pointwise curve;
 *   - MRTM: Eq. 3 with gamma = 0 in its closed (convolution) form;
 *   - lp-ntPET: the differential form of Eq. 3-4, integrated with an adaptive
 *     Dormand-Prince 5(4) scheme, the frame integral carried as an extra state;
 *   - distance: frame-weighted squared Euclidean distance computed directly
 *     (and the frame-weighted L1 distance Sec. V recommends);
 *   - top-k: full sort of (distance, draw index) per voxel, first k kept
 *     (Algorithm 1, step 5; fixed-budget rejection, Sec. II-C);
 *   - model probabilities and preferred model (Sec. III-B, "more than 50 %");
 *   - posterior summaries: mean, SD (ddof = 1), equal-tailed 95 % interval
 *     by type-7 interpolation, and K_i = K1 k3 / (k2 + k3) per accepted sample
 *     (Sec. II-D point estimates; Sec. III-B K_i map);
 *   - the lp-ntPET response function 1 + (gamma / k2a) g(t) and its 95 %
 *     credible band over a time grid (Sec. II-D).
 *
 * Parity status of each function is listed next to it ("pinned by" names the
 * tests that tie it to something other than itself).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_IRR 0
#define ORC_REV 1
#define ORC_MRTM 2
#define ORC_LPNT 3

/* ------------------------------------------------------------------ Philox */
/* Philox4x32-10 as published (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
 * two 32x32->64 multiplies, Weyl key schedule.  Pinned by the published
 * known-answer vectors (tests/test_oracle_rng.py). */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

/* Prior draws (Algorithm 1, steps 1-2).  Draw n of model m, parameter p uses
 * counter (n_lo, n_hi, m, p/4), word p%4, key (seed_lo, seed_hi); the uniform is
 * u = (r >> 8) * 2^-24 and theta = fl32(lo + (hi - lo) * u) evaluated in FP64.
 * Pinned by: uniform moments / box membership and the Philox vectors. */
int orc_sample_prior(uint64_t seed, int model, const double* lo, const double* hi, int P,
                     int64_t N, int64_t first, float* theta, int ldtheta) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t n = 0; n < N; ++n) {
        const uint64_t g = (uint64_t)(first + n);
        for (int p = 0; p < P; ++p) {
            uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), (uint32_t)model, (uint32_t)(p >> 2)};
            uint32_t r[4];
            orc_philox4x32_10(ctr, key, r);
            const double u = (double)(r[p & 3] >> 8) * (1.0 / 16777216.0);
            volatile double span = hi[p] - lo[p];
            volatile double prod = span * u;
            volatile double v = lo[p] + prod;
            theta[n * ldtheta + p] = (float)v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------ poly-exponentials */
typedef struct {
    int n;
    const double *c, *a0, *a1, *a2;
} pexp;

static double pexp_eval(const pexp* e, double t) {
    double s = 0.0;
    for (int i = 0; i < e->n; ++i) s += (e->a0[i] + t * (e->a1[i] + t * e->a2[i])) * exp(-e->c[i] * t);
    return s;
}

static double pexp_deriv(const pexp* e, double t) {
    double s = 0.0;
    for (int i = 0; i < e->n; ++i) {
        const double p = e->a0[i] + t * (e->a1[i] + t * e->a2[i]);
        const double dp = e->a1[i] + 2.0 * t * e->a2[i];
        s += (dp - e->c[i] * p) * exp(-e->c[i] * t);
    }
    return s;
}

/* E_m(d, t) = int_0^t u^m exp(-d u) du for m = 0, 1, 2.
 * Closed form m!/d^(m+1) [1 - exp(-d t) sum_{j<=m} (d t)^j / j!] when |d t| >= 1,
 * else the power series t^(m+1) sum_j (-d t)^j / (j! (m + j + 1)).
 * Pinned by: E_m against numerical quadrature in test_oracle_sim.py. */
static double Em(int m, double d, double t) {
    const double x = d * t;
    if (fabs(x) < 1.0) {
        double term = 1.0, s = 0.0;
        for (int j = 0; j < 40; ++j) {
            if (j > 0) term *= -x / j;
            s += term / (double)(m + j + 1);
        }
        return s * pow(t, m + 1);
    }
    double poly = 1.0, tj = 1.0, fact = 1.0;
    for (int j = 1; j <= m; ++j) { tj *= x; fact *= j; poly += tj / fact; }
    double mf = 1.0;
    for (int j = 2; j <= m; ++j) mf *= j;
    return mf / pow(d, m + 1) * (1.0 - exp(-x) * poly);
}

/* exp(-alpha t) E_m(c - alpha, t), written so that neither factor overflows:
 * for |d t| >= 1 it is m!/d^(m+1) [exp(-alpha t) - exp(-c t) sum_{j<=m} (d t)^j / j!]. */
static double exp_Em(int m, double alpha, double c, double t) {
    const double d = c - alpha, x = d * t;
    if (fabs(x) < 1.0) return exp(-alpha * t) * Em(m, d, t);
    double poly = 1.0, tj = 1.0, fact = 1.0;
    for (int j = 1; j <= m; ++j) { tj *= x; fact *= j; poly += tj / fact; }
    double mf = 1.0;
    for (int j = 2; j <= m; ++j) mf *= j;
    return mf / pow(d, m + 1) * (exp(-alpha * t) - exp(-c * t) * poly);
}

/* (A exp(-alpha t)) convolved with the poly-exponential e, at time t:
 * sum_i sum_m a_m,i A exp(-alpha t) E_m(c_i - alpha, t). */
static double conv_exp_pexp(double A, double alpha, const pexp* e, double t) {
    if (A == 0.0) return 0.0;
    double s = 0.0;
    for (int i = 0; i < e->n; ++i) {
        double v = e->a0[i] * exp_Em(0, alpha, e->c[i], t);
        if (e->a1[i] != 0.0) v += e->a1[i] * exp_Em(1, alpha, e->c[i], t);
        if (e->a2[i] != 0.0) v += e->a2[i] * exp_Em(2, alpha, e->c[i], t);
        s += v;
    }
    return A * s;
}

/* 2TCM impulse response h(t) = sum_r A_r exp(-alpha_r t) (Eq. 1 solved with
 * C_f(0) = C_m(0) = 0).  alpha_{1,2} = (s -/+ sqrt(s^2 - 4 k2 k4)) / 2 with
 * s = k2 + k3 + k4 (alpha_1 via the product form 2 k2 k4 / (s + sqrt)), and
 * A_1 = K1 (k3 + k4 - alpha_1)/(alpha_2 - alpha_1), A_2 = K1 (alpha_2 - k3 - k4)/(alpha_2 - alpha_1).
 * With k4 = 0 this is K1/(k2+k3) [k3 + k2 exp(-(k2+k3) t)]. */
static void irf_2tcm(double K1, double k2, double k3, double k4, double A[2], double al[2]) {
    const double s = k2 + k3 + k4;
    const double D = sqrt(s * s - 4.0 * k2 * k4);
    al[0] = 2.0 * k2 * k4 / (s + D);
    al[1] = 0.5 * (s + D);
    A[0] = K1 * (k3 + k4 - al[0]) / (al[1] - al[0]);
    A[1] = K1 * (al[1] - k3 - k4) / (al[1] - al[0]);
}

typedef struct {
    int model;
    double p[8];
    const pexp* in;
    double A[2], al[2];   /* 2TCM impulse response */
} tac_ctx;

/* Pointwise measured TAC C_t(t) (Eq. 2 for the 2TCM with C_wb = C_p; Eq. 3 with
 * gamma = 0 for MRTM). */
static double tac_point(const tac_ctx* c, double t) {
    if (c->model == ORC_IRR || c->model == ORC_REV) {
        const double Vb = c->model == ORC_IRR ? c->p[3] : c->p[4];
        const double ct = conv_exp_pexp(c->A[0], c->al[0], c->in, t) + conv_exp_pexp(c->A[1], c->al[1], c->in, t);
        return (1.0 - Vb) * ct + Vb * pexp_eval(c->in, t);
    }
    /* MRTM: C = R1 C_r + (k2 - R1 k2a) (C_r conv exp(-k2a t)),  k2a = k2 / (1 + BP) */
    const double R1 = c->p[0], k2 = c->p[1], k2a = c->p[1] / (1.0 + c->p[2]);
    return R1 * pexp_eval(c->in, t) + conv_exp_pexp(k2 - R1 * k2a, k2a, c->in, t);
}

/* ------------------------------------------------------------ quadrature */
static double gl_x[20], gl_w[20];
static int gl_ready = 0;

/* Gauss-Legendre 20-point nodes and weights from Newton's method on P_20. */
static void gl_init(void) {
    if (gl_ready) return;
    const int n = 20;
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
            const double dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
        const double dp = n * (x * p1 - p0) / (x * x - 1.0);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

void orc_gl_nodes(double* x, double* w) { gl_init(); memcpy(x, gl_x, sizeof gl_x); memcpy(w, gl_w, sizeof gl_w); }

typedef double (*fn1)(const void*, double);

static double gl_panel(fn1 f, const void* ctx, double a, double b) {
    const double h = 0.5 * (b - a), m = 0.5 * (a + b);
    double s = 0.0;
    for (int i = 0; i < 20; ++i) s += gl_w[i] * f(ctx, m + h * gl_x[i]);
    return s * h;
}

/* Accept a panel when its two halves agree with the whole to 1e-13 relative (or
 * to the frame-level absolute floor); GL-20 is then accurate far below that. */
static double gl_adapt(fn1 f, const void* ctx, double a, double b, double whole, double floor_abs, int depth) {
    const double m = 0.5 * (a + b);
    const double l = gl_panel(f, ctx, a, m), r = gl_panel(f, ctx, m, b);
    const double err = fabs(l + r - whole);
    if (depth >= 30 || !(err == err) || err <= fmax(1e-13 * fabs(l + r), floor_abs)) return l + r;
    return gl_adapt(f, ctx, a, m, l, floor_abs, depth + 1) + gl_adapt(f, ctx, m, b, r, floor_abs, depth + 1);
}

/* int_a^b f, split at geometric points fast_scale * 2^j so the sharp input rise
 * near t = 0 (rates up to 1000/min) is resolved, then adaptive bisection. */
static double integrate(fn1 f, const void* ctx, double a, double b, double fast_scale) {
    gl_init();
    double pts[64];
    int np = 0;
    pts[np++] = a;
    for (double s = fast_scale / 16.0; s < b && np < 60; s *= 2.0)
        if (s > a) pts[np++] = s;
    pts[np++] = b;
    double w[64], mag = 0.0;
    for (int i = 0; i + 1 < np; ++i) { w[i] = gl_panel(f, ctx, pts[i], pts[i + 1]); mag += fabs(w[i]); }
    const double floor_abs = 1e-16 * mag + 1e-300;
    double total = 0.0;
    for (int i = 0; i + 1 < np; ++i) total += gl_adapt(f, ctx, pts[i], pts[i + 1], w[i], floor_abs, 0);
    return total;
}

static double tac_point_cb(const void* c, double t) { return tac_point((const tac_ctx*)c, t); }

/* ------------------------------------------------------------ lp-ntPET */
/* Gamma-variate activation (normalised to peak 1 at t_P):
 * g(t) = ((t - t_D)/(t_P - t_D))^alpha exp(alpha (1 - (t - t_D)/(t_P - t_D))), t >= t_D; 0 before. */
double orc_gamma_variate(double t, double tD, double tP, double alpha) {
    if (t < tD) return 0.0;
    const double x = (t - tD) / (tP - tD);
    if (alpha == 0.0) return 1.0;
    if (x == 0.0) return 0.0;
    return pow(x, alpha) * exp(alpha * (1.0 - x));
}

typedef struct {
    const pexp* cr;
    double R1, k2, k2a, gam, tD, tP, alpha;
} lp_ctx;

/* dC/dt = R1 C_r' + k2 C_r - (k2a + gamma g(t)) C  (Eq. 3-4 differentiated);
 * dF/dt = C (frame integral carried as a state). */
static void lp_rhs(const lp_ctx* c, double t, const double y[2], double dy[2]) {
    const double g = orc_gamma_variate(t, c->tD, c->tP, c->alpha);
    dy[0] = c->R1 * pexp_deriv(c->cr, t) + c->k2 * pexp_eval(c->cr, t) - (c->k2a + c->gam * g) * y[0];
    dy[1] = y[0];
}

/* Dormand-Prince 5(4) from t0 to t1 with error control on both states. */
static void dopri(const lp_ctx* c, double t0, double t1, double y[2], double rtol, double atol) {
    static const double a21 = 1.0 / 5;
    static const double a31 = 3.0 / 40, a32 = 9.0 / 40;
    static const double a41 = 44.0 / 45, a42 = -56.0 / 15, a43 = 32.0 / 9;
    static const double a51 = 19372.0 / 6561, a52 = -25360.0 / 2187, a53 = 64448.0 / 6561, a54 = -212.0 / 729;
    static const double a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247, a64 = 49.0 / 176,
                        a65 = -5103.0 / 18656;
    static const double b1 = 35.0 / 384, b3 = 500.0 / 1113, b4 = 125.0 / 192, b5 = -2187.0 / 6784, b6 = 11.0 / 84;
    static const double e1 = 71.0 / 57600, e3 = -71.0 / 16695, e4 = 71.0 / 1920, e5 = -17253.0 / 339200,
                        e6 = 22.0 / 525, e7 = -1.0 / 40;
    double t = t0, h = fmin(1e-3, t1 - t0);
    if (h <= 0) return;
    double k1[2], k2[2], k3[2], k4[2], k5[2], k6[2], k7[2], yt[2], yn[2];
    lp_rhs(c, t, y, k1);
    int guard = 0;
    while (t < t1 && guard++ < 10000000) {
        if (t + h > t1) h = t1 - t;
        for (int i = 0; i < 2; ++i) yt[i] = y[i] + h * a21 * k1[i];
        lp_rhs(c, t + h / 5, yt, k2);
        for (int i = 0; i < 2; ++i) yt[i] = y[i] + h * (a31 * k1[i] + a32 * k2[i]);
        lp_rhs(c, t + 3 * h / 10, yt, k3);
        for (int i = 0; i < 2; ++i) yt[i] = y[i] + h * (a41 * k1[i] + a42 * k2[i] + a43 * k3[i]);
        lp_rhs(c, t + 4 * h / 5, yt, k4);
        for (int i = 0; i < 2; ++i) yt[i] = y[i] + h * (a51 * k1[i] + a52 * k2[i] + a53 * k3[i] + a54 * k4[i]);
        lp_rhs(c, t + 8 * h / 9, yt, k5);
        for (int i = 0; i < 2; ++i)
            yt[i] = y[i] + h * (a61 * k1[i] + a62 * k2[i] + a63 * k3[i] + a64 * k4[i] + a65 * k5[i]);
        lp_rhs(c, t + h, yt, k6);
        for (int i = 0; i < 2; ++i)
            yn[i] = y[i] + h * (b1 * k1[i] + b3 * k3[i] + b4 * k4[i] + b5 * k5[i] + b6 * k6[i]);
        lp_rhs(c, t + h, yn, k7);
        double err = 0.0;
        for (int i = 0; i < 2; ++i) {
            const double ei = h * (e1 * k1[i] + e3 * k3[i] + e4 * k4[i] + e5 * k5[i] + e6 * k6[i] + e7 * k7[i]);
            const double sc = atol + rtol * fmax(fabs(y[i]), fabs(yn[i]));
            const double r = ei / sc;
            err += r * r;
        }
        err = sqrt(err / 2.0);
        if (err <= 1.0) {
            t += h;
            y[0] = yn[0]; y[1] = yn[1];
            k1[0] = k7[0]; k1[1] = k7[1];
        }
        const double fac = err == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2)));
        h *= fac;
        if (h < 1e-12) h = 1e-12;
    }
}

/* lp-ntPET frame means: integrate from 0, splitting at t_D and at every frame edge. */
static void lp_frames(const lp_ctx* c, int L, const double* ts, const double* te, double* out, double atol) {
    double y[2] = {0.0, 0.0}, t = 0.0;
    for (int l = 0; l < L; ++l) {
        if (ts[l] > t) {
            if (c->tD > t && c->tD < ts[l]) { dopri(c, t, c->tD, y, 1e-11, atol); t = c->tD; }
            dopri(c, t, ts[l], y, 1e-11, atol);
            t = ts[l];
        }
        const double F0 = y[1];
        if (c->tD > t && c->tD < te[l]) { dopri(c, t, c->tD, y, 1e-11, atol); t = c->tD; }
        dopri(c, t, te[l], y, 1e-11, atol);
        t = te[l];
        out[l] = (y[1] - F0) / (te[l] - ts[l]);
    }
}

/* ------------------------------------------------------------ simulate */
static double max_rate(const pexp* e) {
    double m = 0.0;
    for (int i = 0; i < e->n; ++i) m = fmax(m, e->c[i]);
    return m;
}

/* Frame-mean TACs (Algorithm 1, step 3) for N draws of one model.
 * x[n, l] = (1/dt_l) int_{ts_l}^{te_l} C_t(t) dt.
 * Pinned by: ODE integration of Eq. 1 (2TCM), mass balance, MRTM == 1-tissue
 * target/reference identity, lp-ntPET(gamma = 0) == MRTM, step activation ==
 * piecewise MRTM (tests/test_oracle_sim.py). */
int orc_simulate(int model, int L, const double* ts, const double* te, int nterms, const double* c,
                 const double* a0, const double* a1, const double* a2, const float* theta, int64_t N,
                 int ldtheta, double* x, int ldx, int nthreads) {
    pexp in = {nterms, c, a0, a1, a2};
    const double fast = max_rate(&in) > 0 ? 1.0 / max_rate(&in) : 1.0;
    gl_init();
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t n = 0; n < N; ++n) {
        const float* th = theta + n * ldtheta;
        double* xo = x + n * ldx;
        if (model == ORC_LPNT) {
            lp_ctx lc = {&in, th[0], th[1], th[1] / (1.0 + th[2]), th[3], th[4], (double)th[4] + (double)th[5], th[6]};
            double scale = 0.0;
            for (int i = 0; i < nterms; ++i) scale = fmax(scale, fabs(a0[i]) + fabs(a1[i]));
            lp_frames(&lc, L, ts, te, xo, 1e-13 * scale);
            continue;
        }
        tac_ctx tc;
        memset(&tc, 0, sizeof tc);
        tc.model = model;
        tc.in = &in;
        for (int p = 0; p < 8 && p < ldtheta; ++p) tc.p[p] = th[p];
        if (model == ORC_IRR) irf_2tcm(th[0], th[1], th[2], 0.0, tc.A, tc.al);
        else if (model == ORC_REV) irf_2tcm(th[0], th[1], th[2], th[3], tc.A, tc.al);
        for (int l = 0; l < L; ++l)
            xo[l] = integrate(tac_point_cb, &tc, ts[l], te[l], fast) / (te[l] - ts[l]);
    }
    return 0;
}

/* Pointwise TAC for pins (2TCM / MRTM only). */
double orc_tac_point(int model, const float* theta, int nterms, const double* c, const double* a0,
                     const double* a1, const double* a2, double t) {
    pexp in = {nterms, c, a0, a1, a2};
    tac_ctx tc;
    memset(&tc, 0, sizeof tc);
    tc.model = model;
    tc.in = &in;
    for (int p = 0; p < 8; ++p) tc.p[p] = theta[p];
    if (model == ORC_IRR) irf_2tcm(theta[0], theta[1], theta[2], 0.0, tc.A, tc.al);
    else if (model == ORC_REV) irf_2tcm(theta[0], theta[1], theta[2], theta[3], tc.A, tc.al);
    return tac_point(&tc, t);
}

double orc_Em(int m, double d, double t) { return Em(m, d, t); }

/* ------------------------------------------------------------ distance / top-k */
/* d(y, x) = sum_l w_l (y_l - x_l)^2  (Algorithm 1, step 4; weighted squared L2). */
static double wdist(const float* y, const double* x, const double* w, int L) {
    double s = 0.0;
    for (int l = 0; l < L; ++l) { const double e = (double)y[l] - x[l]; s += w[l] * e * e; }
    return s;
}

typedef struct { double d; int64_t i; } di_pair;

static int di_cmp(const void* a, const void* b) {
    const di_pair* p = (const di_pair*)a;
    const di_pair* q = (const di_pair*)b;
    if (p->d < q->d) return -1;
    if (p->d > q->d) return 1;
    return (p->i > q->i) - (p->i < q->i);
}

/* Algorithm 1, steps 4-5 for voxels [0, J): all N distances, sorted by (d, index),
 * first k kept.  Pinned by brute force and noise-free recovery (test_oracle_topk.py). */
int orc_topk(const float* y, int64_t J, int ldy, const double* x, int64_t N, int ldx, int L, const double* w,
             int k, int32_t* idx, double* dist, int nthreads) {
    if (k < 1 || k > N) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        di_pair* buf = (di_pair*)malloc(sizeof(di_pair) * (size_t)N);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t j = 0; j < J; ++j) {
            for (int64_t n = 0; n < N; ++n) { buf[n].d = wdist(y + j * ldy, x + n * ldx, w, L); buf[n].i = n; }
            qsort(buf, (size_t)N, sizeof(di_pair), di_cmp);
            for (int r = 0; r < k; ++r) { idx[j * k + r] = (int32_t)buf[r].i; dist[j * k + r] = buf[r].d; }
        }
        free(buf);
    }
    return 0;
}

/* Frame-weighted L1 distance sum_l w_l |y_l - x_l| (the distance Sec. V recommends),
 * summed directly in fp64. */
static double wdist_l1(const float* y, const double* x, const double* w, int L) {
    double s = 0.0;
    for (int l = 0; l < L; ++l) s += w[l] * fabs((double)y[l] - x[l]);
    return s;
}

/* Top-k by the L1 distance: full sort of (distance, draw index) per voxel, first k.
 * Pinned by: brute force on tiny inputs, the L1 triangle inequality and the
 * single-frame case (a sort of |y - x|) in tests/test_oracle_topk.py. */
int orc_topk_l1(const float* y, int64_t J, int ldy, const double* x, int64_t N, int ldx, int L, const double* w,
                int k, int32_t* idx, double* dist, int nthreads) {
    if (k < 1 || k > N) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        di_pair* buf = (di_pair*)malloc(sizeof(di_pair) * (size_t)N);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t j = 0; j < J; ++j) {
            for (int64_t n = 0; n < N; ++n) { buf[n].d = wdist_l1(y + j * ldy, x + n * ldx, w, L); buf[n].i = n; }
            qsort(buf, (size_t)N, sizeof(di_pair), di_cmp);
            for (int r = 0; r < k; ++r) { idx[j * k + r] = (int32_t)buf[r].i; dist[j * k + r] = buf[r].d; }
        }
        free(buf);
    }
    return 0;
}

/* Distances of the listed (voxel, draw) pairs, for sampled checks at full size. */
void orc_pair_dist(const float* y, int ldy, const double* x, int ldx, int L, const double* w, const int64_t* vj,
                   const int64_t* dn, int64_t npairs, double* out) {
    for (int64_t p = 0; p < npairs; ++p) out[p] = wdist(y + vj[p] * ldy, x + dn[p] * ldx, w, L);
}

/* ------------------------------------------------------------ model selection */
static int model_of(int64_t i, const int64_t* off, int M) {
    for (int m = 0; m < M; ++m)
        if (i >= off[m] && i < off[m + 1]) return m;
    return -1;
}

/* prob[j, m] = (# accepted draws of model m) / k; preferred = argmax, ties to the
 * lower model position (Sec. III-B: a model is preferred with > 50 % of the n
 * accepted draws; with M = 2 a 50/50 split goes to the first-listed model). */
int orc_model_select(const int32_t* idx, int64_t J, int k, const int64_t* off, int M, double* prob, int8_t* pref) {
    for (int64_t j = 0; j < J; ++j) {
        int cnt[16] = {0};
        for (int r = 0; r < k; ++r) {
            const int m = model_of(idx[j * k + r], off, M);
            if (m < 0) return -1;
            cnt[m]++;
        }
        int best = 0;
        for (int m = 0; m < M; ++m) {
            prob[j * M + m] = (double)cnt[m] / (double)k;
            if (cnt[m] > cnt[best]) best = m;
        }
        pref[j] = (int8_t)best;
    }
    return 0;
}

/* ------------------------------------------------------------ summaries */
static int dcmp(const void* a, const void* b) {
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* mean, SD with ddof = 1 (0 for a single value), and the type-7 quantiles at
 * 0.025 / 0.975 of v[0..n). */
static void stats(double* v, int n, double out[4]) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i];
    const double mean = s / n;
    double ss = 0.0;
    for (int i = 0; i < n; ++i) ss += (v[i] - mean) * (v[i] - mean);
    out[0] = mean;
    out[1] = n > 1 ? sqrt(ss / (n - 1)) : 0.0;
    qsort(v, (size_t)n, sizeof(double), dcmp);
    const double qs[2] = {0.025, 0.975};
    for (int q = 0; q < 2; ++q) {
        const double h = (n - 1) * qs[q];
        const int lo = (int)floor(h);
        const int hi = lo + 1 < n ? lo + 1 : n - 1;
        out[2 + q] = v[lo] + (h - lo) * (v[hi] - v[lo]);
    }
}

/* Posterior summaries per voxel over the accepted draws of the preferred model
 * (pref != NULL) or over all k accepted draws (pref == NULL).  Output rows have
 * ncols = Pmax + 1 entries: parameters 0..P_m-1 of that model, NaN beyond, and
 * K_i = K1 k3/(k2 + k3) (per accepted sample, then summarised) in the last
 * column where the model has ki flag set, else NaN.
 * Pinned by: k = 1, constant-theta and textbook-statistics tests. */
int orc_summarize(const float* theta, int ldtheta, const int64_t* off, int M, const int32_t* nparams,
                  const int32_t* has_ki, const int32_t* ki_cols, const int32_t* idx, int64_t J, int k,
                  const int8_t* pref, int Pmax, double* mean, double* sd, double* lo, double* hi) {
    const int nc = Pmax + 1;
    double* v = (double*)malloc(sizeof(double) * (size_t)k);
    for (int64_t j = 0; j < J; ++j) {
        const int pm = pref ? pref[j] : -1;
        int P = pm >= 0 ? nparams[pm] : Pmax;
        int ki = pm >= 0 ? has_ki[pm] : 1;
        if (pm < 0)
            for (int m = 0; m < M; ++m) { if (nparams[m] < P) P = nparams[m]; if (!has_ki[m]) ki = 0; }
        for (int col = 0; col < nc; ++col) {
            double o[4] = {NAN, NAN, NAN, NAN};
            const int isk = col == Pmax;
            if ((isk && ki) || (!isk && col < P)) {
                int n = 0;
                for (int r = 0; r < k; ++r) {
                    const int32_t i = idx[j * k + r];
                    if (pm >= 0 && model_of(i, off, M) != pm) continue;
                    const float* th = theta + (int64_t)i * ldtheta;
                    if (isk) {
                        const double K1 = th[ki_cols[0]], k2 = th[ki_cols[1]], k3 = th[ki_cols[2]];
                        v[n++] = K1 * k3 / (k2 + k3);
                    } else {
                        v[n++] = th[col];
                    }
                }
                if (n > 0) stats(v, n, o);
            }
            mean[j * nc + col] = o[0];
            sd[j * nc + col] = o[1];
            lo[j * nc + col] = o[2];
            hi[j * nc + col] = o[3];
        }
    }
    free(v);
    return 0;
}

/* Response function of the lp-ntPET model (Sec. II-D, the response-function
 * figure): k2a(t) / k2a = 1 + (gamma / k2a) g(t), with k2a = k2 / (1 + BP_ND) and g
 * the gamma variate above.  For voxel j, over its accepted draws whose global
 * index lies in [first, last) (the lp-ntPET draws: columns R1, k2, BP_ND, gamma,
 * t_D, t_P - t_D, alpha), at each time t[m]: the posterior mean and the 0.025 /
 * 0.975 type-7 quantiles of the response.  NaN where no accepted draw qualifies.
 * Pinned by: gamma = 0 (flat response 1), times before every t_D (1), a single
 * accepted draw at t = t_P (1 + gamma / k2a exactly), and numpy's quantiles of
 * values computed from the closed form of g in tests/test_oracle_sim.py. */
int orc_response_cri(const float* theta, int ldtheta, const int32_t* idx, int64_t J, int k, int64_t first,
                     int64_t last, const double* t, int T, double* mean, double* lo, double* hi) {
    double* v = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int64_t j = 0; j < J; ++j)
        for (int m = 0; m < T; ++m) {
            int n = 0;
            for (int r = 0; r < k; ++r) {
                const int64_t i = idx[j * k + r];
                if (i < first || i >= last) continue;
                const float* th = theta + i * ldtheta;
                const double k2a = (double)th[1] / (1.0 + (double)th[2]);
                const double tD = th[4], tP = (double)th[4] + (double)th[5];
                v[n++] = 1.0 + (double)th[3] / k2a * orc_gamma_variate(t[m], tD, tP, th[6]);
            }
            double o[4] = {NAN, NAN, NAN, NAN};
            if (n > 0) stats(v, n, o);
            mean[j * T + m] = o[0];
            lo[j * T + m] = o[2];
            hi[j * T + m] = o[3];
        }
    free(v);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------ learned proposal (build extra) */
/* Standard normal density, CDF (via erfc) and quantile (Newton iterations on
 * the CDF to full double precision; no tables).  Pinned against scipy's ndtr /
 * ndtri in tests/test_oracle_learned.py. */
static double nphi(double z) { return exp(-0.5 * z * z) / sqrt(2.0 * M_PI); }
double orc_Phi(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }
/* Lower-half quantile (p <= 0.5), where Phi(x) - p keeps full relative precision. */
static double phi_inv_lower(double p) {
    double x = log(p / (1.0 - p)) * 0.6266570686577501;   /* logistic start, sqrt(pi/8) */
    for (int it = 0; it < 200; ++it) {
        const double f = orc_Phi(x) - p;
        const double d = nphi(x);
        double step = d > 1e-300 ? f / d : (f > 0 ? 0.5 : -0.5);
        if (step > 1.0) step = 1.0;
        if (step < -1.0) step = -1.0;
        x -= step;
        if (fabs(step) < 1e-15 * (1.0 + fabs(x))) break;
    }
    return x;
}

double orc_Phi_inv(double p) {
    if (p <= 0.0) return -INFINITY;
    if (p >= 1.0) return INFINITY;
    return p <= 0.5 ? phi_inv_lower(p) : -phi_inv_lower(1.0 - p);   /* 1 - p is exact for p >= 0.5 */
}

/* Truncated normal N(mu, sigma^2) on [0, 1] by inverse CDF of a uniform u in (0,1):
 * t = mu + sigma Phi^-1(Phi(a) + u (Phi(b) - Phi(a))), a = -mu/sigma, b = (1-mu)/sigma. */
double orc_truncnorm01(double mu, double sigma, double u) {
    const double a = -mu / sigma, b = (1.0 - mu) / sigma;
    const double Pa = orc_Phi(a), Pb = orc_Phi(b);
    double t = mu + sigma * orc_Phi_inv(Pa + u * (Pb - Pa));
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    return t;
}

/* log density of that truncated normal at t in [0, 1]. */
double orc_truncnorm01_logpdf(double mu, double sigma, double t) {
    const double a = -mu / sigma, b = (1.0 - mu) / sigma, z = (t - mu) / sigma;
    return -0.5 * z * z - 0.5 * log(2.0 * M_PI) - log(sigma) - log(orc_Phi(b) - orc_Phi(a));
}

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
static double gelu_d(double z) { return orc_Phi(z) + z * nphi(z); }

/* MLP proposal network, FP64.  params layout: W1 (H x D), b1 (H), W2 (H x H), b2 (H),
 * W3 (O x H), b3 (O), row-major; weights are used rounded to bf16 (the caller
 * passes them already rounded).  out: B x O.  z1, z2 (B x H) hold pre-activations. */
void orc_mlp_forward(const double* prm, int D, int H, int O, const double* X, int B, double* out, double* z1,
                     double* z2) {
    const double *W1 = prm, *b1 = W1 + (size_t)H * D, *W2 = b1 + H, *b2 = W2 + (size_t)H * H, *W3 = b2 + H,
                 *b3 = W3 + (size_t)O * H;
    double* h1 = (double*)malloc(sizeof(double) * H);
    double* h2 = (double*)malloc(sizeof(double) * H);
    for (int n = 0; n < B; ++n) {
        const double* x = X + (size_t)n * D;
        for (int o = 0; o < H; ++o) {
            double s = b1[o];
            for (int i = 0; i < D; ++i) s += W1[(size_t)o * D + i] * x[i];
            z1[(size_t)n * H + o] = s;
            h1[o] = gelu(s);
        }
        for (int o = 0; o < H; ++o) {
            double s = b2[o];
            for (int i = 0; i < H; ++i) s += W2[(size_t)o * H + i] * h1[i];
            z2[(size_t)n * H + o] = s;
            h2[o] = gelu(s);
        }
        for (int o = 0; o < O; ++o) {
            double s = b3[o];
            for (int i = 0; i < H; ++i) s += W3[(size_t)o * H + i] * h2[i];
            out[(size_t)n * O + o] = s;
        }
    }
    free(h1);
    free(h2);
}

/* Mean truncated-normal negative log likelihood of targets T (B x P, in [0,1])
 * under the network outputs (mu_p, log sigma_p) = (out[2p], out[2p+1]), with
 * mu clamped to [-3, 4] and log sigma to [-7, 2] (zero gradient outside), and
 * the analytic gradient of that mean w.r.t. every parameter (grad, same layout). */
double orc_mlp_loss_grad(const double* prm, int D, int H, int P, const double* X, const double* T, int B,
                         double* grad) {
    const int O = 2 * P;
    const double *W1 = prm, *W2 = prm + (size_t)H * D + H, *W3 = W2 + (size_t)H * H + H;
    double* out = (double*)malloc(sizeof(double) * (size_t)B * O);
    double* z1 = (double*)malloc(sizeof(double) * (size_t)B * H);
    double* z2 = (double*)malloc(sizeof(double) * (size_t)B * H);
    orc_mlp_forward(prm, D, H, O, X, B, out, z1, z2);
    const size_t np = (size_t)H * D + H + (size_t)H * H + H + (size_t)O * H + O;
    memset(grad, 0, sizeof(double) * np);
    double *gW1 = grad, *gb1 = gW1 + (size_t)H * D, *gW2 = gb1 + H, *gb2 = gW2 + (size_t)H * H, *gW3 = gb2 + H,
           *gb3 = gW3 + (size_t)O * H;
    double loss = 0.0;
    double* dout = (double*)malloc(sizeof(double) * O);
    double* dh2 = (double*)malloc(sizeof(double) * H);
    double* dh1 = (double*)malloc(sizeof(double) * H);
    for (int n = 0; n < B; ++n) {
        for (int p = 0; p < P; ++p) {
            double mu = out[(size_t)n * O + 2 * p], s = out[(size_t)n * O + 2 * p + 1];
            const int mu_in = mu >= -3.0 && mu <= 4.0, s_in = s >= -7.0 && s <= 2.0;
            mu = mu < -3.0 ? -3.0 : (mu > 4.0 ? 4.0 : mu);
            s = s < -7.0 ? -7.0 : (s > 2.0 ? 2.0 : s);
            const double sg = exp(s), t = T[(size_t)n * P + p];
            const double z = (t - mu) / sg, a = -mu / sg, b = (1.0 - mu) / sg;
            const double Z = orc_Phi(b) - orc_Phi(a);
            loss += s + 0.5 * z * z + log(Z) + 0.5 * log(2.0 * M_PI);
            const double dmu = -z / sg + (nphi(a) - nphi(b)) / (sg * Z);
            const double ds = 1.0 - z * z + (a * nphi(a) - b * nphi(b)) / Z;
            dout[2 * p] = mu_in ? dmu / B : 0.0;
            dout[2 * p + 1] = s_in ? ds / B : 0.0;
        }
        const double* x = X + (size_t)n * D;
        /* layer 3 */
        for (int i = 0; i < H; ++i) dh2[i] = 0.0;
        for (int o = 0; o < O; ++o) {
            gb3[o] += dout[o];
            for (int i = 0; i < H; ++i) {
                const double h2 = gelu(z2[(size_t)n * H + i]);
                gW3[(size_t)o * H + i] += dout[o] * h2;
                dh2[i] += dout[o] * W3[(size_t)o * H + i];
            }
        }
        /* layer 2 */
        for (int i = 0; i < H; ++i) dh1[i] = 0.0;
        for (int o = 0; o < H; ++o) {
            const double dz = dh2[o] * gelu_d(z2[(size_t)n * H + o]);
            gb2[o] += dz;
            for (int i = 0; i < H; ++i) {
                gW2[(size_t)o * H + i] += dz * gelu(z1[(size_t)n * H + i]);
                dh1[i] += dz * W2[(size_t)o * H + i];
            }
        }
        /* layer 1 */
        for (int o = 0; o < H; ++o) {
            const double dz = dh1[o] * gelu_d(z1[(size_t)n * H + o]);
            gb1[o] += dz;
            for (int i = 0; i < D; ++i) gW1[(size_t)o * D + i] += dz * x[i];
        }
    }
    free(out); free(z1); free(z2); free(dout); free(dh2); free(dh1);
    return loss / B;
}

/* Importance-weighted local ABC for one voxel (build extra): proposals u (M x P in
 * [0,1]) with their truncated-normal parameters (mu, sigma per p), simulated TACs
 * x (M x L), the voxel TAC y, weights w; the k nearest proposals by (d, index)
 * are accepted, weighted by prior/proposal = 1/q(u) (uniform prior on the box),
 * normalised over the accepted set.  theta = lo + (hi - lo) u.  Outputs per
 * column (P parameters, then K_i if ki): weighted mean, weighted SD (sum W (t-m)^2
 * with W normalised), and weighted 2.5 / 97.5 % quantiles (smallest value whose
 * cumulative weight reaches q); ess = 1 / sum W^2; idx = accepted proposals. */
void orc_local_abc(const double* u, const double* mu, const double* sigma, int P, int M, const double* x, int L,
                   const float* y, const double* w, int k, const double* lo, const double* hi, int ki,
                   int32_t* idx, double* mean, double* sd, double* qlo, double* qhi, double* ess) {
    di_pair* buf = (di_pair*)malloc(sizeof(di_pair) * (size_t)M);
    for (int i = 0; i < M; ++i) { buf[i].d = wdist(y, x + (size_t)i * L, w, L); buf[i].i = i; }
    qsort(buf, (size_t)M, sizeof(di_pair), di_cmp);
    double* lw = (double*)malloc(sizeof(double) * k);
    double mx = -INFINITY;
    for (int r = 0; r < k; ++r) {
        const int i = (int)buf[r].i;
        idx[r] = i;
        double l = 0.0;
        for (int p = 0; p < P; ++p) l -= orc_truncnorm01_logpdf(mu[p], sigma[p], u[(size_t)i * P + p]);
        lw[r] = l;
        if (l > mx) mx = l;
    }
    double sw = 0.0, sw2 = 0.0;
    for (int r = 0; r < k; ++r) { lw[r] = exp(lw[r] - mx); sw += lw[r]; }
    for (int r = 0; r < k; ++r) { lw[r] /= sw; sw2 += lw[r] * lw[r]; }
    *ess = 1.0 / sw2;
    const int nc = P + (ki ? 1 : 0);
    double* v = (double*)malloc(sizeof(double) * k);
    di_pair* srt = (di_pair*)malloc(sizeof(di_pair) * (size_t)k);
    for (int c = 0; c < nc; ++c) {
        double m = 0.0;
        for (int r = 0; r < k; ++r) {
            const double* uu = u + (size_t)idx[r] * P;
            if (c < P) v[r] = lo[c] + (hi[c] - lo[c]) * uu[c];
            else {
                const double K1 = lo[0] + (hi[0] - lo[0]) * uu[0], k2 = lo[1] + (hi[1] - lo[1]) * uu[1],
                             k3 = lo[2] + (hi[2] - lo[2]) * uu[2];
                v[r] = K1 * k3 / (k2 + k3);
            }
            m += lw[r] * v[r];
        }
        double var = 0.0;
        for (int r = 0; r < k; ++r) var += lw[r] * (v[r] - m) * (v[r] - m);
        for (int r = 0; r < k; ++r) { srt[r].d = v[r]; srt[r].i = r; }
        qsort(srt, (size_t)k, sizeof(di_pair), di_cmp);
        double cum = 0.0, ql = srt[k - 1].d, qh = srt[k - 1].d;
        int got_l = 0, got_h = 0;
        for (int r = 0; r < k; ++r) {
            cum += lw[srt[r].i];
            if (!got_l && cum >= 0.025) { ql = srt[r].d; got_l = 1; }
            if (!got_h && cum >= 0.975) { qh = srt[r].d; got_h = 1; }
        }
        mean[c] = m; sd[c] = sqrt(var); qlo[c] = ql; qhi[c] = qh;
    }
    free(buf); free(lw); free(v); free(srt);
}
