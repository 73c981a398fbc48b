/*
 * hawkes_oracle.c -- plain FP64 CPU oracle for the spatiotemporal Hawkes
 * log-likelihood with per-event rates, its gradient and its Hessian diagonal.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares nothing with
 * the CUDA library: no headers, no helpers, no constants.
 *
 * What it computes (Holbrook, Ji & Suchard, arXiv 2103.03348):
 *
 *   intensity (Section 2.1)       lambda(x,t) = mu(x,t) + xi(x,t)
 *   background (Section 2.1, with the temporal bandwidth reading below)
 *       mu(x,t) = mu0 * sum_{n'} tau_x^-2 phi2((x-x_n')/tau_x) tau_t^-1 phi1((t-t_n')/tau_t) I[x != x_n']
 *   self-excitation (Section 2.1, rates theta_n = exp(r_n), Section 2.2)
 *       xi(x,t) = theta0*omega*h^-2 sum_{t_n' < t} theta_n' exp(-omega (t-t_n')) phi2((x-x_n')/h)
 *   integral (Appendix A Claim, background integrated exactly over R^2 x [0,t_N])
 *       Lambda = mu0 sum_n' [Phi((t_N-t_n')/tau_t) - Phi(-t_n'/tau_t)]
 *              + theta0 sum_n' theta_n' (1 - exp(-omega (t_N - t_n')))
 *   log-likelihood (Eq. 1)        l = sum_n log lambda(x_n, t_n) - Lambda
 *   gradient w.r.t. log-rates (Eq. 4 times theta_m) and Hessian diagonal
 *   w.r.t. log-rates (Eq. 5 times theta_m^2 plus the chain-rule term); the
 *   gradient and Hessian diagonal w.r.t. the six globals come from the same
 *   definitions, differentiated term by term.
 *
 * Readings where the paper is silent or inconsistent:
 *   - tau_t: the paper's background is spatial only.  tau_t = +inf selects the
 *     paper's mu(x) = mu0 tau_x^-2 sum phi2(...) I[...], whose integral is
 *     mu0 * N * t_N.  A finite tau_t multiplies every background kernel by a
 *     normalised Gaussian in time.
 *   - The background indicator excludes a source whose stored location equals
 *     the target's exactly (which includes the event itself).
 *   - Excitation is strict: t_n' < t_n.  Simultaneous events do not excite.
 *   - t_N is the largest event time; integration starts at time 0.
 *
 * Everything is a straightforward double loop in FP64 with libm exp/log/erfc,
 * sources visited in input order.  OpenMP, when compiled in, only splits the
 * independent outer rows; every per-row sum keeps the sequential order, and
 * the cross-row totals are summed sequentially afterwards, so the result does
 * not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NPAR 6
enum { P_MU0 = 0, P_TAUX = 1, P_TAUT = 2, P_THETA0 = 3, P_OMEGA = 4, P_H = 5 };

static const double TWO_PI = 6.283185307179586476925286766559;

/* Standard normal pdf and cdf, from their definitions (cdf via libm erfc). */
static double std_normal_pdf(double z) { return exp(-0.5 * z * z) / sqrt(TWO_PI); }
static double std_normal_cdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

/*
 * One source's contribution to the intensity at (xq, yq, tq), and the first and
 * second derivatives of that contribution with respect to each global
 * parameter.  Returns the contribution; fills d1[6], d2[6] when non-NULL.
 *
 * Background term  g = mu0 (2 pi tau_x^2)^-1 exp(-d^2/(2 tau_x^2))
 *                        * (2 pi tau_t^2)^-1/2 exp(-dt^2/(2 tau_t^2))     (tau_t finite)
 * For a factor f(tau) = tau^-k exp(-s/(2 tau^2)):
 *     f'/f  = s/tau^3 - k/tau,
 *     f''/f = (s/tau^3 - k/tau)^2 - 3 s/tau^4 + k/tau^2.
 * Excitation term  e = theta0 omega (2 pi h^2)^-1 theta_src exp(-omega dt) exp(-d^2/(2 h^2))
 *     de/domega = e (1/omega - dt),  d2e/domega2 = e (dt^2 - 2 dt/omega).
 */
static double source_term(double xq, double yq, double tq,
                          double xs, double ys, double ts, double rs,
                          const double *p, int strict_bg_exclusion,
                          double *bg_out, double *d1, double *d2)
{
    const double mu0 = p[P_MU0], tx = p[P_TAUX], tt = p[P_TAUT];
    const double th0 = p[P_THETA0], om = p[P_OMEGA], h = p[P_H];
    const double dx = xq - xs, dy = yq - ys, dt = tq - ts;
    const double dsq = dx * dx + dy * dy;
    double total = 0.0, g = 0.0, e = 0.0;
    int k;
    if (d1) for (k = 0; k < NPAR; k++) { d1[k] = 0.0; d2[k] = 0.0; }

    /* background: excluded when the locations coincide exactly */
    if (!(strict_bg_exclusion && xq == xs && yq == ys)) {
        const double space = exp(-dsq / (2.0 * tx * tx)) / (TWO_PI * tx * tx);
        double time = 1.0;
        if (isfinite(tt)) time = exp(-dt * dt / (2.0 * tt * tt)) / (sqrt(TWO_PI) * tt);
        g = mu0 * space * time;
        total += g;
        if (d1) {
            double a, b;
            d1[P_MU0] += g / mu0;
            a = dsq / (tx * tx * tx) - 2.0 / tx;
            d1[P_TAUX] += g * a;
            d2[P_TAUX] += g * (a * a - 3.0 * dsq / (tx * tx * tx * tx) + 2.0 / (tx * tx));
            if (isfinite(tt)) {
                const double s = dt * dt;
                b = s / (tt * tt * tt) - 1.0 / tt;
                d1[P_TAUT] += g * b;
                d2[P_TAUT] += g * (b * b - 3.0 * s / (tt * tt * tt * tt) + 1.0 / (tt * tt));
            }
        }
    }
    /* self-excitation: strictly earlier sources only */
    if (ts < tq) {
        /* e_unit = e / theta0, so that de/dtheta0 stays finite at theta0 = 0 */
        const double e_unit = om * exp(rs) * exp(-om * dt) * exp(-dsq / (2.0 * h * h)) / (TWO_PI * h * h);
        e = th0 * e_unit;
        total += e;
        if (d1) {
            double c;
            d1[P_THETA0] += e_unit;
            d1[P_OMEGA] += e * (1.0 / om - dt);
            d2[P_OMEGA] += e * (dt * dt - 2.0 * dt / om);
            c = dsq / (h * h * h) - 2.0 / h;
            d1[P_H] += e * c;
            d2[P_H] += e * (c * c - 3.0 * dsq / (h * h * h * h) + 2.0 / (h * h));
        }
    }
    if (bg_out) *bg_out = g;
    return total;
}

/* Excitation term from source m at target n alone (0 unless t_m < t_n). */
static double excitation_term(double xn, double yn, double tn,
                              double xm, double ym, double tm, double rm, const double *p)
{
    const double th0 = p[P_THETA0], om = p[P_OMEGA], h = p[P_H];
    const double dx = xn - xm, dy = yn - ym, dt = tn - tm;
    if (!(tm < tn)) return 0.0;
    return th0 * om * exp(rm) * exp(-om * dt) * exp(-(dx * dx + dy * dy) / (2.0 * h * h)) / (TWO_PI * h * h);
}

static int params_ok(const double *p)
{
    int k;
    for (k = 0; k < NPAR; k++) {
        if (k == P_TAUT && isinf(p[k]) && p[k] > 0) continue;
        if (!isfinite(p[k])) return 0;
    }
    /* theta0 = 0 is allowed here (the background-only limit); the rest must be > 0 */
    return p[P_MU0] > 0 && p[P_TAUX] > 0 && p[P_TAUT] > 0 && p[P_THETA0] >= 0 && p[P_OMEGA] > 0 && p[P_H] > 0;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Intensity lambda(x_q, t_q) at arbitrary query points, given the events.
 * A query at an event's own location excludes that event's background kernel,
 * exactly as lambda_n does.  Returns 0, or -1 on bad arguments.
 */
int oracle_intensity(int64_t n, const double *x, const double *y, const double *t, const double *r,
                     const double *params, int64_t q, const double *xq, const double *yq,
                     const double *tq, double *out, int nthreads)
{
    int64_t i;
    if (n < 0 || q < 0 || !params_ok(params)) return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < q; i++) {
        int64_t j;
        double s = 0.0;
        for (j = 0; j < n; j++)
            s += source_term(xq[i], yq[i], tq[i], x[j], y[j], t[j], r[j], params, 1, NULL, NULL, NULL);
        out[i] = s;
    }
    return 0;
}

/*
 * The integral term Lambda and its derivatives (Appendix A Claim, with the
 * background integrated exactly).  dL[6], d2L[6] w.r.t. the globals and
 * dLr[n] (= d2 Lambda / d r_m^2 as well) w.r.t. the log-rates; any may be NULL.
 */
static double integral_term(int64_t n, const double *t, const double *r, const double *p,
                            double *dL, double *d2L, double *dLr)
{
    const double mu0 = p[P_MU0], tt = p[P_TAUT], th0 = p[P_THETA0], om = p[P_OMEGA];
    double tN = -INFINITY, bg = 0.0, ex = 0.0;
    double d_tt = 0.0, d2_tt = 0.0, d_th0 = 0.0, d_om = 0.0, d2_om = 0.0;
    int64_t i;
    int k;
    for (i = 0; i < n; i++) if (t[i] > tN) tN = t[i];
    for (i = 0; i < n; i++) {
        const double a = tN - t[i], b = -t[i];
        const double th = exp(r[i]);
        const double decay = exp(-om * a);
        if (isfinite(tt)) {
            const double za = a / tt, zb = b / tt;
            bg += std_normal_cdf(za) - std_normal_cdf(zb);
            /* d/dtau Phi(c/tau) = -(c/tau^2) phi(c/tau);
               d2/dtau2 Phi(c/tau) = phi(c/tau) (2c/tau^3 - c^3/tau^5) */
            d_tt += -(a / (tt * tt)) * std_normal_pdf(za) + (b / (tt * tt)) * std_normal_pdf(zb);
            d2_tt += std_normal_pdf(za) * (2.0 * a / (tt * tt * tt) - a * a * a / pow(tt, 5))
                   - std_normal_pdf(zb) * (2.0 * b / (tt * tt * tt) - b * b * b / pow(tt, 5));
        } else {
            bg += tN; /* each spatial kernel integrates to 1 over R^2, for a duration t_N */
        }
        ex += th * (1.0 - decay);
        d_th0 += th * (1.0 - decay);
        d_om += th0 * th * a * decay;
        d2_om += -th0 * th * a * a * decay;
        if (dLr) dLr[i] = th0 * th * (1.0 - decay);
    }
    if (dL) {
        for (k = 0; k < NPAR; k++) { dL[k] = 0.0; d2L[k] = 0.0; }
        dL[P_MU0] = bg;
        dL[P_TAUT] = mu0 * d_tt;
        d2L[P_TAUT] = mu0 * d2_tt;
        dL[P_THETA0] = d_th0;
        dL[P_OMEGA] = d_om;
        d2L[P_OMEGA] = d2_om;
    }
    return mu0 * bg + th0 * ex;
}

/*
 * Full evaluation.
 *   want: 0 = log-likelihood only, 1 = + gradient, 2 = + gradient + Hessian diagonal.
 *   grad, hdiag: [6 + n], globals first (mu0, tau_x, tau_t, theta0, omega, h),
 *   then the log-rates in input order.  lambda_out[n] and Lambda_out optional.
 * Returns 0; -1 on bad arguments; 1 when some lambda_n is 0 (loglik = -inf).
 */
int oracle_eval(int64_t n, const double *x, const double *y, const double *t, const double *r,
                const double *params, int want, double *loglik, double *grad, double *hdiag,
                double *lambda_out, double *Lambda_out, int nthreads)
{
    double *lam, *rowd1, *rowd2, *c1, *c2;
    double dL[NPAR], d2L[NPAR], Lam, ll = 0.0;
    double *dLr;
    int64_t i;
    int k, zero = 0;
    if (n < 1 || !params_ok(params) || !x || !y || !t || !r || !loglik) return -1;
    if (want >= 1 && !grad) return -1;
    if (want >= 2 && !hdiag) return -1;
    set_threads(nthreads);

    lam = (double *)malloc(sizeof(double) * n);
    rowd1 = (double *)calloc((size_t)n * NPAR, sizeof(double));
    rowd2 = (double *)calloc((size_t)n * NPAR, sizeof(double));
    c1 = (double *)calloc((size_t)n, sizeof(double));
    c2 = (double *)calloc((size_t)n, sizeof(double));
    dLr = (double *)calloc((size_t)n, sizeof(double));
    if (!lam || !rowd1 || !rowd2 || !c1 || !c2 || !dLr) {
        free(lam); free(rowd1); free(rowd2); free(c1); free(c2); free(dLr);
        return -1;
    }

    /* rows: lambda_n and sum over sources of the per-pair derivatives */
#pragma omp parallel for schedule(dynamic, 8)
    for (i = 0; i < n; i++) {
        double s = 0.0, a1[NPAR] = {0}, a2[NPAR] = {0}, p1[NPAR], p2[NPAR];
        int64_t j;
        int kk;
        for (j = 0; j < n; j++) {
            s += source_term(x[i], y[i], t[i], x[j], y[j], t[j], r[j], params, 1, NULL,
                             want >= 1 ? p1 : NULL, want >= 1 ? p2 : NULL);
            if (want >= 1)
                for (kk = 0; kk < NPAR; kk++) { a1[kk] += p1[kk]; a2[kk] += p2[kk]; }
        }
        lam[i] = s;
        for (kk = 0; kk < NPAR; kk++) { rowd1[i * NPAR + kk] = a1[kk]; rowd2[i * NPAR + kk] = a2[kk]; }
    }

    Lam = integral_term(n, t, r, params, dL, d2L, dLr);
    for (i = 0; i < n; i++) {
        if (!(lam[i] > 0.0)) zero = 1;
        ll += log(lam[i]);
    }
    *loglik = ll - Lam;
    if (lambda_out) memcpy(lambda_out, lam, sizeof(double) * n);
    if (Lambda_out) *Lambda_out = Lam;

    if (want >= 1) {
        /* globals: sum_n dlambda_n/lambda_n - dLambda; Hessian diagonal adds
           sum_n [d2lambda_n/lambda_n - (dlambda_n/lambda_n)^2] - d2Lambda */
        for (k = 0; k < NPAR; k++) {
            double g = 0.0, hh = 0.0;
            for (i = 0; i < n; i++) {
                const double q1 = rowd1[i * NPAR + k] / lam[i];
                g += q1;
                hh += rowd2[i * NPAR + k] / lam[i] - q1 * q1;
            }
            grad[k] = g - dL[k];
            if (want >= 2) hdiag[k] = hh - d2L[k];
        }
        if (!isfinite(params[P_TAUT])) {
            grad[P_TAUT] = 0.0;
            if (want >= 2) hdiag[P_TAUT] = 0.0;
        }
        /* log-rates (Eqs. 4, 5): sum over later targets n of e_nm / lambda_n */
#pragma omp parallel for schedule(dynamic, 8)
        for (i = 0; i < n; i++) {
            double s1 = 0.0, s2 = 0.0;
            int64_t j;
            for (j = 0; j < n; j++) {
                const double e = excitation_term(x[j], y[j], t[j], x[i], y[i], t[i], r[i], params);
                if (e != 0.0) {
                    const double w = e / lam[j];
                    s1 += w;
                    s2 += w * w;
                }
            }
            c1[i] = s1;
            c2[i] = s2;
        }
        for (i = 0; i < n; i++) {
            grad[NPAR + i] = c1[i] - dLr[i];
            if (want >= 2) hdiag[NPAR + i] = c1[i] - c2[i] - dLr[i];
        }
    }
    free(lam); free(rowd1); free(rowd2); free(c1); free(c2); free(dLr);
    return zero ? 1 : 0;
}

/*
 * Integral term alone, exposed for the closed-form checks (Appendix A Claim).
 */
double oracle_integral(int64_t n, const double *t, const double *r, const double *params)
{
    if (n < 1 || !params_ok(params)) return NAN;
    return integral_term(n, t, r, params, NULL, NULL, NULL);
}

/*
 * Sampled rows: lambda_n and the sums over sources of the per-pair first and
 * second derivatives (w.r.t. the six globals) for the k rows listed in idx.
 * Same per-pair code and order as oracle_eval's rows.  lam[k], d1[k*6], d2[k*6].
 */
int oracle_rows(int64_t n, const double *x, const double *y, const double *t, const double *r,
                const double *params, int64_t k, const int64_t *idx, double *lam, double *d1, double *d2,
                int nthreads)
{
    int64_t q;
    if (n < 1 || k < 0 || !params_ok(params)) return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (q = 0; q < k; q++) {
        const int64_t i = idx[q];
        double s = 0.0, a1[NPAR] = {0}, a2[NPAR] = {0}, p1[NPAR], p2[NPAR];
        int64_t j;
        int kk;
        for (j = 0; j < n; j++) {
            s += source_term(x[i], y[i], t[i], x[j], y[j], t[j], r[j], params, 1, NULL, p1, p2);
            for (kk = 0; kk < NPAR; kk++) { a1[kk] += p1[kk]; a2[kk] += p2[kk]; }
        }
        lam[q] = s;
        for (kk = 0; kk < NPAR; kk++) { d1[q * NPAR + kk] = a1[kk]; d2[q * NPAR + kk] = a2[kk]; }
    }
    return 0;
}

/*
 * Sampled log-rate outputs (Eqs. 4-5 times theta_m): for each source m in idx,
 *   g_m = sum_{t_n > t_m} e_nm / lambda_n - theta0 theta_m (1 - exp(-omega (t_N - t_m)))
 *   h_m = g_m - sum_{t_n > t_m} (e_nm / lambda_n)^2
 * given lambda[n] for every target n with t_n > t_m (other entries unused).
 */
int oracle_rate_terms(int64_t n, const double *x, const double *y, const double *t, const double *r,
                      const double *params, const double *lambda, int64_t k, const int64_t *idx,
                      double *g, double *h, int nthreads)
{
    int64_t q, j;
    double tN = -INFINITY;
    if (n < 1 || k < 0 || !params_ok(params)) return -1;
    set_threads(nthreads);
    for (j = 0; j < n; j++) if (t[j] > tN) tN = t[j];
#pragma omp parallel for schedule(dynamic, 1)
    for (q = 0; q < k; q++) {
        const int64_t m = idx[q];
        double s1 = 0.0, s2 = 0.0, dl;
        int64_t j;
        for (j = 0; j < n; j++) {
            const double e = excitation_term(x[j], y[j], t[j], x[m], y[m], t[m], r[m], params);
            if (e != 0.0) {
                const double w = e / lambda[j];
                s1 += w;
                s2 += w * w;
            }
        }
        dl = params[P_THETA0] * exp(r[m]) * (1.0 - exp(-params[P_OMEGA] * (tN - t[m])));
        g[q] = s1 - dl;
        h[q] = s1 - s2 - dl;
    }
    return 0;
}
