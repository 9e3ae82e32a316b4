/*
 * Plain FP64 CPU oracle — see pepic_oracle.h for the contract.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the GPU product path.
 *
 * Compiled with -O2 -ffp-contract=off so that no multiply-add is fused behind
 * the reader's back. Every loop is the textbook statement of its step.
 */
#include "pepic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define THETA_ONE 16777216.0 /* 2^24: resolution of the in-cell offset in the deposit rule */

uint64_t orc_splitmix64(uint64_t x)
{
    /* splitmix64 output function applied to the counter x (Steele, Lea, Flood 2014). */
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

int32_t orc_fx_shift(double cap)
{
    int e = 0;
    double m = frexp(cap, &e); /* cap = m 2^e, m in [0.5, 1) */
    int ceil_log2 = (m == 0.5) ? e - 1 : e;
    return 22 - ceil_log2;
}

static int32_t wrap(int64_t j, int32_t n)
{
    int64_t r = j % n;
    if (r < 0) r += n;
    return (int32_t)r;
}

/* ---------------------------------------------------------------- deposit */

void orc_deposit_fx(int64_t n, const int32_t* cell, const double* theta, const double* w,
                    int32_t ncell, int32_t s_w, int64_t* rho)
{
    memset(rho, 0, sizeof(int64_t) * (size_t)ncell);
    const double wscale = ldexp(1.0, s_w);
    for (int64_t p = 0; p < n; ++p) {
        int64_t tq = llrint(theta[p] * THETA_ONE); /* round half to even */
        int64_t wq = llrint(w[p] * wscale);
        int64_t qr = wq * tq;
        int64_t ql = wq * (int64_t)THETA_ONE - qr;
        int32_t j = cell[p];
        rho[j] += ql;
        rho[wrap((int64_t)j + 1, ncell)] += qr;
    }
}

void orc_deposit_f64(int64_t n, const int32_t* cell, const double* theta, const double* w,
                     const double* vel, int32_t ncell, double* dens, double* mom)
{
    memset(dens, 0, sizeof(double) * (size_t)ncell);
    if (mom) memset(mom, 0, sizeof(double) * (size_t)ncell);
    for (int64_t p = 0; p < n; ++p) {
        int32_t j = cell[p], j1 = wrap((int64_t)j + 1, ncell);
        dens[j] += w[p] * (1.0 - theta[p]);
        dens[j1] += w[p] * theta[p];
        if (mom) {
            double wv = w[p] * vel[p];
            mom[j] += wv * (1.0 - theta[p]);
            mom[j1] += wv * theta[p];
        }
    }
}

/* ---------------------------------------------------------------- field */

static void thomas(int32_t n, double a, const double* b, double c, const double* d, double* x)
{
    double* cp = (double*)malloc(sizeof(double) * (size_t)n);
    double* dp = (double*)malloc(sizeof(double) * (size_t)n);
    cp[0] = c / b[0];
    dp[0] = d[0] / b[0];
    for (int32_t i = 1; i < n; ++i) {
        double m = b[i] - a * cp[i - 1];
        cp[i] = c / m;
        dp[i] = (d[i] - a * dp[i - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int32_t i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp);
    free(dp);
}

void orc_cyclic_tridiag(int32_t n, double a, const double* b, double c, const double* d, double* x)
{
    /* A = T + u v^T with u = (gamma, 0, .., 0, c)^T, v = (1, 0, .., 0, a/gamma)^T:
     * the corner entries A[0][n-1] = a and A[n-1][0] = c move into u v^T. */
    double gamma = -b[0];
    double* bb = (double*)malloc(sizeof(double) * (size_t)n);
    double* u = (double*)calloc((size_t)n, sizeof(double));
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(bb, b, sizeof(double) * (size_t)n);
    bb[0] = b[0] - gamma;
    bb[n - 1] = b[n - 1] - c * a / gamma;
    u[0] = gamma;
    u[n - 1] = c;
    thomas(n, a, bb, c, d, y);
    thomas(n, a, bb, c, u, z);
    double fact = (y[0] + a * y[n - 1] / gamma) / (1.0 + z[0] + a * z[n - 1] / gamma);
    for (int32_t i = 0; i < n; ++i) x[i] = y[i] - fact * z[i];
    free(bb);
    free(u);
    free(y);
    free(z);
}

int orc_newton_pb(int32_t ncell, double dx, int32_t mode, const double* n, double* phi,
                  double tol, int32_t maxit, int32_t* iters)
{
    const double inv_dx2 = 1.0 / (dx * dx);
    double* b = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* rhs = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* delta = (double*)malloc(sizeof(double) * (size_t)ncell);
    int status = 1;
    int32_t it = 0;
    for (it = 0; it < maxit; ++it) {
        for (int32_t j = 0; j < ncell; ++j) {
            double lap = (phi[wrap(j - 1, ncell)] - 2.0 * phi[j] + phi[wrap(j + 1, ncell)]) * inv_dx2;
            double g = (mode == 0) ? exp(phi[j]) : 1.0 + phi[j];
            double gp = (mode == 0) ? exp(phi[j]) : 1.0;
            double F = -lap + g - n[j];
            b[j] = 2.0 * inv_dx2 + gp;
            rhs[j] = -F;
        }
        orc_cyclic_tridiag(ncell, -inv_dx2, b, -inv_dx2, rhs, delta);
        double m = 0.0;
        for (int32_t j = 0; j < ncell; ++j) m = fmax(m, fabs(delta[j]));
        double scale = (m > 2.0) ? 2.0 / m : 1.0; /* damped step: |update| <= 2 */
        for (int32_t j = 0; j < ncell; ++j) phi[j] += scale * delta[j];
        if (m < tol) {
            status = 0;
            ++it;
            break;
        }
    }
    if (iters) *iters = it;
    free(b);
    free(rhs);
    free(delta);
    return status;
}

void orc_efield(int32_t ncell, double dx, const double* phi, double* E)
{
    for (int32_t j = 0; j < ncell; ++j)
        E[j] = -(phi[wrap(j + 1, ncell)] - phi[wrap(j - 1, ncell)]) / (2.0 * dx);
}

double orc_gather(const double* F, int32_t ncell, int32_t cell, double theta)
{
    return (1.0 - theta) * F[cell] + theta * F[wrap((int64_t)cell + 1, ncell)];
}

/* ---------------------------------------------------------------- push */

static void drift(int32_t* cell, double* theta, double shift_cells, int32_t ncell)
{
    double s = *theta + shift_cells;
    double k = floor(s);
    *theta = s - k;
    *cell = wrap((int64_t)*cell + (int64_t)k, ncell);
}

void orc_push(int64_t n, int32_t* cell, double* theta, double* v, const double* E,
              int32_t ncell, double dx, double dt, double qm, double kick)
{
    for (int64_t p = 0; p < n; ++p) {
        double Ep = orc_gather(E, ncell, cell[p], theta[p]);
        v[p] += kick * qm * dt * Ep;
        drift(&cell[p], &theta[p], v[p] * dt / dx, ncell);
    }
}

void orc_restrict_sample(int64_t n, const int32_t* cell, const double* theta, const double* vbar,
                         const double* w, const double* E0, int32_t ncell, double dx,
                         double tau, double qm, double* dens, double* mom)
{
    memset(dens, 0, sizeof(double) * (size_t)ncell);
    memset(mom, 0, sizeof(double) * (size_t)ncell);
    for (int64_t p = 0; p < n; ++p) {
        double E0p = orc_gather(E0, ncell, cell[p], theta[p]);
        int32_t c = cell[p];
        double th = theta[p];
        drift(&c, &th, tau * vbar[p] / dx, ncell);      /* X~ = X + tau V  */
        double vt = vbar[p] + qm * tau * E0p;            /* V~ = V + qm tau E_n(X) */
        int32_t c1 = wrap((int64_t)c + 1, ncell);
        dens[c] += w[p] * (1.0 - th);
        dens[c1] += w[p] * th;
        mom[c] += w[p] * vt * (1.0 - th);
        mom[c1] += w[p] * vt * th;
    }
}

/* ---------------------------------------------------------------- wavelets */

void orc_dwt_level(const double* h, int32_t len, const double* x, int32_t n, double* approx, double* detail)
{
    for (int32_t k = 0; k < n / 2; ++k) {
        double a = 0.0, d = 0.0;
        for (int32_t m = 0; m < len; ++m) {
            double g = ((m & 1) ? -1.0 : 1.0) * h[len - 1 - m];
            double xv = x[wrap(2 * (int64_t)k + m, n)];
            a += h[m] * xv;
            d += g * xv;
        }
        approx[k] = a;
        if (detail) detail[k] = d;
    }
}

void orc_idwt_level(const double* h, int32_t len, const double* approx, const double* detail,
                    int32_t nhalf, double* x)
{
    int32_t n = 2 * nhalf;
    memset(x, 0, sizeof(double) * (size_t)n);
    for (int32_t k = 0; k < nhalf; ++k) {
        for (int32_t m = 0; m < len; ++m) {
            double g = ((m & 1) ? -1.0 : 1.0) * h[len - 1 - m];
            x[wrap(2 * (int64_t)k + m, n)] += h[m] * approx[k] + g * (detail ? detail[k] : 0.0);
        }
    }
}

static int32_t ilog2(int32_t n)
{
    int32_t l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

void orc_coarsen(const double* h, int32_t len, const double* fine, int32_t nfine,
                 double* coarse, int32_t ncoarse)
{
    double* a = (double*)malloc(sizeof(double) * (size_t)nfine);
    double* t = (double*)malloc(sizeof(double) * (size_t)nfine);
    double s = pow(2.0, -0.5 * ilog2(nfine)); /* scaling coefficients at the finest level */
    for (int32_t j = 0; j < nfine; ++j) a[j] = s * fine[j];
    for (int32_t n = nfine; n > ncoarse; n /= 2) {
        orc_dwt_level(h, len, a, n, t, NULL);
        memcpy(a, t, sizeof(double) * (size_t)(n / 2));
    }
    memcpy(coarse, a, sizeof(double) * (size_t)ncoarse);
    free(a);
    free(t);
}

void orc_refine(const double* h, int32_t len, const double* coarse, int32_t ncoarse,
                double* fine, int32_t nfine)
{
    double* a = (double*)malloc(sizeof(double) * (size_t)nfine);
    double* t = (double*)malloc(sizeof(double) * (size_t)nfine);
    memcpy(a, coarse, sizeof(double) * (size_t)ncoarse);
    for (int32_t n = ncoarse; n < nfine; n *= 2) {
        orc_idwt_level(h, len, a, NULL, n, t);
        memcpy(a, t, sizeof(double) * (size_t)(2 * n));
    }
    double s = pow(2.0, 0.5 * ilog2(nfine));
    for (int32_t j = 0; j < nfine; ++j) fine[j] = s * a[j];
    free(a);
    free(t);
}

/* ---------------------------------------------------------------- projection */

double orc_ls_slope(int32_t K, double dt, const double* y, int64_t stride)
{
    double S0 = 0, S1 = 0, S2 = 0, Sy = 0, Sty = 0;
    for (int32_t p = 0; p <= K; ++p) {
        double t = p * dt, yp = y[(int64_t)p * stride];
        S0 += 1.0;
        S1 += t;
        S2 += t * t;
        Sy += yp;
        Sty += t * yp;
    }
    return (S0 * Sty - S1 * Sy) / (S0 * S2 - S1 * S1);
}

void orc_ls_project(int32_t K, int32_t ncoef, double dt, double dT, const double* samples,
                    double* coarse_out, double* slope_out)
{
    for (int32_t i = 0; i < ncoef; ++i) {
        double s = orc_ls_slope(K, dt, samples + i, ncoef);
        if (slope_out) slope_out[i] = s;
        coarse_out[i] = samples[(int64_t)K * ncoef + i] + (dT - K * dt) * s;
    }
}

/* ---------------------------------------------------------------- lifting */

static double std_normal_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

double orc_ndtri(double p)
{
    if (!(p > 0.0 && p < 1.0)) return (p <= 0.0) ? -INFINITY : INFINITY;
    int upper = p > 0.5;
    double q = upper ? 1.0 - p : p; /* tail probability, q <= 1/2 */
    double t = sqrt(-2.0 * log(q));
    /* Abramowitz & Stegun 26.2.23: upper-tail quantile, |error| < 4.5e-4 */
    double xq = t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                        (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t);
    double x = -xq; /* Phi(x) = q */
    for (int it = 0; it < 8; ++it) {
        double f = std_normal_cdf(x) - q;
        double dens = exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
        double step = f / dens;
        x -= step;
        if (fabs(step) < 1e-16 * fmax(1.0, fabs(x))) break;
    }
    return upper ? -x : x;
}

static uint32_t brev32(uint32_t x)
{
    uint32_t r = 0;
    for (int b = 0; b < 32; ++b) r |= ((x >> b) & 1u) << (31 - b);
    return r;
}

void orc_quiet_start(int64_t N, int32_t ncell, const double* nprof, const double* uprof,
                     double v_th, uint64_t seed, int32_t* cell, double* theta, double* v, double* w)
{
    int64_t ppc = N / ncell;
    uint32_t half = (uint32_t)(2147483648.0 / (double)N);
    uint32_t shift = (uint32_t)(orc_splitmix64(seed) >> 32);
    int m = 0;
    while (((int64_t)1 << m) < ppc) ++m;
    int pow2 = ((int64_t)1 << m) == ppc;
    for (int64_t s = 0; s < N; ++s) {
        /* storage slot s holds Hammersley point i; for ppc = 2^m a cell stores its points in
         * ascending velocity quantile: i = s with its low m bits reversed */
        int64_t i = s;
        if (pow2 && m > 0) {
            uint32_t k = (uint32_t)(s & (ppc - 1));
            uint32_t r = brev32(k) >> (32 - m);
            i = (s & ~(ppc - 1)) | (int64_t)r;
        }
        int32_t c = (int32_t)(i / ppc);
        double th = (2.0 * (double)(i % ppc) + 1.0) / (2.0 * (double)ppc);
        int32_t c1 = wrap((int64_t)c + 1, ncell);
        double nX = (1.0 - th) * nprof[c] + th * nprof[c1];
        double uX = (1.0 - th) * uprof[c] + th * uprof[c1];
        uint32_t B = brev32((uint32_t)i) + half + shift; /* mod 2^32 */
        double b = ((double)B + 0.5) * 2.3283064365386963e-10; /* 2^-32 */
        cell[s] = c;
        theta[s] = th;
        w[s] = nX / (double)ppc;
        v[s] = uX + v_th * orc_ndtri(b);
    }
}

void orc_lift_profile(int32_t ncell, double* n, const double* m, double* u)
{
    double sum0 = 0.0, sum1 = 0.0, nmax = 0.0;
    int clamped = 0;
    for (int32_t j = 0; j < ncell; ++j) sum0 += n[j];
    for (int32_t j = 0; j < ncell; ++j) {
        if (n[j] < 0.0) {
            n[j] = 0.0;
            clamped = 1;
        }
        sum1 += n[j];
    }
    if (clamped && sum1 > 0.0 && sum0 > 0.0)
        for (int32_t j = 0; j < ncell; ++j) n[j] *= sum0 / sum1;
    for (int32_t j = 0; j < ncell; ++j) nmax = fmax(nmax, n[j]);
    for (int32_t j = 0; j < ncell; ++j) u[j] = (n[j] > 1e-12 * nmax) ? m[j] / n[j] : 0.0;
}

/* ---------------------------------------------------------------- bursts */

static int field_from_particles(int64_t n, const int32_t* cell, const double* theta, const double* w,
                                int32_t ncell, double dx, int32_t mode, int32_t s_w, double tol,
                                int32_t maxit, double* phi, double* E)
{
    int64_t* rho = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    double* dens = (double*)malloc(sizeof(double) * (size_t)ncell);
    orc_deposit_fx(n, cell, theta, w, ncell, s_w, rho);
    double scale = ldexp(1.0, -(s_w + 24));
    for (int32_t j = 0; j < ncell; ++j) dens[j] = (double)rho[j] * scale;
    int32_t iters = 0;
    int fail = orc_newton_pb(ncell, dx, mode, dens, phi, tol, maxit, &iters);
    orc_efield(ncell, dx, phi, E);
    free(rho);
    free(dens);
    return fail;
}

int orc_burst(int64_t n, int32_t* cell, double* theta, double* v, const double* w,
              int32_t ncell, double dx, double dt, double qm, int32_t K, double dT,
              int32_t comoving, int32_t mode, int32_t s_w, double tol, int32_t maxit,
              int32_t vel_at_integer, double* phi, double* samples)
{
    double* E = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* E0 = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* vbar = (double*)malloc(sizeof(double) * (size_t)n);
    int fails = field_from_particles(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    memcpy(E0, E, sizeof(double) * (size_t)ncell); /* E_n, stored at burst start */
    double kick = vel_at_integer ? 0.5 : 1.0;
    for (int32_t p = 0; p <= K; ++p) {
        /* integer-time velocity: the half kick that takes v to time t_n + p dt */
        for (int64_t i = 0; i < n; ++i)
            vbar[i] = v[i] + (kick - 0.5) * qm * dt * orc_gather(E, ncell, cell[i], theta[i]);
        double tau = comoving ? dT - p * dt : 0.0;
        double* dens = samples + (size_t)p * 2 * ncell;
        orc_restrict_sample(n, cell, theta, vbar, w, E0, ncell, dx, tau, qm, dens, dens + ncell);
        if (p == K) break;
        orc_push(n, cell, theta, v, E, ncell, dx, dt, qm, kick);
        kick = 1.0;
        fails += field_from_particles(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    }
    free(E);
    free(E0);
    free(vbar);
    return fails;
}

int orc_pic_steps(int64_t n, int32_t* cell, double* theta, double* v, const double* w,
                  int32_t ncell, double dx, double dt, double qm, int32_t nsteps,
                  int32_t mode, int32_t s_w, double tol, int32_t maxit,
                  int32_t vel_at_integer, double* phi)
{
    double* E = (double*)malloc(sizeof(double) * (size_t)ncell);
    int fails = 0;
    double kick = vel_at_integer ? 0.5 : 1.0;
    for (int32_t s = 0; s < nsteps; ++s) {
        fails += field_from_particles(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
        orc_push(n, cell, theta, v, E, ncell, dx, dt, qm, kick);
        kick = 1.0;
    }
    free(E);
    return fails;
}

/* ---------------------------------------------------------------- diagnostics */

/* Conserved quantities of the ion-particle / Boltzmann-electron system. Velocities are
 * taken at integer time, Vbar = v + (kick - 1/2) qm dt E(X) (kick 1/2: v already at integer
 * time). Each particle carries charge w dx (n_j = sum_p w_p S_j(X_p) with unit mean).
 * The electron free energy follows from -phi'' + exp(phi) = n: with ion continuity the sum
 * int n u^2/2 + int [E^2/2 + phi e^phi - e^phi + 1] dx is constant in time (for the
 * linearised response 1 + phi the last bracket becomes E^2/2 + phi^2/2). */
void orc_moments(int64_t n, const int32_t* cell, const double* theta, const double* v, const double* w,
                 const double* E, const double* phi, int32_t ncell, double dx, double dt, double qm,
                 double kick, int32_t s_w, int32_t mode, int64_t* charge_fx, double* out)
{
    double mom = 0.0, kin = 0.0, vmax = 0.0, wsum = 0.0;
    int64_t q = 0;
    for (int64_t i = 0; i < n; ++i) {
        double vb = v[i] + (kick - 0.5) * qm * dt * orc_gather(E, ncell, cell[i], theta[i]);
        mom += w[i] * vb;
        kin += 0.5 * w[i] * vb * vb;
        wsum += w[i];
        if (fabs(vb) > vmax) vmax = fabs(vb);
        q += (int64_t)llrint(ldexp(w[i], s_w)) * ((int64_t)1 << 24);
    }
    double fe = 0.0, ee = 0.0;
    for (int32_t j = 0; j < ncell; ++j) {
        fe += 0.5 * E[j] * E[j];
        if (mode == 0)
            ee += phi[j] * exp(phi[j]) - exp(phi[j]) + 1.0;
        else
            ee += 0.5 * phi[j] * phi[j];
    }
    *charge_fx = q;
    out[0] = wsum * dx;          /* charge */
    out[1] = mom * dx;           /* momentum */
    out[2] = kin * dx;           /* ion kinetic energy */
    out[3] = fe * dx;            /* field energy */
    out[4] = ee * dx;            /* electron free energy */
    out[5] = out[2] + out[3] + out[4];
    out[6] = vmax;               /* max |Vbar| */
    out[7] = vmax * dt / dx;     /* particle CFL number */
}

/* Relative L2 distance of Section 4.1.1: sqrt( sum (a-b)^2 / sum (a^2 + b^2) ). */
double orc_rel_l2(int64_t n, const double* a, const double* b)
{
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        num += (a[i] - b[i]) * (a[i] - b[i]);
        den += a[i] * a[i] + b[i] * b[i];
    }
    return den > 0.0 ? sqrt(num / den) : 0.0;
}

/* ---------------------------------------------------------------- phase-space coarse variable */

void orc_ps_sample_fx(int64_t n, const int32_t* cell, const double* theta, const double* vbar, const double* w,
                      const double* E0, int32_t ncell, double dx, double tau, double qm, int32_t bin_shift,
                      double vmin, double dv, int32_t nv, int32_t s_w, int64_t* F)
{
    int32_t nxc = ncell >> bin_shift;
    memset(F, 0, sizeof(int64_t) * (size_t)nxc * (size_t)nv);
    for (int64_t p = 0; p < n; ++p) {
        double E0p = orc_gather(E0, ncell, cell[p], theta[p]);
        int32_t c = cell[p];
        double th = theta[p];
        drift(&c, &th, tau * vbar[p] / dx, ncell);   /* X~ = X + tau V         (Eq. explicitflow) */
        double vt = vbar[p] + qm * tau * E0p;         /* V~ = V + qm tau E_n(X) */
        double jf = floor((vt - vmin) / dv);          /* nearest-grid-point cell in v */
        int32_t j = jf < 0.0 ? 0 : (jf >= (double)nv ? nv - 1 : (int32_t)jf);
        int64_t wq = (int64_t)llrint(ldexp(w[p], s_w));
        int64_t tq = (int64_t)llrint(th * THETA_ONE);
        int64_t qr = wq * tq, ql = wq * ((int64_t)THETA_ONE - tq);
        int32_t b0 = c >> bin_shift, b1 = wrap((int64_t)c + 1, ncell) >> bin_shift;
        F[(size_t)b0 * nv + j] += ql;
        F[(size_t)b1 * nv + j] += qr;
    }
}

/* Edge reconstruction (Appendix C) of the entries below 0 of F[0..N]: with k0 the largest
 * index where F < 0, a ramp F[k] = (k - k_-) dF on [k_-, k_+) (zero below k_-) whose slope
 * keeps sum_{k < k_+} F[k] (the first moment of the histogram); the range grows (k_- down,
 * then k_+ up with k_- reset to k0 - 1) until 0 <= (k_+ - k_- - 1) dF <= F[k_+]. Returns 1 if
 * no admissible range exists (the caller then clamps). */
static int cdf_edge_low(int32_t N, double* F)
{
    int32_t k0 = -1;
    for (int32_t k = N; k >= 0; --k)
        if (F[k] < 0.0) {
            k0 = k;
            break;
        }
    if (k0 < 0) return 0;
    int32_t km = k0 - 1, kp = k0 + 1;
    for (;;) {
        if (kp > N || km < 0) return 1;
        double S = 0.0;
        for (int32_t k = 0; k < kp; ++k) S += F[k];
        double L = (double)(kp - km);
        double dF = 2.0 * S / (L * (L - 1.0));
        double top = (L - 1.0) * dF;
        if (top >= 0.0 && top <= F[kp]) {
            for (int32_t k = 0; k < km; ++k) F[k] = 0.0;
            for (int32_t k = km; k < kp; ++k) F[k] = (double)(k - km) * dF;
            return 0;
        }
        if (km > 0) {
            km -= 1;
        } else {
            kp += 1;
            km = k0 - 1;
        }
    }
}

/* Interior reconstruction (Appendix C) from the low indices: at the first descent k0, k1 the
 * first index after it with F[k1] >= F[k0], k_+ the (first) minimum on (k0, k1], k_- the last
 * index before k0 with F <= F[k_+]; a ramp F[k_-] + (k - k_-) dF on (k_-, k_+) whose slope keeps
 * sum_{k_- <= k < k_+} F[k]; k_+ grows until dF >= 0 and the ramp ends at or below F[k_+]. The
 * admissibility test reads the printed condition with the ramp's base F[k_-] added (the form
 * that makes the result monotone; the two agree when F[k_-] = 0). Repeated until monotone.
 * A descent with no admissible range (near F = 1 the ramp cannot keep the sum without ending
 * above 1) is filled by a running max instead, which moves only the few values of the
 * descent; 1 is returned then. */
static int cdf_interior_fwd(int32_t N, double* F)
{
    int bad = 0;
    int32_t start = 0;
    for (;;) {
        int32_t k0 = -1;
        for (int32_t k = start; k < N; ++k)
            if (F[k] > F[k + 1]) {
                k0 = k;
                break;
            }
        if (k0 < 0) return bad;
        int32_t k1 = k0 + 1;
        while (k1 < N && F[k1] < F[k0]) ++k1;
        int32_t kp = k0 + 1;
        for (int32_t k = k0 + 1; k <= k1; ++k)
            if (F[k] < F[kp]) kp = k;
        int32_t km = 0;
        for (int32_t k = k0 - 1; k >= 0; --k)
            if (F[k] <= F[kp]) {
                km = k;
                break;
            }
        int done = 0;
        for (; kp <= N; ++kp) {
            double S = 0.0;
            for (int32_t k = km; k < kp; ++k) S += F[k];
            double L = (double)(kp - km);
            double dF = 2.0 / (L - 1.0) * (S / L - F[km]);
            double end = F[km] + (L - 1.0) * dF;
            if (dF >= 0.0 && end <= F[kp]) {
                for (int32_t k = km + 1; k < kp; ++k) F[k] = F[km] + (double)(k - km) * dF;
                done = 1;
                break;
            }
        }
        if (!done) {
            bad = 1;
            for (int32_t k = k0 + 1; k <= N; ++k)
                if (F[k] < F[k - 1]) F[k] = F[k - 1];
        }
        start = km;
    }
}

static void cdf_mirror(int32_t N, const double* F, double* G)
{
    for (int32_t k = 0; k <= N; ++k) G[k] = 1.0 - F[N - k];
}

int orc_cdf_reconstruct(int32_t N, double* F)
{
    double* G = (double*)malloc(sizeof(double) * (size_t)(N + 1));
    double* P = (double*)malloc(sizeof(double) * (size_t)(N + 1));
    int bad = 0;
    F[0] = 0.0;
    F[N] = 1.0;
    /* entries below 0, then entries above 1 (the low-edge procedure on the mirrored array) */
    bad |= cdf_edge_low(N, F);
    cdf_mirror(N, F, G);
    bad |= cdf_edge_low(N, G);
    cdf_mirror(N, G, F);
    if (bad)
        for (int32_t k = 0; k <= N; ++k) F[k] = F[k] < 0.0 ? 0.0 : (F[k] > 1.0 ? 1.0 : F[k]);
    /* F+ from the low indices, F- from the high indices, averaged */
    memcpy(P, F, sizeof(double) * (size_t)(N + 1));
    bad |= cdf_interior_fwd(N, P);
    cdf_mirror(N, F, G);
    bad |= cdf_interior_fwd(N, G);
    cdf_mirror(N, G, F);
    for (int32_t k = 0; k <= N; ++k) F[k] = 0.5 * (P[k] + F[k]);
    free(G);
    free(P);
    return bad;
}

int orc_ps_lift_tables(int32_t nxc, int32_t nv, const double* H, double* mass, double* cdf)
{
    int bad = 0;
    double tot = 0.0, pos = 0.0;
    for (int32_t i = 0; i < nxc; ++i) {
        double s = 0.0;
        for (int32_t j = 0; j < nv; ++j) s += H[(size_t)i * nv + j];
        mass[i] = s;
        tot += s;
        pos += s > 0.0 ? s : 0.0;
    }
    double scale = pos > 0.0 ? tot / pos : 0.0; /* negative masses clamped, total kept */
    for (int32_t i = 0; i < nxc; ++i) {
        double* F = cdf + (size_t)i * (nv + 1);
        double m = mass[i];
        if (m > 0.0) {
            double s = 0.0;
            F[0] = 0.0;
            for (int32_t j = 0; j < nv; ++j) {
                s += H[(size_t)i * nv + j];
                F[j + 1] = s / m;
            }
            bad |= orc_cdf_reconstruct(nv, F);
        } else {
            for (int32_t j = 0; j <= nv; ++j) F[j] = (double)j / (double)nv;
        }
        mass[i] = m > 0.0 ? m * scale : 0.0;
    }
    return bad;
}

void orc_cdf_cell_slopes(int32_t nv, const double* F, double* sigma)
{
    for (int32_t k = 0; k < nv; ++k) {
        double p = F[k + 1] - F[k];
        double pl = k > 0 ? F[k] - F[k - 1] : 0.0;
        double pr = k + 1 < nv ? F[k + 2] - F[k + 1] : 0.0;
        double s = p > 0.0 ? (pr - pl) / (4.0 * p) : 0.0;
        sigma[k] = s > 1.0 ? 1.0 : (s < -1.0 ? -1.0 : s);
    }
}

double orc_cdf_inverse(int32_t nv, const double* F, const double* sigma, double b, double vmin, double dv)
{
    int32_t k = 0;
    while (k < nv - 1 && !(F[k + 1] > b)) ++k;  /* first k with F[k+1] > b */
    double den = F[k + 1] - F[k];
    double r = den > 0.0 ? (b - F[k]) / den : 0.5;
    if (r < 0.0) r = 0.0;
    if (r > 1.0) r = 1.0;
    /* inside the cell the density is 1 + sigma (2t - 1) (t in [0, 1]): the cell's CDF fraction is
     * t + sigma (t^2 - t), inverted in the form that stays exact as sigma -> 0 */
    double sg = sigma ? sigma[k] : 0.0;
    double den2 = (1.0 - sg) + sqrt((1.0 - sg) * (1.0 - sg) + 4.0 * sg * r);
    double t = den2 > 0.0 ? 2.0 * r / den2 : 0.0; /* den2 = 0 only for sigma = 1, r = 0 */
    return vmin + dv * ((double)k + t);
}

void orc_ps_quiet_start(int64_t N, int32_t ncell, int32_t bin_shift, const double* mass, const double* cdf,
                        int32_t nv, double vmin, double dv, uint64_t seed, int32_t* cell, double* theta,
                        double* v, double* w)
{
    int64_t ppc = N / ncell;
    uint32_t half = (uint32_t)(2147483648.0 / (double)N);
    uint32_t shift = (uint32_t)(orc_splitmix64(seed) >> 32);
    int m = 0;
    while (((int64_t)1 << m) < ppc) ++m;
    int pow2 = ((int64_t)1 << m) == ppc;
    double per_node = ldexp(1.0, -bin_shift); /* Haar synthesis: a bin's mass spread evenly over its nodes */
    int32_t nbins = ncell >> bin_shift;
    double* sig = (double*)malloc(sizeof(double) * (size_t)nbins * (size_t)nv);
    for (int32_t i = 0; i < nbins; ++i) orc_cdf_cell_slopes(nv, cdf + (size_t)i * (nv + 1), sig + (size_t)i * nv);
    for (int64_t s = 0; s < N; ++s) {
        int64_t i = s;
        if (pow2 && m > 0) {
            uint32_t k = (uint32_t)(s & (ppc - 1));
            uint32_t r = brev32(k) >> (32 - m);
            i = (s & ~(ppc - 1)) | (int64_t)r;
        }
        int32_t c = (int32_t)(i / ppc);
        double th = (2.0 * (double)(i % ppc) + 1.0) / (2.0 * (double)ppc);
        /* position measured from the centre of the particle's bin, in bin widths: the lifted
         * f(x, v) is linear in x between neighbouring bin centres (Section 3.3's linear
         * interpolation), mass and velocity quantiles alike. A bin sums the CIC charge of its
         * 2^b nodes, i.e. covers x/dx in [i 2^b - 1/2, (i+1) 2^b - 1/2). */
        int32_t nxc = ncell >> bin_shift;
        double t = th + 0.5;
        int32_t cc = c;
        if (t >= 1.0) {
            t -= 1.0;
            cc = wrap((int64_t)c + 1, ncell);
        }
        int32_t bin = cc >> bin_shift;
        double pos = ((double)(cc & ((1 << bin_shift) - 1)) + t) * per_node; /* in [0, 1) */
        int32_t b0, b1;
        double phi;
        if (pos >= 0.5) {
            b0 = bin;
            b1 = (bin + 1) % nxc;
            phi = pos - 0.5;
        } else {
            b0 = (bin + nxc - 1) % nxc;
            b1 = bin;
            phi = pos + 0.5;
        }
        double nX = ((1.0 - phi) * mass[b0] + phi * mass[b1]) * per_node;
        uint32_t B = brev32((uint32_t)i) + half + shift;
        double b = ((double)B + 0.5) * 2.3283064365386963e-10;
        double v0 = orc_cdf_inverse(nv, cdf + (size_t)b0 * (nv + 1), sig + (size_t)b0 * nv, b, vmin, dv);
        double v1 = orc_cdf_inverse(nv, cdf + (size_t)b1 * (nv + 1), sig + (size_t)b1 * nv, b, vmin, dv);
        cell[s] = c;
        theta[s] = th;
        w[s] = nX / (double)ppc;
        v[s] = (1.0 - phi) * v0 + phi * v1;
    }
    free(sig);
}

int orc_ps_burst(int64_t n, int32_t* cell, double* theta, double* v, const double* w, int32_t ncell, double dx,
                 double dt, double qm, int32_t K, double dT, int32_t mode, int32_t s_w, double tol, int32_t maxit,
                 int32_t vel_at_integer, int32_t bin_shift, double vmin, double dv, int32_t nv, double* phi,
                 int64_t* samples)
{
    double* E = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* E0 = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* vbar = (double*)malloc(sizeof(double) * (size_t)n);
    size_t row = (size_t)(ncell >> bin_shift) * (size_t)nv;
    int fails = field_from_particles(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    memcpy(E0, E, sizeof(double) * (size_t)ncell);
    double kick = vel_at_integer ? 0.5 : 1.0;
    for (int32_t p = 0; p <= K; ++p) {
        for (int64_t i = 0; i < n; ++i)
            vbar[i] = v[i] + (kick - 0.5) * qm * dt * orc_gather(E, ncell, cell[i], theta[i]);
        orc_ps_sample_fx(n, cell, theta, vbar, w, E0, ncell, dx, dT - p * dt, qm, bin_shift, vmin, dv, nv, s_w,
                         samples + (size_t)p * row);
        if (p == K) break;
        orc_push(n, cell, theta, v, E, ncell, dx, dt, qm, kick);
        kick = 1.0;
        fails += field_from_particles(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    }
    free(E);
    free(E0);
    free(vbar);
    return fails;
}

/* ---------------------------------------------------------------- kinetic electrons
 * Section 4.1: in the paper's ion-acoustic runs both species are particles in the PIC
 * bursts (q_e/m_e = -1800 against q_i/m_i = 1, a time step that resolves the electron
 * plasma period); the Boltzmann relation only serves the lifting. The field is then the
 * plain Poisson equation for the net charge n_i - n_e: an electron of weight w carries
 * charge -w dx, an ion +w dx. */

/* Periodic Poisson equation -(phi_{j+1} - 2 phi_j + phi_{j-1}) / dx^2 = r_j - <r> with
 * <phi> = 0, and the centred field E_j = -(phi_{j+1} - phi_{j-1}) / (2 dx). Solved through
 * the face fields F_{j+1/2} = -(phi_{j+1} - phi_j) / dx: consecutive faces differ by
 * dx (r_j - <r>) (the discrete Gauss law) and the faces sum to zero (phi is periodic);
 * E_j = (F_{j+1/2} + F_{j-1/2}) / 2. */
void orc_poisson_periodic(int32_t ncell, double dx, const double* r, double* phi, double* E)
{
    double* F = (double*)malloc(sizeof(double) * (size_t)ncell);
    double mean = 0.0;
    for (int32_t j = 0; j < ncell; ++j) mean += r[j];
    mean /= ncell;
    double acc = 0.0, fsum = 0.0;
    for (int32_t j = 0; j < ncell; ++j) { /* F_{j+1/2} - F_{-1/2} */
        acc += dx * (r[j] - mean);
        F[j] = acc;
        fsum += acc;
    }
    for (int32_t j = 0; j < ncell; ++j) F[j] -= fsum / ncell;
    double p = 0.0, psum = 0.0;
    for (int32_t j = 0; j < ncell; ++j) { /* phi_0 = 0, phi_{j+1} = phi_j - dx F_{j+1/2} */
        phi[j] = p;
        psum += p;
        p -= dx * F[j];
    }
    for (int32_t j = 0; j < ncell; ++j) phi[j] -= psum / ncell;
    for (int32_t j = 0; j < ncell; ++j) E[j] = 0.5 * (F[j] + F[wrap((int64_t)j - 1, ncell)]);
    free(F);
}

/* Field of a two-species state: fixed-point deposits of ions and electrons (the same rule
 * and shift s_w), net density (rho_i - rho_e) 2^-(s_w+24), periodic Poisson, centred E. */
static void field_kinetic(int64_t ni, const int32_t* ci, const double* ti, const double* wi, int64_t ne,
                          const int32_t* ce, const double* te, const double* we, int32_t ncell, double dx,
                          int32_t s_w, double* phi, double* E)
{
    int64_t* rho_i = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t* rho_e = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    double* r = (double*)malloc(sizeof(double) * (size_t)ncell);
    orc_deposit_fx(ni, ci, ti, wi, ncell, s_w, rho_i);
    orc_deposit_fx(ne, ce, te, we, ncell, s_w, rho_e);
    const double scale = ldexp(1.0, -(s_w + 24));
    for (int32_t j = 0; j < ncell; ++j) r[j] = (double)(rho_i[j] - rho_e[j]) * scale;
    orc_poisson_periodic(ncell, dx, r, phi, E);
    free(rho_i);
    free(rho_e);
    free(r);
}

void orc_field_kinetic(int64_t ni, const int32_t* ci, const double* ti, const double* wi, int64_t ne,
                       const int32_t* ce, const double* te, const double* we, int32_t ncell, double dx, int32_t s_w,
                       double* phi, double* E)
{
    field_kinetic(ni, ci, ti, wi, ne, ce, te, we, ncell, dx, s_w, phi, E);
}

/* Plain two-species PIC steps (Section 2.2 leapfrog for each species in the field of both).
 * vel_at_integer / e_vel_at_integer: the ions' / electrons' stored velocities are at integer
 * time (just loaded), so their first kick is a half kick. */
void orc_pic_steps_kinetic(int64_t ni, int32_t* ci, double* ti, double* vi, const double* wi, int64_t ne,
                           int32_t* ce, double* te, double* ve, const double* we, int32_t ncell, double dx, double dt,
                           double qm_i, double qm_e, int32_t nsteps, int32_t s_w, int32_t vel_at_integer,
                           int32_t e_vel_at_integer, double* phi)
{
    double* E = (double*)malloc(sizeof(double) * (size_t)ncell);
    double kick_i = vel_at_integer ? 0.5 : 1.0, kick_e = e_vel_at_integer ? 0.5 : 1.0;
    for (int32_t s = 0; s < nsteps; ++s) {
        field_kinetic(ni, ci, ti, wi, ne, ce, te, we, ncell, dx, s_w, phi, E);
        orc_push(ni, ci, ti, vi, E, ncell, dx, dt, qm_i, kick_i);
        orc_push(ne, ce, te, ve, E, ncell, dx, dt, qm_e, kick_e);
        kick_i = kick_e = 1.0;
    }
    free(E);
}

/* Burst of K two-species steps with the co-moving restriction of the ions (Appendix B), as
 * orc_burst / orc_ps_burst: nv = 0 records the ion density and momentum samples (double,
 * [K+1][2][ncell]) in samples; nv > 0 the fixed-point phase-space samples ([K+1][nxc][nv])
 * in samples_fx. */
void orc_burst_kinetic(int64_t ni, int32_t* ci, double* ti, double* vi, const double* wi, int64_t ne,
                       int32_t* ce, double* te, double* ve, const double* we, int32_t ncell, double dx, double dt,
                       double qm_i, double qm_e, int32_t K, double dT, int32_t s_w, int32_t vel_at_integer,
                       int32_t bin_shift, double vmin, double dv, int32_t nv, double* phi, double* samples,
                       int64_t* samples_fx)
{
    double* E = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* E0 = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* vbar = (double*)malloc(sizeof(double) * (size_t)ni);
    const size_t row = nv > 0 ? (size_t)(ncell >> bin_shift) * (size_t)nv : 2 * (size_t)ncell;
    field_kinetic(ni, ci, ti, wi, ne, ce, te, we, ncell, dx, s_w, phi, E);
    memcpy(E0, E, sizeof(double) * (size_t)ncell); /* E_n, stored at burst start */
    double kick = vel_at_integer ? 0.5 : 1.0;
    for (int32_t p = 0; p <= K; ++p) {
        for (int64_t i = 0; i < ni; ++i)
            vbar[i] = vi[i] + (kick - 0.5) * qm_i * dt * orc_gather(E, ncell, ci[i], ti[i]);
        const double tau = dT - p * dt;
        if (nv > 0) {
            orc_ps_sample_fx(ni, ci, ti, vbar, wi, E0, ncell, dx, tau, qm_i, bin_shift, vmin, dv, nv, s_w,
                             samples_fx + (size_t)p * row);
        } else {
            double* dens = samples + (size_t)p * row;
            orc_restrict_sample(ni, ci, ti, vbar, wi, E0, ncell, dx, tau, qm_i, dens, dens + ncell);
        }
        if (p == K) break;
        orc_push(ni, ci, ti, vi, E, ncell, dx, dt, qm_i, kick);
        orc_push(ne, ce, te, ve, E, ncell, dx, dt, qm_e, kick);
        kick = 1.0;
        field_kinetic(ni, ci, ti, wi, ne, ce, te, we, ncell, dx, s_w, phi, E);
    }
    free(E);
    free(E0);
    free(vbar);
}

/* Electrons of the lifting (Section 3.3, Eq. electronpassive: n_e = n_0 exp(phi), V_e = V_i,
 * T_e = T_e0): density exp(phi) of the Poisson-Boltzmann potential of the ion density, mean
 * velocity u[ncell] the ions' (NULL: none), Maxwellian of thermal speed v_th_e, quiet start on
 * that profile. */
void orc_boltzmann_electrons(int64_t N, int32_t ncell, const double* phi, const double* u, double v_th_e,
                             uint64_t seed, int32_t* cell, double* theta, double* v, double* w)
{
    double* n = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* u0 = (double*)calloc((size_t)ncell, sizeof(double));
    for (int32_t j = 0; j < ncell; ++j) n[j] = exp(phi[j]);
    orc_quiet_start(N, ncell, n, u ? u : u0, v_th_e, seed, cell, theta, v, w);
    free(n);
    free(u0);
}

/* ---------------------------------------------------------------- bounded domain
 * Walls at node 0 (x = 0) and node ncell-1 (x = (ncell-1) dx); the particles live in the
 * ncell-1 cells between them. Section 4.2 runs the slab expansion with an absorbing
 * boundary; the potential satisfies phi' = 0 at both walls (mirror ghosts phi_{-1} = phi_1,
 * phi_{ncell} = phi_{ncell-2}). A wall node's CIC control volume is the half cell inside the
 * domain, so its density is twice its deposit. */

/* Tridiagonal solve a_j x_{j-1} + b_j x_j + c_j x_{j+1} = d_j (Thomas; a_0 and c_{n-1} unused). */
static void thomas_var(int32_t n, const double* a, const double* b, const double* c, const double* d, double* x)
{
    double* cp = (double*)malloc(sizeof(double) * (size_t)n);
    double* dp = (double*)malloc(sizeof(double) * (size_t)n);
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (int32_t i = 1; i < n; ++i) {
        double m = b[i] - a[i] * cp[i - 1];
        cp[i] = c[i] / m;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int32_t i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp);
    free(dp);
}

int orc_newton_pb_walls(int32_t ncell, double dx, int32_t mode, const double* dep, double* phi, double tol,
                        int32_t maxit, int32_t* iters)
{
    const double inv_dx2 = 1.0 / (dx * dx);
    double* a = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* b = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* c = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* rhs = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* delta = (double*)malloc(sizeof(double) * (size_t)ncell);
    int status = 1;
    int32_t it = 0;
    for (it = 0; it < maxit; ++it) {
        for (int32_t j = 0; j < ncell; ++j) {
            /* mirror ghosts at the walls */
            double pl = (j == 0) ? phi[1] : phi[j - 1];
            double pr = (j == ncell - 1) ? phi[ncell - 2] : phi[j + 1];
            double nj = (j == 0 || j == ncell - 1) ? 2.0 * dep[j] : dep[j];
            double lap = (pl - 2.0 * phi[j] + pr) * inv_dx2;
            double g = (mode == 0) ? exp(phi[j]) : 1.0 + phi[j];
            double gp = (mode == 0) ? exp(phi[j]) : 1.0;
            rhs[j] = -(-lap + g - nj);
            b[j] = 2.0 * inv_dx2 + gp;
            a[j] = (j == ncell - 1) ? -2.0 * inv_dx2 : -inv_dx2; /* d lap / d phi_{j-1} */
            c[j] = (j == 0) ? -2.0 * inv_dx2 : -inv_dx2;         /* d lap / d phi_{j+1} */
        }
        thomas_var(ncell, a, b, c, rhs, delta);
        double m = 0.0;
        for (int32_t j = 0; j < ncell; ++j) m = fmax(m, fabs(delta[j]));
        double scale = (m > 2.0) ? 2.0 / m : 1.0;
        for (int32_t j = 0; j < ncell; ++j) phi[j] += scale * delta[j];
        if (m < tol) {
            status = 0;
            ++it;
            break;
        }
    }
    if (iters) *iters = it;
    free(a);
    free(b);
    free(c);
    free(rhs);
    free(delta);
    return status;
}

void orc_efield_walls(int32_t ncell, double dx, const double* phi, double* E)
{
    E[0] = 0.0; /* -(phi_1 - phi_{-1}) / (2 dx) with the mirror ghost */
    E[ncell - 1] = 0.0;
    for (int32_t j = 1; j < ncell - 1; ++j) E[j] = -(phi[j + 1] - phi[j - 1]) / (2.0 * dx);
}

/* Leapfrog kick-drift in the bounded domain: a particle whose drift ends outside
 * [0, (ncell-1) dx) is absorbed: w = 0, v = 0, parked on the wall node it crossed
 * (cell 0 or ncell-1, theta 0). Particles with w = 0 are not moved. */
void orc_push_walls(int64_t n, int32_t* cell, double* theta, double* v, double* w, const double* E,
                    int32_t ncell, double dx, double dt, double qm, double kick)
{
    for (int64_t p = 0; p < n; ++p) {
        if (w[p] == 0.0) continue;
        double Ep = (1.0 - theta[p]) * E[cell[p]] + theta[p] * E[cell[p] + 1];
        v[p] += kick * qm * dt * Ep;
        double s = theta[p] + v[p] * dt / dx;
        double k = floor(s);
        double cn = (double)cell[p] + k;
        if (!(cn >= 0.0 && cn < (double)(ncell - 1))) {
            cell[p] = (cn < 0.0) ? 0 : ncell - 1;
            theta[p] = 0.0;
            v[p] = 0.0;
            w[p] = 0.0;
            continue;
        }
        cell[p] = (int32_t)cn;
        theta[p] = s - k;
    }
}

/* Appendix B restriction sample in the bounded domain: as orc_restrict_sample; a
 * particle whose co-moving position X~ lies outside [0, (ncell-1) dx) has left the
 * domain by t_{n+1} and is not counted. Particles with w = 0 contribute nothing. */
void orc_restrict_sample_walls(int64_t n, const int32_t* cell, const double* theta, const double* vbar,
                               const double* w, const double* E0, int32_t ncell, double dx, double tau,
                               double qm, double* dens, double* mom)
{
    memset(dens, 0, sizeof(double) * (size_t)ncell);
    memset(mom, 0, sizeof(double) * (size_t)ncell);
    for (int64_t p = 0; p < n; ++p) {
        if (w[p] == 0.0) continue;
        double E0p = (1.0 - theta[p]) * E0[cell[p]] + theta[p] * E0[cell[p] + 1];
        double s = theta[p] + tau * vbar[p] / dx;
        double k = floor(s);
        double cn = (double)cell[p] + k;
        if (!(cn >= 0.0 && cn < (double)(ncell - 1))) continue;
        int32_t c = (int32_t)cn;
        double th = s - k;
        double vt = vbar[p] + qm * tau * E0p;
        dens[c] += w[p] * (1.0 - th);
        dens[c + 1] += w[p] * th;
        mom[c] += w[p] * vt * (1.0 - th);
        mom[c + 1] += w[p] * vt * th;
    }
}

/* Appendix C loading with equal weights in the bounded domain: the nodal density profile
 * n_j (wall nodes included as densities) is linear inside each of the ncell-1 cells, with
 * cell mass m_c = (n_c + n_{c+1}) / 2 and cumulative mass C_c = m_0 + ... + m_{c-1}, total M.
 * Particle i sits at the quantile s_i = (i + 1/2) M / N of the cumulative mass: in the cell c
 * with C_c <= s_i < C_{c+1} and m_c > 0, at the offset t that solves
 * t + sigma (t^2 - t) = r, r = (s_i - C_c) / m_c, sigma = (n_{c+1} - n_c) / (n_{c+1} + n_c)
 * (the mass of the linear density up to t). Every particle has w = M / N, so the number of
 * particles per cell follows the mass (empty cells get none). V = u(X) + v_th Phi^{-1}(b_i)
 * with the Hammersley second coordinate b_i of orc_quiet_start. Storage: within each aligned
 * block of 4096 slots (all but a ragged tail), slot s holds point i = s with its low 12 bits
 * reversed, i.e. the block's points in ascending velocity quantile (their positions are
 * within 4096 mass quantiles of each other); tail slots hold i = s. */
void orc_quiet_start_equal(int64_t N, int32_t ncell, const double* nprof, const double* uprof, double v_th,
                           uint64_t seed, int32_t* cell, double* theta, double* v, double* w)
{
    const int32_t ncl = ncell - 1;
    double* C = (double*)malloc(sizeof(double) * (size_t)(ncl + 1));
    C[0] = 0.0;
    for (int32_t c = 0; c < ncl; ++c) C[c + 1] = C[c] + 0.5 * (nprof[c] + nprof[c + 1]);
    const double M = C[ncl];
    uint32_t half = (uint32_t)(2147483648.0 / (double)N);
    uint32_t shift = (uint32_t)(orc_splitmix64(seed) >> 32);
    int32_t c = 0;
    for (int64_t i = 0; i < N; ++i) {
        double s = ((double)i + 0.5) * M / (double)N;
        while (c < ncl - 1 && !(s < C[c + 1] && C[c + 1] > C[c])) ++c;
        double mc = C[c + 1] - C[c];
        double r = (mc > 0.0) ? (s - C[c]) / mc : 0.5;
        if (r < 0.0) r = 0.0;
        if (r > 1.0) r = 1.0;
        double n0 = nprof[c], n1 = nprof[c + 1];
        double sig = (n0 + n1 > 0.0) ? (n1 - n0) / (n1 + n0) : 0.0;
        double den = (1.0 - sig) + sqrt((1.0 - sig) * (1.0 - sig) + 4.0 * sig * r);
        double t = (den > 0.0) ? 2.0 * r / den : 0.0;
        if (t >= 1.0) t = nextafter(1.0, 0.0); /* stay inside the cell */
        const int32_t cc = c;
        double uX = (1.0 - t) * uprof[cc] + t * uprof[cc + 1];
        uint32_t B = brev32((uint32_t)i) + half + shift;
        double b = ((double)B + 0.5) * 2.3283064365386963e-10;
        int64_t slot = i; /* bit reversal inside full blocks of 4096 is its own inverse */
        if ((i | 4095) < N) slot = (i & ~(int64_t)4095) | (int64_t)(brev32((uint32_t)(i & 4095)) >> 20);
        cell[slot] = cc;
        theta[slot] = t;
        w[slot] = M / (double)N;
        v[slot] = uX + v_th * orc_ndtri(b);
    }
    free(C);
}

static int field_walls(int64_t n, const int32_t* cell, const double* theta, const double* w, int32_t ncell,
                       double dx, int32_t mode, int32_t s_w, double tol, int32_t maxit, double* phi, double* E)
{
    int64_t* rho = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    double* dens = (double*)malloc(sizeof(double) * (size_t)ncell);
    orc_deposit_fx(n, cell, theta, w, ncell, s_w, rho);
    double scale = ldexp(1.0, -(s_w + 24));
    for (int32_t j = 0; j < ncell; ++j) dens[j] = (double)rho[j] * scale;
    int32_t iters = 0;
    int fail = orc_newton_pb_walls(ncell, dx, mode, dens, phi, tol, maxit, &iters);
    orc_efield_walls(ncell, dx, phi, E);
    free(rho);
    free(dens);
    return fail;
}

int orc_burst_walls(int64_t n, int32_t* cell, double* theta, double* v, double* w, int32_t ncell, double dx,
                    double dt, double qm, int32_t K, double dT, int32_t comoving, int32_t mode, int32_t s_w,
                    double tol, int32_t maxit, int32_t vel_at_integer, double* phi, double* samples)
{
    double* E = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* E0 = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* vbar = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int fails = field_walls(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    memcpy(E0, E, sizeof(double) * (size_t)ncell);
    double kick = vel_at_integer ? 0.5 : 1.0;
    for (int32_t p = 0; p <= K; ++p) {
        for (int64_t i = 0; i < n; ++i)
            vbar[i] = (w[i] == 0.0) ? v[i]
                                    : v[i] + (kick - 0.5) * qm * dt *
                                                 ((1.0 - theta[i]) * E[cell[i]] + theta[i] * E[cell[i] + 1]);
        double tau = comoving ? dT - p * dt : 0.0;
        double* dens = samples + (size_t)p * 2 * ncell;
        orc_restrict_sample_walls(n, cell, theta, vbar, w, E0, ncell, dx, tau, qm, dens, dens + ncell);
        if (p == K) break;
        orc_push_walls(n, cell, theta, v, w, E, ncell, dx, dt, qm, kick);
        kick = 1.0;
        fails += field_walls(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    }
    free(E);
    free(E0);
    free(vbar);
    return fails;
}

int orc_pic_steps_walls(int64_t n, int32_t* cell, double* theta, double* v, double* w, int32_t ncell, double dx,
                        double dt, double qm, int32_t nsteps, int32_t mode, int32_t s_w, double tol, int32_t maxit,
                        int32_t vel_at_integer, double* phi)
{
    double* E = (double*)malloc(sizeof(double) * (size_t)ncell);
    int fails = 0;
    double kick = vel_at_integer ? 0.5 : 1.0;
    for (int32_t s = 0; s < nsteps; ++s) {
        fails += field_walls(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
        orc_push_walls(n, cell, theta, v, w, E, ncell, dx, dt, qm, kick);
        kick = 1.0;
    }
    free(E);
    return fails;
}

/* ---------------------------------------------------------------- phase space, bounded grid */

/* orc_ps_sample_fx on the bounded grid: ions of weight 0 carry nothing, and an ion whose
 * co-moving target X~ lies outside [0, (ncell-1) dx) has left the domain by t_{n+1} and is
 * not counted (as orc_restrict_sample_walls). */
void orc_ps_sample_fx_walls(int64_t n, const int32_t* cell, const double* theta, const double* vbar,
                            const double* w, const double* E0, int32_t ncell, double dx, double tau, double qm,
                            int32_t bin_shift, double vmin, double dv, int32_t nv, int32_t s_w, int64_t* F)
{
    int32_t nxc = ncell >> bin_shift;
    memset(F, 0, sizeof(int64_t) * (size_t)nxc * (size_t)nv);
    for (int64_t p = 0; p < n; ++p) {
        if (w[p] == 0.0) continue;
        double E0p = (1.0 - theta[p]) * E0[cell[p]] + theta[p] * E0[cell[p] + 1];
        double s = theta[p] + tau * vbar[p] / dx;
        double k = floor(s);
        double cn = (double)cell[p] + k;
        if (!(cn >= 0.0 && cn < (double)(ncell - 1))) continue;
        int32_t c = (int32_t)cn;
        double th = s - k;
        double vt = vbar[p] + qm * tau * E0p;
        double jf = floor((vt - vmin) / dv);
        int32_t j = jf < 0.0 ? 0 : (jf >= (double)nv ? nv - 1 : (int32_t)jf);
        int64_t wq = (int64_t)llrint(ldexp(w[p], s_w));
        int64_t tq = (int64_t)llrint(th * THETA_ONE);
        int64_t qr = wq * tq, ql = wq * ((int64_t)THETA_ONE - tq);
        F[(size_t)(c >> bin_shift) * nv + j] += ql;
        F[(size_t)((c + 1) >> bin_shift) * nv + j] += qr;
    }
}

/* Appendix C loading of the phase-space tables on the bounded grid, with equal weights.
 * Bin i sums the CIC charge of its 2^b nodes, i.e. spans x/dx in [i 2^b - 1/2, (i+1) 2^b - 1/2)
 * cut to the domain [0, ncell-1]: the first and last bins span 2^b - 1/2 node widths. The lifted
 * density in x is linear between the bins' span midpoints, with value mass_i / width_i there,
 * and constant beyond the first and last midpoints (no wrap): its values at the nodes, n_j, are
 * the profile that orc_quiet_start_equal loads (positions by mass quantile, storage order in
 * velocity-ordered blocks); every ion then gets w = (sum of the bin masses) / N, so lifting keeps
 * the charge, and V = (1 - f) G_b0(b_i) + f G_b1(b_i) blended between the inverse CDFs of the two
 * bins whose midpoints bracket its position, b_i its Hammersley quantile, with f b1's share of
 * the density there, phi d_b1 / ((1 - phi) d_b0 + phi d_b1) (phi the fraction of the way from
 * b0's midpoint): a bin without ions lends no velocities. (Blending by phi alone, as the
 * periodic loader does, gave the ions just outside the expansion front velocities drawn halfway
 * from an empty bin's placeholder table.) */
static double ps_mid(int32_t i, int32_t nxc, double width, int32_t ncell)
{
    if (i == 0) return 0.5 * (width - 0.5);
    if (i == nxc - 1) return 0.5 * ((nxc - 1) * width - 0.5 + (double)(ncell - 1));
    return (i + 0.5) * width - 0.5;
}

/* The bins b0 <= b1 whose midpoints bracket x (nodes), and the fraction phi of the way. */
static void ps_bins_at(double x, int32_t nxc, double width, int32_t ncell, int32_t* b0, int32_t* b1, double* phi)
{
    if (nxc < 2 || x <= ps_mid(0, nxc, width, ncell)) {
        *b0 = *b1 = 0;
        *phi = 0.0;
        return;
    }
    if (x >= ps_mid(nxc - 1, nxc, width, ncell)) {
        *b0 = *b1 = nxc - 1;
        *phi = 0.0;
        return;
    }
    int32_t i = (int32_t)floor((x + 0.5) / width - 0.5);
    if (i < 0) i = 0;
    if (i > nxc - 2) i = nxc - 2;
    while (i > 0 && x < ps_mid(i, nxc, width, ncell)) --i;
    while (i < nxc - 2 && x >= ps_mid(i + 1, nxc, width, ncell)) ++i;
    const double m0 = ps_mid(i, nxc, width, ncell), m1 = ps_mid(i + 1, nxc, width, ncell);
    *b0 = i;
    *b1 = i + 1;
    *phi = (x - m0) / (m1 - m0);
}

void orc_ps_quiet_start_equal(int64_t N, int32_t ncell, int32_t bin_shift, const double* mass, const double* cdf,
                              int32_t nv, double vmin, double dv, uint64_t seed, int32_t* cell, double* theta,
                              double* v, double* w)
{
    const int32_t nxc = ncell >> bin_shift;
    const double width = ldexp(1.0, bin_shift);
    double* prof = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* zero = (double*)calloc((size_t)ncell, sizeof(double));
    double* dens = (double*)malloc(sizeof(double) * (size_t)nxc);
    double* sig = (double*)malloc(sizeof(double) * (size_t)nxc * (size_t)nv);
    for (int32_t i = 0; i < nxc; ++i) orc_cdf_cell_slopes(nv, cdf + (size_t)i * (nv + 1), sig + (size_t)i * nv);
    double total = 0.0;
    for (int32_t i = 0; i < nxc; ++i) {
        total += mass[i];
        const double wi = (i == 0 || i == nxc - 1) ? width - 0.5 : width;
        dens[i] = mass[i] / wi;
    }
    for (int32_t j = 0; j < ncell; ++j) {
        int32_t b0, b1;
        double phi;
        ps_bins_at((double)j, nxc, width, ncell, &b0, &b1, &phi);
        prof[j] = (1.0 - phi) * dens[b0] + phi * dens[b1];
    }
    orc_quiet_start_equal(N, ncell, prof, zero, 0.0, seed, cell, theta, v, w);
    uint32_t half = (uint32_t)(2147483648.0 / (double)N);
    uint32_t shift = (uint32_t)(orc_splitmix64(seed) >> 32);
    for (int64_t s = 0; s < N; ++s) {
        int64_t i = s; /* point held by slot s (the loader's block order) */
        if ((s | 4095) < N) i = (s & ~(int64_t)4095) | (int64_t)(brev32((uint32_t)(s & 4095)) >> 20);
        int32_t b0, b1;
        double phi;
        ps_bins_at((double)cell[s] + theta[s], nxc, width, ncell, &b0, &b1, &phi);
        if ((1.0 - phi) * dens[b0] + phi * dens[b1] <= 0.0) {
            /* the cell's linear profile reaches past the midpoint interpolation's zero (next to
             * an empty bin): take the velocities at the cell's denser node */
            const int32_t c = cell[s];
            ps_bins_at(prof[c + 1] > prof[c] ? (double)(c + 1) : (double)c, nxc, width, ncell, &b0, &b1, &phi);
        }
        uint32_t B = brev32((uint32_t)i) + half + shift;
        double b = ((double)B + 0.5) * 2.3283064365386963e-10;
        double v0 = orc_cdf_inverse(nv, cdf + (size_t)b0 * (nv + 1), sig + (size_t)b0 * nv, b, vmin, dv);
        double v1 = orc_cdf_inverse(nv, cdf + (size_t)b1 * (nv + 1), sig + (size_t)b1 * nv, b, vmin, dv);
        /* quantiles blended by each bin's share of the density at x: a bin without ions (whose
         * table is a placeholder) contributes nothing */
        double r0 = (1.0 - phi) * dens[b0], r1 = phi * dens[b1];
        double f = (r0 + r1 > 0.0) ? r1 / (r0 + r1) : phi;
        v[s] = (1.0 - f) * v0 + f * v1;
        w[s] = total / (double)N;
    }
    free(prof);
    free(zero);
    free(dens);
    free(sig);
}

int orc_ps_burst_walls(int64_t n, int32_t* cell, double* theta, double* v, double* w, int32_t ncell, double dx,
                       double dt, double qm, int32_t K, double dT, int32_t mode, int32_t s_w, double tol,
                       int32_t maxit, int32_t vel_at_integer, int32_t bin_shift, double vmin, double dv, int32_t nv,
                       double* phi, int64_t* samples)
{
    double* E = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* E0 = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* vbar = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    size_t row = (size_t)(ncell >> bin_shift) * (size_t)nv;
    int fails = field_walls(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    memcpy(E0, E, sizeof(double) * (size_t)ncell);
    double kick = vel_at_integer ? 0.5 : 1.0;
    for (int32_t p = 0; p <= K; ++p) {
        for (int64_t i = 0; i < n; ++i)
            vbar[i] = (w[i] == 0.0) ? v[i]
                                    : v[i] + (kick - 0.5) * qm * dt *
                                                 ((1.0 - theta[i]) * E[cell[i]] + theta[i] * E[cell[i] + 1]);
        orc_ps_sample_fx_walls(n, cell, theta, vbar, w, E0, ncell, dx, dT - p * dt, qm, bin_shift, vmin, dv, nv,
                               s_w, samples + (size_t)p * row);
        if (p == K) break;
        orc_push_walls(n, cell, theta, v, w, E, ncell, dx, dt, qm, kick);
        kick = 1.0;
        fails += field_walls(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    }
    free(E);
    free(E0);
    free(vbar);
    return fails;
}

/* ---------------------------------------------------------------- phase space, wavelet form
 * Section 3.3 ("A wavelet-based equation-free scheme") as the paper states it: the active
 * variables are the coarse scaling coefficients of the phase-space histogram of Eq.
 * (waveletapproximation). Restriction: the fine histogram, hat (CIC) weights on the n_xf fine
 * nodes in x and nearest grid point on n_vf velocity cells, sampled at the co-moving targets
 * of Appendix B (Eq. explicitflow and the deposit that follows it); then the 1-2-1 rule of
 * Eq. (restriction) in x down to the coarse nodes and the periodized DWT in v down to n_vc
 * coefficients (both in the Python layer). Lifting: synthesis in v, linear interpolation in x
 * (Eq. interpolation), the CDF reconstruction of Appendix C per coarse node (the Remark there
 * allows it before the lift in space), and the loading below. FP64 throughout; velocities
 * outside [vmin, vmin + n_vf dv) are counted in the first or last cell. */
void orc_ps_hist_fine(int64_t n, const int32_t* cell, const double* theta, const double* vbar, const double* w,
                      const double* E0, int32_t ncell, double dx, double tau, double qm, double vmin, double dv,
                      int32_t nvf, double* H)
{
    memset(H, 0, sizeof(double) * (size_t)ncell * (size_t)nvf);
    for (int64_t p = 0; p < n; ++p) {
        double E0p = orc_gather(E0, ncell, cell[p], theta[p]);
        int32_t kx = cell[p];
        double th = theta[p];
        drift(&kx, &th, tau * vbar[p] / dx, ncell);   /* X~ = X + tau V   (Eq. explicitflow) */
        double vt = vbar[p] + qm * tau * E0p;         /* V~ = V + qm tau E_n(X)          */
        double kf = floor((vt - vmin) / dv);          /* k_v = floor((V~ - V_min) / dv)   */
        int32_t kv = kf < 0.0 ? 0 : (kf >= (double)nvf ? nvf - 1 : (int32_t)kf);
        H[(size_t)kx * nvf + kv] += (1.0 - th) * w[p];
        H[(size_t)wrap((int64_t)kx + 1, ncell) * nvf + kv] += th * w[p];
    }
}

/* K fine steps in place with the fine co-moving histogram of each of the K + 1 states
 * (samples: [K+1][ncell][nvf]); the fine steps are orc_ps_burst's. */
int orc_ps_burst_fine(int64_t n, int32_t* cell, double* theta, double* v, const double* w, int32_t ncell, double dx,
                      double dt, double qm, int32_t K, double dT, int32_t mode, int32_t s_w, double tol, int32_t maxit,
                      int32_t vel_at_integer, double vmin, double dv, int32_t nvf, double* phi, double* samples)
{
    double* E = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* E0 = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* vbar = (double*)malloc(sizeof(double) * (size_t)n);
    size_t row = (size_t)ncell * (size_t)nvf;
    int fails = field_from_particles(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    memcpy(E0, E, sizeof(double) * (size_t)ncell);
    double kick = vel_at_integer ? 0.5 : 1.0;
    for (int32_t p = 0; p <= K; ++p) {
        for (int64_t i = 0; i < n; ++i)
            vbar[i] = v[i] + (kick - 0.5) * qm * dt * orc_gather(E, ncell, cell[i], theta[i]);
        orc_ps_hist_fine(n, cell, theta, vbar, w, E0, ncell, dx, dT - p * dt, qm, vmin, dv, nvf,
                         samples + (size_t)p * row);
        if (p == K) break;
        orc_push(n, cell, theta, v, E, ncell, dx, dt, qm, kick);
        kick = 1.0;
        fails += field_from_particles(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    }
    free(E);
    free(E0);
    free(vbar);
    return fails;
}

/* Inverse of the CDF G[0..nv] of fine node j at b (Appendix C: lookup, then linear
 * interpolation inside the cell, i.e. a uniform density there). G is the CDF of the fine
 * node's histogram: the linear interpolation in x (Eq. interpolation) of the reconstructed
 * histograms of its two coarse nodes i0, i1 with weights (1 - phi) and phi, i.e. the mixture
 * of their CDFs weighted by (1 - phi) mass[i0] and phi mass[i1]. */
static double ps_node_inverse(int32_t nv, const double* F0, const double* F1, double a0, double a1, double b,
                              double vmin, double dv)
{
    double tot = a0 + a1;
    int32_t k = 0;
    for (; k < nv - 1; ++k) {
        double g = (a0 * F0[k + 1] + a1 * F1[k + 1]) / tot;
        if (g > b) break;
    }
    double g0 = (a0 * F0[k] + a1 * F1[k]) / tot;
    double g1 = (a0 * F0[k + 1] + a1 * F1[k + 1]) / tot;
    double r = g1 > g0 ? (b - g0) / (g1 - g0) : 0.5;
    if (r < 0.0) r = 0.0;
    if (r > 1.0) r = 1.0;
    return vmin + dv * ((double)k + r);
}

/* Appendix C loading on the coarse-node tables of the wavelet form: mass[nxc] (the node
 * values after the clamp of negative ones, orc_ps_lift_tables: Eq. (restriction) averages, so
 * a coarse node holds mass per fine node) and the reconstructed CDFs cdf[nxc][nvf + 1].
 * Coarse node i sits at fine node i 2^b. Fine node j has phi_j = (j mod 2^b) / 2^b of the way
 * from coarse node i0 = j >> b to i1 = i0 + 1 (periodic), density n_j = (1 - phi_j) mass[i0]
 * + phi_j mass[i1] (the repeated Eq. (interpolation) of the coarse values) and the mixture CDF
 * of ps_node_inverse. Slot s takes
 * the Hammersley point, cell and offset of orc_quiet_start; its weight is n(X) / ppc and its
 * velocity the inverse CDF at b_s, both linear in x between the fine nodes c and c + 1. */
void orc_ps_quiet_start_nodes(int64_t N, int32_t ncell, int32_t bin_shift, const double* mass, const double* cdf,
                              int32_t nvf, double vmin, double dv, uint64_t seed, int32_t* cell, double* theta,
                              double* v, double* w)
{
    int64_t ppc = N / ncell;
    uint32_t half = (uint32_t)(2147483648.0 / (double)N);
    uint32_t shift = (uint32_t)(orc_splitmix64(seed) >> 32);
    int m = 0;
    while (((int64_t)1 << m) < ppc) ++m;
    int pow2 = ((int64_t)1 << m) == ppc;
    int32_t nxc = ncell >> bin_shift;
    double per_node = ldexp(1.0, -bin_shift);
    for (int64_t s = 0; s < N; ++s) {
        int64_t i = s;
        if (pow2 && m > 0) {
            uint32_t k = (uint32_t)(s & (ppc - 1));
            uint32_t r = brev32(k) >> (32 - m);
            i = (s & ~(ppc - 1)) | (int64_t)r;
        }
        int32_t c = (int32_t)(i / ppc);
        double th = (2.0 * (double)(i % ppc) + 1.0) / (2.0 * (double)ppc);
        uint32_t B = brev32((uint32_t)i) + half + shift;
        double b = ((double)B + 0.5) * 2.3283064365386963e-10;
        double vn[2], nn[2];
        for (int e = 0; e < 2; ++e) {
            int32_t j = wrap((int64_t)c + e, ncell);
            int32_t i0 = j >> bin_shift, i1 = (i0 + 1) % nxc;
            double phi = (double)(j & ((1 << bin_shift) - 1)) * per_node;
            double a0 = (1.0 - phi) * mass[i0], a1 = phi * mass[i1];
            nn[e] = a0 + a1;
            vn[e] = (a0 + a1 > 0.0)
                        ? ps_node_inverse(nvf, cdf + (size_t)i0 * (nvf + 1), cdf + (size_t)i1 * (nvf + 1), a0, a1, b,
                                          vmin, dv)
                        : vmin + dv * (double)nvf * b;
        }
        cell[s] = c;
        theta[s] = th;
        w[s] = ((1.0 - th) * nn[0] + th * nn[1]) / (double)ppc;
        v[s] = (1.0 - th) * vn[0] + th * vn[1];
    }
}

/* ---------------------------------------------------------------- ion pressure (Section 3.2)
 * EFREE's third ion variable: besides n and nV the ions' second velocity moment is active,
 * S_j = sum_p w_p V~_p^2 S_j(X~_p), restricted along the same approximate characteristics
 * (Appendix B) and with the same CIC weights as the density and the momentum. At the lift the
 * pressure is P = S - (nV)^2 / n and the temperature (velocity variance) T = P / n. */

void orc_restrict_second_moment(int64_t n, const int32_t* cell, const double* theta, const double* vbar,
                                const double* w, const double* E0, int32_t ncell, double dx, double tau,
                                double qm, double* sec)
{
    memset(sec, 0, sizeof(double) * (size_t)ncell);
    for (int64_t p = 0; p < n; ++p) {
        double E0p = orc_gather(E0, ncell, cell[p], theta[p]);
        int32_t c = cell[p];
        double th = theta[p];
        drift(&c, &th, tau * vbar[p] / dx, ncell);      /* X~ = X + tau V  */
        double vt = vbar[p] + qm * tau * E0p;            /* V~ = V + qm tau E_n(X) */
        int32_t c1 = wrap((int64_t)c + 1, ncell);
        double e = w[p] * vt * vt;
        sec[c] += e * (1.0 - th);
        sec[c1] += e * th;
    }
}

/* orc_burst with the three moments: samples[(K+1)][3][ncell] = density, momentum, second
 * moment of each sample p = 0..K. */
int orc_burst_pressure(int64_t n, int32_t* cell, double* theta, double* v, const double* w,
                       int32_t ncell, double dx, double dt, double qm, int32_t K, double dT,
                       int32_t comoving, int32_t mode, int32_t s_w, double tol, int32_t maxit,
                       int32_t vel_at_integer, double* phi, double* samples)
{
    double* E = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* E0 = (double*)malloc(sizeof(double) * (size_t)ncell);
    double* vbar = (double*)malloc(sizeof(double) * (size_t)n);
    int fails = field_from_particles(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    memcpy(E0, E, sizeof(double) * (size_t)ncell); /* E_n, stored at burst start */
    double kick = vel_at_integer ? 0.5 : 1.0;
    for (int32_t p = 0; p <= K; ++p) {
        for (int64_t i = 0; i < n; ++i)
            vbar[i] = v[i] + (kick - 0.5) * qm * dt * orc_gather(E, ncell, cell[i], theta[i]);
        double tau = comoving ? dT - p * dt : 0.0;
        double* row = samples + (size_t)p * 3 * ncell;
        orc_restrict_sample(n, cell, theta, vbar, w, E0, ncell, dx, tau, qm, row, row + ncell);
        orc_restrict_second_moment(n, cell, theta, vbar, w, E0, ncell, dx, tau, qm, row + 2 * (size_t)ncell);
        if (p == K) break;
        orc_push(n, cell, theta, v, E, ncell, dx, dt, qm, kick);
        kick = 1.0;
        fails += field_from_particles(n, cell, theta, w, ncell, dx, mode, s_w, tol, maxit, phi, E);
    }
    free(E);
    free(E0);
    free(vbar);
    return fails;
}

/* Lifting profiles of the three moments: n clamped and rescaled and u = nV / n as in
 * orc_lift_profile, then T = S / n - u^2 where n is above the same floor, clamped at 0 (a
 * projected second moment can fall below the kinetic part n u^2); T = 0 where n is not. */
void orc_lift_profile_pressure(int32_t ncell, double* n, const double* m, const double* s, double* u, double* T)
{
    double nmax = 0.0;
    orc_lift_profile(ncell, n, m, u);
    for (int32_t j = 0; j < ncell; ++j) nmax = fmax(nmax, n[j]);
    for (int32_t j = 0; j < ncell; ++j) {
        double t = (n[j] > 1e-12 * nmax) ? s[j] / n[j] - u[j] * u[j] : 0.0;
        T[j] = t > 0.0 ? t : 0.0;
    }
}

/* Appendix C's loading (orc_quiet_start: the same positions, weights, quantiles and storage
 * order) with a local temperature: V = u(X) + sqrt(T(X)) Phi^-1(b), T linear between the nodes
 * like n and u. */
void orc_quiet_start_thermal(int64_t N, int32_t ncell, const double* nprof, const double* uprof,
                             const double* tprof, uint64_t seed, int32_t* cell, double* theta, double* v,
                             double* w)
{
    double* z = (double*)malloc(sizeof(double) * (size_t)N);
    double* u0 = (double*)calloc((size_t)ncell, sizeof(double));
    /* the loader with u = 0 and v_th = 1 gives each slot its cell, offset, weight and Phi^-1(b) */
    orc_quiet_start(N, ncell, nprof, u0, 1.0, seed, cell, theta, z, w);
    for (int64_t s = 0; s < N; ++s) {
        int32_t c = cell[s];
        int32_t c1 = wrap((int64_t)c + 1, ncell);
        double th = theta[s];
        double uX = (1.0 - th) * uprof[c] + th * uprof[c1];
        double TX = (1.0 - th) * tprof[c] + th * tprof[c1];
        v[s] = uX + sqrt(TX) * z[s];
    }
    free(z);
    free(u0);
}
