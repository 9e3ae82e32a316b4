/*
 * Plain FP64 CPU oracle for the projective-integration PIC hot path
 * (Cazeaux & Hesthaven, "Projective multiscale time-integration for
 * electrostatic particle-in-cell methods").
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library. The GPU product
 * path never calls it, and it shares no source with the GPU path.
 *
 * Every function is a direct, unoptimised statement of one step of the
 * method, in the paper's order, with the paper's notation where it has one.
 * Particle states are (cell, theta, v, w) with theta in [0,1) the offset
 * inside the cell, so that X = (cell + theta) * dx.
 *
 * Units: Debye length, ion plasma frequency, sound speed, e, m_i, T_e and
 * n_0 are 1; ions have charge-to-mass ratio qm; E = -dphi/dx.
 *
 * Parity status: every function below is pinned by a closed form, an
 * invariant, brute force or a library routine in the CPU tests; none is
 * "parity unpinned" except the nonlinear steepening of the full macro-step,
 * which the paper only shows in figures that are not available.
 */
#ifndef PEPIC_ORACLE_H
#define PEPIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Counter-based generator: splitmix64 (Steele, Lea & Flood 2014). */
uint64_t orc_splitmix64(uint64_t x);

/* Fixed-point scale rule: s = 22 - ceil(log2(cap)), so |value * 2^s| <= 2^22. */
int32_t orc_fx_shift(double cap);

/* Section 2.2: CIC charge deposit with the deterministic fixed-point rule
 * theta_q = rn(theta 2^24), w_q = rn(w 2^s_w), q_R = w_q theta_q,
 * q_L = w_q 2^24 - q_R, summed in int64. Overwrites rho[ncell]. Periodic. */
void orc_deposit_fx(int64_t n, const int32_t* cell, const double* theta, const double* w,
                    int32_t ncell, int32_t s_w, int64_t* rho);

/* Plain FP64 CIC deposit of w and of w*vel (vel may be NULL). Overwrites. */
void orc_deposit_f64(int64_t n, const int32_t* cell, const double* theta, const double* w,
                     const double* vel, int32_t ncell, double* dens, double* mom);

/* Cyclic tridiagonal solve a x_{j-1} + b_j x_j + c x_{j+1} = d_j (Thomas with
 * Sherman-Morrison); constant off-diagonals a, c. */
void orc_cyclic_tridiag(int32_t n, double a, const double* b, double c, const double* d, double* x);

/* Section 3.3, Poisson-Boltzmann: -lambda^2 Lap phi + exp(phi) = n_i/n_0 (lambda = n_0 = 1)
 * on the periodic nodal grid, solved by Newton. mode 0: exp(phi); mode 1: the
 * linearised electron response 1 + phi. phi holds the initial guess on entry.
 * Returns 0 on convergence (max |update| < tol), 1 otherwise; *iters gets the
 * number of Newton updates applied. */
int orc_newton_pb(int32_t ncell, double dx, int32_t mode, const double* n, double* phi,
                  double tol, int32_t maxit, int32_t* iters);

/* E_j = -(phi_{j+1} - phi_{j-1}) / (2 dx), periodic. */
void orc_efield(int32_t ncell, double dx, const double* phi, double* E);

/* CIC gather of a nodal field at one particle. */
double orc_gather(const double* F, int32_t ncell, int32_t cell, double theta);

/* Leapfrog kick-drift (Section 2.2): v += kick*qm*dt*E(X); X += v dt; periodic wrap. */
void orc_push(int64_t n, int32_t* cell, double* theta, double* v, const double* E,
              int32_t ncell, double dx, double dt, double qm, double kick);

/* Appendix B, restriction along approximate characteristics: with tau = Delta t - p dt,
 * X~ = X + tau Vbar, V~ = Vbar + qm tau E_n(X); deposits w and w V~ (plain FP64 CIC)
 * at X~. vbar is the integer-time velocity. Overwrites dens/mom [ncell]. */
void orc_restrict_sample(int64_t n, const int32_t* cell, const double* theta, const double* vbar,
                         const double* w, const double* E0, int32_t ncell, double dx,
                         double tau, double qm, double* dens, double* mom);

/* Orthonormal periodized filter bank (Appendix A). h has len taps. One analysis level:
 * approx[k] = sum_m h_m x[(2k+m) mod n], detail[k] = sum_m g_m x[(2k+m) mod n],
 * g_m = (-1)^m h_{len-1-m}. n even. */
void orc_dwt_level(const double* h, int32_t len, const double* x, int32_t n, double* approx, double* detail);
/* One synthesis level, exact inverse of orc_dwt_level. */
void orc_idwt_level(const double* h, int32_t len, const double* approx, const double* detail,
                    int32_t nhalf, double* x);

/* Restriction to scaling coefficients: fine values f_j (j < nfine) are taken as
 * scaling coefficients 2^{-J_f/2} f_j at level J_f, then analysed down to
 * ncoarse coefficients, details discarded (linear thresholding). */
void orc_coarsen(const double* h, int32_t len, const double* fine, int32_t nfine,
                 double* coarse, int32_t ncoarse);
/* Inverse: synthesis with all details zero, then f_j = 2^{J_f/2} a_j. */
void orc_refine(const double* h, int32_t len, const double* coarse, int32_t ncoarse,
                double* fine, int32_t nfine);

/* Section 3.3 extrapolation: least-squares slope of samples y_0..y_K taken at
 * t_p = p dt, from the normal equations of the line fit. */
double orc_ls_slope(int32_t K, double dt, const double* y, int64_t stride);

/* Forward-Euler leap from the last sample: c = y_K + (dT - K dt) slope, for ncoef
 * coefficients stored as samples[p*ncoef + i]. */
void orc_ls_project(int32_t K, int32_t ncoef, double dt, double dT, const double* samples,
                    double* coarse_out, double* slope_out);

/* Inverse of the standard normal CDF (start from Abramowitz-Stegun 26.2.23, then
 * Newton steps on Phi(x) = erfc(-x/sqrt 2)/2). */
double orc_ndtri(double p);

/* Appendix C quiet start on a nodal profile (n_j, u_j), j < ncell, periodic:
 * Hammersley point i of N = ppc*ncell sits at X/dx = floor(i/ppc) + (2 (i mod ppc) + 1)/(2 ppc),
 * weight w = n(X)/ppc, velocity V = u(X) + v_th Phi^{-1}(b_i) with
 * b_i = (B_i + 1/2) 2^-32, B_i = brev32(i) + floor(2^31/N) + (splitmix64(seed) >> 32) mod 2^32
 * (Hammersley second coordinate with a Cranley-Patterson shift). n(X), u(X): linear
 * interpolation between nodes. Storage slot s holds point i = s, except that for
 * ppc = 2^m each cell stores its points in ascending velocity quantile (i = s with its
 * low m bits reversed); the point set is unchanged. */
void orc_quiet_start(int64_t N, int32_t ncell, const double* nprof, const double* uprof,
                     double v_th, uint64_t seed, int32_t* cell, double* theta, double* v, double* w);

/* Lifting profile: clamp negative densities to 0 and rescale to keep sum(n) (C18),
 * u_j = m_j / n_j where n_j > 1e-12 max n, else 0. In place on n; u written. */
void orc_lift_profile(int32_t ncell, double* n, const double* m, double* u);

/* One resolved PIC burst of K steps with co-moving restriction samples.
 * State holds v at integer time on entry (vel_at_integer = 1) or at half-integer
 * time (0). On exit v is at half-integer time. samples: [(K+1)][2][ncell]
 * (density, momentum). phi is the Newton warm start and is updated.
 * Returns the number of Newton failures. */
int orc_burst(int64_t n, int32_t* cell, double* theta, double* v, const double* w,
              int32_t ncell, double dx, double dt, double qm, int32_t K, double dT,
              int32_t comoving, int32_t mode, int32_t s_w, double tol, int32_t maxit,
              int32_t vel_at_integer, double* phi, double* samples);

/* Plain PIC: nsteps leapfrog steps (deposit, Newton, gather+push). Same v convention. */
int orc_pic_steps(int64_t n, int32_t* cell, double* theta, double* v, const double* w,
                  int32_t ncell, double dx, double dt, double qm, int32_t nsteps,
                  int32_t mode, int32_t s_w, double tol, int32_t maxit,
                  int32_t vel_at_integer, double* phi);

/* Diagnostics (Section 4: conservation checks; particle CFL number). Integer-time
 * velocities Vbar = v + (kick - 1/2) qm dt E(X). charge_fx = sum_p rn(w 2^s_w) 2^24 (the
 * sum of the fixed-point deposit). out[8] = {charge sum w dx, momentum sum w Vbar dx,
 * kinetic sum w Vbar^2 dx / 2, field sum E^2 dx / 2, electron free energy
 * sum (phi e^phi - e^phi + 1) dx (mode 0) or sum phi^2 dx / 2 (mode 1), total,
 * max |Vbar|, max |Vbar| dt / dx}. */
void orc_moments(int64_t n, const int32_t* cell, const double* theta, const double* v, const double* w,
                 const double* E, const double* phi, int32_t ncell, double dx, double dt, double qm,
                 double kick, int32_t s_w, int32_t mode, int64_t* charge_fx, double* out);

/* Section 4.1.1 error measure: sqrt(sum (a-b)^2 / sum (a^2 + b^2)); 0 if both vanish. */
double orc_rel_l2(int64_t n, const double* a, const double* b);

/* ---- phase-space coarse variable (Section 3.3 "A wavelet-based equation-free scheme",
 * Appendices B and C), Haar reading: the active variables are the masses H[i][j] of the
 * phase-space cells (coarse x-bin i of 2^b nodes, velocity cell j of width dv from vmin).
 * These are the Haar scaling coefficients of the histogram up to one constant factor. */

/* Co-moving phase-space restriction sample in the fixed-point rule: particle at
 * X~ = X + tau Vbar (CIC nodes c, c+1 with offset theta~), V~ = Vbar + qm tau E_n(X), velocity
 * cell j = floor((V~ - vmin)/dv) clamped to [0, nv): q_L = w_q (2^24 - theta~_q) to
 * (c >> b, j), q_R = w_q theta~_q to ((c+1) >> b, j). F[(ncell >> b)][nv] int64, overwritten. */
void orc_ps_sample_fx(int64_t n, const int32_t* cell, const double* theta, const double* vbar, const double* w,
                      const double* E0, int32_t ncell, double dx, double tau, double qm, int32_t bin_shift,
                      double vmin, double dv, int32_t nv, int32_t s_w, int64_t* F);

/* Appendix C, momentum-conserving reconstruction of a cumulative distribution F[0..N]
 * (F[0] = 0 and F[N] = 1 are imposed): edge reconstruction of entries below 0 and above 1,
 * then the interior reconstruction from the low indices and from the high indices,
 * averaged. In place. Returns 1 if a pathological case needed a clamp or running max. */
int orc_cdf_reconstruct(int32_t N, double* F);

/* Lifting tables of the phase-space histogram H[nxc][nv]: bin masses (negative masses
 * clamped to 0, the rest rescaled to keep the total) into mass[nxc], and per bin the
 * reconstructed CDF over velocity cells into cdf[nxc][nv+1] (uniform where the raw mass is
 * not positive). Returns 1 if any reconstruction was pathological. */
int orc_ps_lift_tables(int32_t nxc, int32_t nv, const double* H, double* mass, double* cdf);

/* Relative density slope of each velocity cell of a CDF table F[0..nv]:
 * sigma_k = (p_{k+1} - p_{k-1}) / (4 p_k) clamped to [-1, 1], p_k = F[k+1] - F[k] (p = 0 outside),
 * so that the cell's density 1 + sigma (2t - 1), t in [0, 1], follows its neighbours and stays
 * non-negative. */
void orc_cdf_cell_slopes(int32_t nv, const double* F, double* sigma);

/* Inverse of a monotone CDF table F[0..nv] at b in (0, 1): with k the first index where
 * F[k+1] > b and r = (b - F[k]) / (F[k+1] - F[k]), V = vmin + dv (k + t) where t solves
 * t + sigma_k (t^2 - t) = r (linear density inside the cell; sigma NULL: uniform, t = r). */
double orc_cdf_inverse(int32_t nv, const double* F, const double* sigma, double b, double vmin, double dv);

/* Appendix C particle loading on the phase-space tables: the Hammersley points of
 * orc_quiet_start (same positions, quantiles b and storage order). The lifted f(x, v) is
 * linear in x between neighbouring bin centres: with phi the particle's distance from the
 * centre of the bin b0 at or left of it, in bin widths, and b1 = b0 + 1 (periodic),
 * w = ((1 - phi) mass[b0] + phi mass[b1]) 2^-b / ppc and V = (1 - phi) G_b0(b) + phi G_b1(b),
 * G the CDF inverse of a bin (quantile interpolation) with linear density inside each velocity
 * cell (orc_cdf_cell_slopes): uniform cells would add dv^2/12 to the temperature at every
 * lift. */
void orc_ps_quiet_start(int64_t N, int32_t ncell, int32_t bin_shift, const double* mass, const double* cdf,
                        int32_t nv, double vmin, double dv, uint64_t seed, int32_t* cell, double* theta,
                        double* v, double* w);

/* orc_burst with phase-space samples: samples[(K+1)][(ncell >> b)][nv] int64. */
int orc_ps_burst(int64_t n, int32_t* cell, double* theta, double* v, const double* w, int32_t ncell, double dx,
                 double dt, double qm, int32_t K, double dT, int32_t mode, int32_t s_w, double tol, int32_t maxit,
                 int32_t vel_at_integer, int32_t bin_shift, double vmin, double dv, int32_t nv, double* phi,
                 int64_t* samples);

/* ---- bounded grid (Section 4.2): walls at node 0 and node ncell-1, absorbing for the ions,
 * phi' = 0 for the potential (mirror ghosts), wall nodes at half control volume. */
int orc_newton_pb_walls(int32_t ncell, double dx, int32_t mode, const double* dep, double* phi, double tol,
                        int32_t maxit, int32_t* iters);
void orc_efield_walls(int32_t ncell, double dx, const double* phi, double* E);
void orc_push_walls(int64_t n, int32_t* cell, double* theta, double* v, double* w, const double* E,
                    int32_t ncell, double dx, double dt, double qm, double kick);
void orc_restrict_sample_walls(int64_t n, const int32_t* cell, const double* theta, const double* vbar,
                               const double* w, const double* E0, int32_t ncell, double dx, double tau,
                               double qm, double* dens, double* mom);
void orc_quiet_start_equal(int64_t N, int32_t ncell, const double* nprof, const double* uprof, double v_th,
                           uint64_t seed, int32_t* cell, double* theta, double* v, double* w);
int orc_burst_walls(int64_t n, int32_t* cell, double* theta, double* v, double* w, int32_t ncell, double dx,
                    double dt, double qm, int32_t K, double dT, int32_t comoving, int32_t mode, int32_t s_w,
                    double tol, int32_t maxit, int32_t vel_at_integer, double* phi, double* samples);
int orc_pic_steps_walls(int64_t n, int32_t* cell, double* theta, double* v, double* w, int32_t ncell, double dx,
                        double dt, double qm, int32_t nsteps, int32_t mode, int32_t s_w, double tol, int32_t maxit,
                        int32_t vel_at_integer, double* phi);
void orc_ps_sample_fx_walls(int64_t n, const int32_t* cell, const double* theta, const double* vbar,
                            const double* w, const double* E0, int32_t ncell, double dx, double tau, double qm,
                            int32_t bin_shift, double vmin, double dv, int32_t nv, int32_t s_w, int64_t* F);
void orc_ps_quiet_start_equal(int64_t N, int32_t ncell, int32_t bin_shift, const double* mass, const double* cdf,
                              int32_t nv, double vmin, double dv, uint64_t seed, int32_t* cell, double* theta,
                              double* v, double* w);
int orc_ps_burst_walls(int64_t n, int32_t* cell, double* theta, double* v, double* w, int32_t ncell, double dx,
                       double dt, double qm, int32_t K, double dT, int32_t mode, int32_t s_w, double tol,
                       int32_t maxit, int32_t vel_at_integer, int32_t bin_shift, double vmin, double dv, int32_t nv,
                       double* phi, int64_t* samples);

/* Phase space, wavelet form (Section 3.3 as stated: fine histogram, 1-2-1 in x, DWT in v). */
void orc_ps_hist_fine(int64_t n, const int32_t* cell, const double* theta, const double* vbar, const double* w,
                      const double* E0, int32_t ncell, double dx, double tau, double qm, double vmin, double dv,
                      int32_t nvf, double* H);
int orc_ps_burst_fine(int64_t n, int32_t* cell, double* theta, double* v, const double* w, int32_t ncell, double dx,
                      double dt, double qm, int32_t K, double dT, int32_t mode, int32_t s_w, double tol, int32_t maxit,
                      int32_t vel_at_integer, double vmin, double dv, int32_t nvf, double* phi, double* samples);
void orc_ps_quiet_start_nodes(int64_t N, int32_t ncell, int32_t bin_shift, const double* mass, const double* cdf,
                              int32_t nvf, double vmin, double dv, uint64_t seed, int32_t* cell, double* theta,
                              double* v, double* w);

/* Kinetic electrons (Section 4.1's two-species bursts). */
void orc_poisson_periodic(int32_t ncell, double dx, const double* r, double* phi, double* E);
void orc_field_kinetic(int64_t ni, const int32_t* ci, const double* ti, const double* wi, int64_t ne,
                       const int32_t* ce, const double* te, const double* we, int32_t ncell, double dx, int32_t s_w,
                       double* phi, double* E);
void orc_pic_steps_kinetic(int64_t ni, int32_t* ci, double* ti, double* vi, const double* wi, int64_t ne,
                           int32_t* ce, double* te, double* ve, const double* we, int32_t ncell, double dx, double dt,
                           double qm_i, double qm_e, int32_t nsteps, int32_t s_w, int32_t vel_at_integer,
                           int32_t e_vel_at_integer, double* phi);
void orc_burst_kinetic(int64_t ni, int32_t* ci, double* ti, double* vi, const double* wi, int64_t ne,
                       int32_t* ce, double* te, double* ve, const double* we, int32_t ncell, double dx, double dt,
                       double qm_i, double qm_e, int32_t K, double dT, int32_t s_w, int32_t vel_at_integer,
                       int32_t bin_shift, double vmin, double dv, int32_t nv, double* phi, double* samples,
                       int64_t* samples_fx);
void orc_boltzmann_electrons(int64_t N, int32_t ncell, const double* phi, const double* u, double v_th_e,
                             uint64_t seed, int32_t* cell, double* theta, double* v, double* w);

/* ---- ion pressure (Section 3.2, EFREE's n, V, P): the second velocity moment as a third
 * restriction sample and the lifting at a local temperature. */
/* sec[j] = sum_p w_p V~_p^2 S_j(X~_p), with X~, V~ as in orc_restrict_sample. */
void orc_restrict_second_moment(int64_t n, const int32_t* cell, const double* theta, const double* vbar,
                                const double* w, const double* E0, int32_t ncell, double dx, double tau,
                                double qm, double* sec);
/* orc_burst with samples[(K+1)][3][ncell]: density, momentum, second moment. */
int orc_burst_pressure(int64_t n, int32_t* cell, double* theta, double* v, const double* w,
                       int32_t ncell, double dx, double dt, double qm, int32_t K, double dT,
                       int32_t comoving, int32_t mode, int32_t s_w, double tol, int32_t maxit,
                       int32_t vel_at_integer, double* phi, double* samples);
/* orc_lift_profile, then T = max(S / n - u^2, 0) (0 where n is below the floor). */
void orc_lift_profile_pressure(int32_t ncell, double* n, const double* m, const double* s, double* u, double* T);
/* orc_quiet_start with V = u(X) + sqrt(T(X)) Phi^-1(b). */
void orc_quiet_start_thermal(int64_t N, int32_t ncell, const double* nprof, const double* uprof,
                             const double* tprof, uint64_t seed, int32_t* cell, double* theta, double* v,
                             double* w);

#ifdef __cplusplus
}
#endif
#endif
