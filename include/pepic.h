/*
 * pepic.h — C ABI of the GB300 (sm_103a) projective-integration PIC library
 * (libpepic.so). Method: Cazeaux & Hesthaven, "Projective multiscale
 * time-integration for electrostatic particle-in-cell methods".
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Units: Debye length, ion plasma frequency, sound speed, e, m_i, T_e, n_0 = 1.
 * - Periodic domain [0, L) with ncell cells (ncell a power of two, >= 8), nodes
 *   x_j = j dx, dx = L / ncell.
 * - A particle is (cell int32, theta float, v float, w float): X = (cell + theta) dx,
 *   theta in [0, 1). Arrays are structure-of-arrays, device memory, each base
 *   pointer 16-byte aligned (any torch CUDA allocation is). Any n >= 0 is allowed.
 * - Fixed-point deposit rule (deterministic, order independent): theta_q =
 *   rn(theta 2^24), w_q = rn(w 2^s_w), q_R = w_q theta_q, q_L = w_q (2^24 - theta_q),
 *   summed in int64 at nodes cell and cell+1. Density n_j = rho_j 2^-(s_w+24).
 *   Momentum uses the same split with m_q = rn(w V 2^s_p). Choose s_w so that
 *   w 2^s_w <= 2^22 (pe_config.w_cap does this for the context API).
 * - "stream" is a cudaStream_t (NULL = legacy default stream). All device work is
 *   asynchronous on it; no entry point allocates or frees device memory: the
 *   caller owns every buffer.
 * - Errors: a return value != PE_OK means nothing was launched (bad arguments or a
 *   launch error). Faults found on the device (particle cell out of range,
 *   fixed-point overflow, Newton non-convergence) are OR-ed into a caller-owned
 *   device status word (uint32) as PE_FLAG_* bits and never trap; the caller reads
 *   it after synchronising (the context API does this in pe_sync_status). The only
 *   spin-waits are the tensor-core GEMM's mbarrier waits (pe_tc_gemm_bf16 and the
 *   surrogate's products): each is bounded by a clock budget, after which the kernel sets
 *   PE_FLAG_TIMEOUT, waits (bounded again) for its copies in flight, frees its tensor
 *   memory and returns (PE_ETIMEOUT from pe_mlp_sync_status). Every other device-side wait
 *   is a block or cluster barrier that every thread reaches.
 */
#ifndef PEPIC_H
#define PEPIC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PE_API __attribute__((visibility("default")))
#else
#define PE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define PE_OK 0
#define PE_EINVAL 1    /* invalid argument (size, alignment, power of two, ...) */
#define PE_ECUDA 2     /* CUDA runtime error while launching */
#define PE_ENOCONV 3   /* Newton did not converge within newton_maxit */
#define PE_EOVERFLOW 4 /* a weight or momentum exceeded its fixed-point range */
#define PE_ERANGE 5    /* a particle cell index was outside [0, ncell) */
#define PE_ESTATE 6    /* call out of order for the context state */
#define PE_ETIMEOUT 7  /* a bounded device-side wait timed out (the tensor-core GEMM's mbarrier waits) */

#define PE_FLAG_NOCONV 1u
#define PE_FLAG_OVERFLOW 2u
#define PE_FLAG_RANGE 4u
#define PE_FLAG_TIMEOUT 8u

#define PE_WAVELET_HAAR 0 /* orthonormal Haar filter */
#define PE_WAVELET_D4 1   /* Daubechies 4-tap orthonormal filter */
#define PE_WAVELET_COIF4 2 /* order-4 coiflet of Appendix A (12 taps, k = -4..7): four vanishing
                              wavelet moments, scaling-function moments 1..3 vanish; its taps are
                              solved from those equations by the library at first use */

#define PE_POISSON_BOLTZMANN 0  /* -Lap phi + exp(phi) = n   (Section 3.3, Eq. poisson2rescaled) */
#define PE_POISSON_LINEARIZED 1 /* -Lap phi + 1 + phi = n    (its small-amplitude limit) */

#define PE_COARSE_MOMENTS 0     /* density and momentum, wavelet in x (Section 3.2 variables) */
#define PE_COARSE_PHASE_SPACE 1 /* phase-space cell masses (Section 3.3), Haar in x and v */
#define PE_COARSE_MOMENTS_PRESSURE 2 /* density, momentum and the second velocity moment, wavelet
                                        in x (Section 3.2: EFREE's ion n, V and P = n T active) */

#define PE_PROFILE_SINE 0 /* n = 1 + a cos(2 pi x / L), u = a cos(2 pi x / L) (Section 4.1) */
#define PE_PROFILE_SLAB 1 /* n = 1 on the nodes 7 ncell/16 .. 9 ncell/16, 0 elsewhere; u = 0
                             (Section 4.2's slab in vacuum, uniform variant; bounded grids) */

/* Boundary of the grid. Periodic: nodes j = 0..ncell-1 wrap. Absorbing (Section 4.2, the
 * slab expansion): walls at node 0 (x = 0) and node ncell-1 (x = (ncell-1) dx); the ions
 * live in the ncell-1 cells between them, phi' = 0 at both walls (mirror ghosts, so E = 0
 * there), a wall node's density is twice its deposit (half control volume), and an ion whose
 * drift ends outside [0, (ncell-1) dx) is absorbed: its weight becomes 0, v = 0, and it is
 * parked on the wall node it crossed (cell 0 or cell ncell-1, theta 0). Particles of weight
 * 0 are not moved and add nothing to deposits, samples or diagnostics. */
#define PE_BOUNDARY_PERIODIC 0
#define PE_BOUNDARY_ABSORBING 1

/* Electrons. Boltzmann: a fluid in equilibrium with the potential (Eq. electronpassive), so the
 * field is the Poisson-Boltzmann equation (pe_field). Kinetic (Section 4.1: the paper's PIC
 * bursts move both species): nparticles electron particles beside the ions, charge-to-mass
 * ratio qm_e, pushed with the same kernels; the field is the Poisson equation for the net
 * charge (pe_field_kinetic). Every load and every lift places the electrons in Boltzmann
 * equilibrium with the ions: the Poisson-Boltzmann potential of the ion density, then a quiet
 * start on exp(phi) with thermal speed v_th_e drifting with the ions' mean velocity
 * (pe_boltzmann_profile). Kinetic
 * electrons need a periodic grid and a time step that resolves the electron plasma period
 * (|qm_e|^(-1/2) in these units). */
#define PE_ELECTRONS_BOLTZMANN 0
#define PE_ELECTRONS_KINETIC 1

PE_API const char* pe_strerror(int code);
PE_API const char* pe_version(void);

/* =================================================================== kernels
 * Stateless entry points: one hot-path step each, on caller buffers.
 */

/* Charge deposit, Section 2.2 (particles projected on the nodes with the CIC
 * shape). rho_fx[ncell] (int64) is overwritten with the fixed-point nodal charge
 * of the n particles. Exact and independent of particle order. */
PE_API int pe_deposit(const int32_t* cell, const float* theta, const float* w, int64_t n,
                      int32_t ncell, int32_t s_w, int64_t* rho_fx, uint32_t* status, void* stream);

/* Field solve, Section 3.3, Eq. (poisson2rescaled) discretised on the nodes:
 * -(phi_{j+1} - 2 phi_j + phi_{j-1}) / dx^2 + g(phi_j) = n_j with g = exp (mode
 * PE_POISSON_BOLTZMANN) or 1 + phi (PE_POISSON_LINEARIZED), n_j = rho_fx_j 2^-(s_w+24).
 * Newton iteration in FP64 from the initial guess in phi[ncell] (in/out), each
 * update a cyclic tridiagonal solve, damped to |update| <= 2, stopped when
 * max|update| < tol. Then E_j = -(phi_{j+1} - phi_{j-1}) / (2 dx) into E[ncell]
 * (FP64) and Ef[ncell] (FP32 copy used by the particle kernels).
 * diag (device, int32[4], may be NULL) gets {iterations, converged, blocks, threads
 * per block}: grids of 1024 nodes or more are solved by one thread-block cluster
 * (up to 16 blocks, one per SM), smaller ones by a single block. Non-convergence
 * sets PE_FLAG_NOCONV. */
PE_API int pe_field(const int64_t* rho_fx, int32_t ncell, double dx, int32_t s_w, int32_t mode,
                    double tol, int32_t maxit, double* phi, double* E, float* Ef, int32_t* diag,
                    uint32_t* status, void* stream);

/* pe_field with a boundary (PE_BOUNDARY_*). With PE_BOUNDARY_ABSORBING the equations at the
 * wall nodes use the mirror ghosts and twice the deposit, E is 0 on the walls, and the
 * Jacobian solve runs in FP64 (vacuum regions make it ill-conditioned for FP32).
 * pe_field is pe_field_ex with PE_BOUNDARY_PERIODIC. */
PE_API int pe_field_ex(const int64_t* rho_fx, int32_t ncell, double dx, int32_t s_w, int32_t mode,
                       int32_t boundary, double tol, int32_t maxit, double* phi, double* E, float* Ef,
                       int32_t* diag, uint32_t* status, void* stream);

/* Field of a two-species (kinetic-electron) state, Section 4.1: the paper's ion-acoustic
 * bursts move the electrons as particles (q_e/m_e = -1800), so the field is the plain
 * Poisson equation for the net charge on the periodic grid,
 *   -(phi_{j+1} - 2 phi_j + phi_{j-1}) / dx^2 = r_j - <r>,  r_j = (rho_i_j - rho_e_j) 2^-(s_w+24),
 * with <phi> = 0 (the mean of r, a fixed-point rounding remainder of a neutral system, is
 * a uniform background), and E_j = -(phi_{j+1} - phi_{j-1}) / (2 dx).
 * rho_i[ncell], rho_e[ncell]: fixed-point deposits (pe_deposit / pe_push rule, same s_w) of
 * the ions and of the electrons (both with positive weights). Writes phi[ncell], E[ncell]
 * (FP64) and Ef[ncell] (FP32). One block: a prefix sum of the net charge (the per-node int64
 * difference is exact, the sums FP64 in a fixed order) gives the face fields
 * F_{j+1/2} = -(phi_{j+1} - phi_j)/dx (discrete Gauss law), their mean is removed (phi
 * periodic), then E_j = (F_{j+1/2} + F_{j-1/2}) / 2 and phi by a second sum. Periodic grids
 * only; ncell a power of two, 8..8192. */
PE_API int pe_field_kinetic(const int64_t* rho_i, const int64_t* rho_e, int32_t ncell, double dx, int32_t s_w,
                            double* phi, double* E, float* Ef, void* stream);

/* Boltzmann electron profile of the lifting, Eq. (electronpassive): n_e = exp(phi) and
 * V_e = V_i. n_prof[j] = exp(phi[j]) (FP32), the profile pe_quiet_start loads the electrons
 * from (with their thermal speed); phi[ncell] is the Poisson-Boltzmann potential of the ion
 * density (pe_field). u_prof[j] = the ions' mean velocity at node j, m_j 2^-s_p / (n_j 2^-s_w),
 * from their nodal moment sample ion_moments (int64[2][ncell], density then momentum: pe_sample
 * with tau = 0 and bin_shift = 0, shifts s_w and s_p); 0 where n_j <= 0, and everywhere when
 * ion_moments is NULL. u_prof may be NULL when ion_moments is: only n_prof is written (the
 * caller's u_prof already holds the ions' velocity, e.g. the lifting profile). */
PE_API int pe_boltzmann_profile(const double* phi, const int64_t* ion_moments, int32_t s_w, int32_t s_p,
                                int32_t ncell, float* n_prof, float* u_prof, void* stream);

/* Mean ion velocity of a phase-space coarse state at the nodes, for V_e = V_i when the ions are
 * lifted from it (Section 3.3: the ion density and velocity follow by integrating the coarse
 * distribution along v): per x-bin b the mean sum_k (v_min + (k + 1/2) dv) (F_b[k+1] - F_b[k])
 * of its reconstructed CDF row (pe_ps_lift_tables' cdf[nxc][n_v + 1]), then linear between bin
 * midpoints (periodic) into u_prof[ncell] (FP32); ncell = nxc 2^bin_shift <= 8192. */
PE_API int pe_ps_mean_velocity(const double* cdf, int32_t nxc, int32_t n_v, double v_min, double dv,
                               int32_t bin_shift, int32_t ncell, float* u_prof, void* stream);

/* Co-moving restriction sample, Appendix B (Eq. explicitflow and the deposit that
 * follows it): each particle, at its integer-time velocity Vbar, is carried to
 * X~ = X + tau Vbar, V~ = Vbar + qm tau E_n(X), and w and w V~ are deposited
 * (CIC, fixed point) at X~. tau = Delta t - p delta t (0 disables the frame).
 * With bin_shift = b > 0 the sample holds, for each bin of 2^b nodes, the exact sum
 * of the nodal fixed-point sample over the bin (the Haar restriction only needs these
 * sums; a particle whose two CIC nodes share a bin then adds its whole w 2^24).
 * With n_v > 0 the sample is instead the phase-space histogram of Section 3.3 at the same
 * co-moving targets (Appendix B): each particle adds its fixed-point w, CIC-split in x, to
 * the coarse x-bins of its two nodes (bins of 2^b nodes; b = 0 for nodes) and to the
 * velocity cell j = floor((V~ - v_min) / dv) clamped to [0, n_v). Exact and order
 * independent like the deposit. */
typedef struct pe_sample_args {
    const float* E0f;  /* E_n, the field stored at burst start, float[ncell] */
    float tau;         /* Delta t - p delta t */
    float qm;          /* ion charge-to-mass ratio */
    float inv_dx;      /* 1 / dx */
    int32_t s_w;       /* density fixed-point shift (pe_push requires the same s_w) */
    int32_t s_p;       /* momentum fixed-point shift: |w V~| 2^s_p must stay <= 2^22 */
    int32_t bin_shift; /* 0: nodal sample; b > 0: sums over bins of 2^b consecutive nodes */
    int64_t* sample_fx; /* int64[2][ncell >> bin_shift]: density then momentum; overwritten
                           (phase-space sample: int64[ncell >> bin_shift][n_v]) */
    int32_t n_v;        /* 0: moment sample; > 0: phase-space sample with n_v velocity cells */
    float v_min;        /* phase space: lower velocity bound V_min */
    float inv_dv;       /* phase space: 1 / dv, dv = (V_max - V_min) / n_v */
    int32_t boundary;   /* PE_BOUNDARY_*: with walls, a particle whose target X~ lies outside
                           [0, (ncell-1) dx) is not counted (it has left the domain by t_{n+1}) */
    int32_t x_tent;     /* phase space, periodic: 0 sums the CIC weights over bins of 2^b nodes;
                           1 samples row i = coarse node i (fine node i 2^b) with the hat of
                           half-width 2^b, i.e. Eq. (restriction) applied b times to the CIC
                           histogram: a target at fine position y adds w (1 - f) to node
                           i = floor(y / 2^b) and w f to node i + 1, f = y / 2^b - i, in fixed
                           point f_q = rn(fl32((y mod 2^b)) 2^(24-b)); the rows hold 2^b times
                           the averaged values of that rule */
    int32_t second_moment; /* 1: a third nodal moment, the ions' second velocity moment
                              S_j = sum_p w V~^2 S_j(X~) (Section 3.2: EFREE's pressure
                              P = S - (nV)^2 / n is active), in fixed point
                              e_q = rn(fl32(fl32(w V~) V~) 2^s_e) split like the density (and
                              summed over bins like it when bin_shift > 0); then sample_fx is
                              int64[3][ncell >> bin_shift] (density, momentum, S); needs n_v = 0
                              and a periodic grid */
    int32_t s_e;           /* second-moment fixed-point shift: |w V~^2| 2^s_e must stay <= 2^22 */
} pe_sample_args;

/* Leapfrog gather + push, Section 2.2, fused with the charge deposit of the new
 * positions and (if sample != NULL) with the co-moving restriction sample of the
 * current positions:
 *   E(X) = (1 - theta) Ef[cell] + theta Ef[cell+1]
 *   Vbar = v + (kick - 1/2) qm_dt E(X)        (integer-time velocity, sample only)
 *   v   += kick qm_dt E(X)                      (kick = 1/2 when v is at integer time)
 *   X   += v dt, periodic; cell/theta/v updated in place.
 * rho_fx[ncell] is overwritten with the deposit of the pushed particles. */
PE_API int pe_push(int32_t* cell, float* theta, float* v, const float* w, int64_t n,
                   const float* Ef, int32_t ncell, float dt_over_dx, float qm_dt, float kick,
                   int32_t s_w, int64_t* rho_fx, const pe_sample_args* sample,
                   uint32_t* status, void* stream);

/* pe_push with a boundary (PE_BOUNDARY_*). With PE_BOUNDARY_ABSORBING, w is written: an ion
 * absorbed during this step gets w = 0 (see PE_BOUNDARY_ABSORBING); a live particle found on
 * cell ncell-1 sets PE_FLAG_RANGE and is left unchanged. sample->boundary must equal boundary.
 * pe_push is pe_push_ex with PE_BOUNDARY_PERIODIC (w only read). */
PE_API int pe_push_ex(int32_t* cell, float* theta, float* v, float* w, int64_t n, const float* Ef,
                      int32_t ncell, float dt_over_dx, float qm_dt, float kick, int32_t s_w,
                      int32_t boundary, int64_t* rho_fx, const pe_sample_args* sample,
                      uint32_t* status, void* stream);

/* Restriction sample only (no push), e.g. the last sample p = N_e of a burst:
 * the same sample as pe_push, with Vbar = v + (kick - 1/2) qm_dt E(X). */
PE_API int pe_sample(const int32_t* cell, const float* theta, const float* v, const float* w,
                     int64_t n, const float* Ef, int32_t ncell, float qm_dt, float kick,
                     const pe_sample_args* sample, uint32_t* status, void* stream);

/* Restriction to coarse variables, Section 3.3 and Appendix A (Eq.
 * ScalingCoeffHistogram): for each of nsamples samples and each moment
 * (density, momentum) the fine nodal values f_j = sample_fx 2^-(s+24) are taken as
 * scaling coefficients 2^{-J_f/2} f_j at level J_f = log2(ncell), then the periodized
 * orthonormal DWT is applied down to n_coarse scaling coefficients; details are
 * discarded. coarse[nsamples][2][n_coarse] (FP64) is overwritten.
 * bin_shift = b > 0 (Haar only) takes samples of bin sums over 2^b nodes
 * (sample_fx[nsamples][2][ncell >> b]); the Haar analysis of b levels is then the
 * exact bin sum scaled by 2^{-(J_f + b)/2}. */
PE_API int pe_coarsen(const int64_t* sample_fx, int32_t nsamples, int32_t ncell, int32_t s_w,
                      int32_t s_p, int32_t wavelet, int32_t n_coarse, int32_t bin_shift, double* coarse,
                      void* stream);

/* Projective forward-Euler step, Section 3.3, Eqs. (extrapolation2) and
 * (leastsquares): slope_i = sum_p 6 (K - 2p) / (K (K+1) (K+2) dt) [c_{K-p,i} - c_{p,i}],
 * out_i = c_{K,i} + (dT - K dt) slope_i, for ncoef coefficients of samples
 * c[(K+1)][ncoef]. slope (may be NULL) and out are FP64[ncoef]. */
PE_API int pe_ls_project(const double* samples, int32_t K, int32_t ncoef, double dt, double dT,
                         double* out, double* slope, void* stream);

/* Lifting profile, Section 3.3 ("increasing the resolution"): inverse DWT of the
 * coarse density and momentum coefficients coarse[2][n_coarse] with zero details,
 * f_j = 2^{J_f/2} a_j; negative densities clamped to 0 and the density rescaled to
 * keep its sum; u_j = m_j / n_j (0 where n_j <= 1e-12 max n). Writes float
 * prof_n[ncell], prof_u[ncell]. */
PE_API int pe_refine(const double* coarse, int32_t n_coarse, int32_t wavelet, int32_t ncell,
                     float* prof_n, float* prof_u, void* stream);

/* pe_refine with FP64 profiles (the lifting of the FP64-particle path). */
PE_API int pe_refine_f64(const double* coarse, int32_t n_coarse, int32_t wavelet, int32_t ncell,
                         double* prof_n, double* prof_u, void* stream);

/* Quiet-start loading, Appendix C, on nodal profiles (linear interpolation): the
 * Hammersley point h of n = ppc*ncell: cell = h / ppc, theta = (2 (h mod ppc) + 1) / (2 ppc),
 * w = n(X) / ppc, V = u(X) + v_th Phi^-1(b_h), b_h = (B_h + 1/2) 2^-32 with
 * B_h = brev32(h) + floor(2^31 / n) + (splitmix64(seed) >> 32) mod 2^32 (second Hammersley
 * coordinate with a Cranley-Patterson shift). Storage slot i holds point h = i, except
 * that with ppc = 2^m each cell stores its points in ascending order of the velocity
 * quantile (h = i with its low m bits reversed): the same point set, ordered so that
 * positions at any later time, and co-moving targets, vary smoothly along the array.
 * Output is sorted by cell. If rho_fx != NULL it is overwritten with the charge deposit
 * of the new particles. */
PE_API int pe_quiet_start(int32_t* cell, float* theta, float* v, float* w, int64_t n,
                          int32_t ncell, const float* prof_n, const float* prof_u, float v_th,
                          uint64_t seed, int32_t s_w, int64_t* rho_fx, uint32_t* status,
                          void* stream);

/* The storage slots [first, first + n) of pe_quiet_start's point set of n_total points,
 * written to local arrays of n particles (local particle k = global slot first + k): the
 * particles one rank holds when a realisation's particles are split over ranks (Appendix C's
 * point set is defined for the whole realisation, so every slice of it is loaded exactly as
 * the unsplit run would). If rho_fx != NULL it is overwritten with the charge deposit of
 * the slice; the deposits of the slices of a partition of [0, n_total) sum to the deposit of
 * the whole point set, bit for bit (fixed-point integers). Requires n_total a multiple of
 * ncell and below 2^32, 0 <= first <= n_total - n, n >= 1; arrays as pe_quiet_start's. */
PE_API int pe_quiet_start_slice(int32_t* cell, float* theta, float* v, float* w, int64_t first,
                                int64_t n, int64_t n_total, int32_t ncell, const float* prof_n,
                                const float* prof_u, float v_th, uint64_t seed, int32_t s_w,
                                int64_t* rho_fx, uint32_t* status, void* stream);

/* The fixed-point shifts of the deposit rule (s_w for weights, s_p for momenta) that a context
 * of nparticles ions on ncell cells uses: s = 22 - ceil(log2 cap) with the weight cap w_cap
 * (0: 8 ncell / nparticles) and the momentum cap w_cap v_cap (v_cap 0: 32). A realisation
 * split over ranks uses the shifts of its total particle count on every rank. */
/* FP64 particles (Section 2.2 and Appendices B and C as pe_push, pe_sample and pe_quiet_start,
 * with theta, v and w in double precision): the small workload runs both ways, so that the
 * error of a run against an FP64 reference separates into the FP32 particles' precision and
 * the method itself. cell int32[n]; theta, v, w double[n] (any alignment); E and E0 the FP64
 * nodal fields (pe_field's E); prof_n, prof_u FP64 nodal profiles. The fixed-point rule is
 * the FP32 particles' (theta_q = rn(theta 2^24), w_q = rn(w 2^s_w), m_q = rn(w V 2^s_p)).
 * pe_push_f64: kick by kick qm_dt E(X), drift by v dt_over_dx cells; if E0 != NULL it first
 * writes the co-moving restriction sample of the current state to sample_fx[2][ncell]
 * (density then momentum, nodal, fixed point): target X + tau Vbar, velocity
 * Vbar + qm tau E0(X), Vbar = v + (kick - 1/2) qm_dt E(X), with tau_over_dx = tau / dx and
 * qm_tau = qm tau. If rho_fx != NULL it is overwritten with the deposit of the pushed
 * particles. pe_sample_f64 writes the sample only. pe_quiet_start_f64 loads the point set of
 * pe_quiet_start (storage order included), with Phi^-1 in double precision, and the deposit
 * into rho_fx if not NULL. One thread per particle, 64-bit global atomics: meant for small
 * particle counts. Errors as pe_push (PE_FLAG_RANGE, PE_FLAG_OVERFLOW in status). */
PE_API int pe_push_f64(int32_t* cell, double* theta, double* v, const double* w, int64_t n,
                       const double* E, int32_t ncell, double dt_over_dx, double qm_dt, double kick,
                       int32_t s_w, int64_t* rho_fx, const double* E0, double tau_over_dx, double qm_tau,
                       int32_t s_p, int64_t* sample_fx, uint32_t* status, void* stream);
PE_API int pe_sample_f64(const int32_t* cell, const double* theta, const double* v, const double* w,
                         int64_t n, const double* E, int32_t ncell, double qm_dt, double kick, int32_t s_w,
                         const double* E0, double tau_over_dx, double qm_tau, int32_t s_p,
                         int64_t* sample_fx, uint32_t* status, void* stream);
PE_API int pe_quiet_start_f64(int32_t* cell, double* theta, double* v, double* w, int64_t n,
                              int32_t ncell, const double* prof_n, const double* prof_u, double v_th,
                              uint64_t seed, int32_t s_w, int64_t* rho_fx, uint32_t* status,
                              void* stream);

/* The initial nodal profiles of pe_load_initial, written to host arrays prof_n[ncell] and
 * prof_u[ncell] (FP32): PE_PROFILE_SINE, the ion-acoustic wave of Section 4.1,
 * n = 1 + amplitude cos(2 pi x_j / L), u = amplitude cos(2 pi x_j / L) at x_j = j L / ncell;
 * PE_PROFILE_SLAB, n = 1 on the nodes 7 ncell / 16 .. 9 ncell / 16 and 0 elsewhere, u = 0. */
PE_API int pe_initial_profile(int32_t profile, int32_t ncell, double L, double amplitude, float* prof_n,
                              float* prof_u);

PE_API int pe_fixed_point_shifts(int64_t nparticles, int32_t ncell, double w_cap, double v_cap,
                                 int32_t* s_w, int32_t* s_p);

/* Shift of the second-moment sample (pe_sample_args.s_e) for the same caps: the largest
 * |w V~^2| = w_cap v_cap^2 maps below 2^23 (w_cap, v_cap 0 = the defaults of
 * pe_fixed_point_shifts). */
PE_API int pe_second_moment_shift(int64_t nparticles, int32_t ncell, double w_cap, double v_cap, int32_t* s_e);

/* Ion pressure as an active variable (Section 3.2, EFREE: ion n, V and P = n T are active,
 * the ions shifted Maxwellians). pe_coarsen for samples of the three moments,
 * sample_fx int64[nsamples][3][ncell >> bin_shift] (density at 2^-(s_w+24), momentum at
 * 2^-(s_p+24), second moment at 2^-(s_e+24)): each row is analysed like pe_coarsen's (bin sums
 * over 2^bin_shift nodes with the Haar wavelet only) into coarse[nsamples][3][n_coarse]. */
PE_API int pe_coarsen_pressure(const int64_t* sample_fx, int32_t nsamples, int32_t ncell, int32_t s_w,
                               int32_t s_p, int32_t s_e, int32_t wavelet, int32_t n_coarse, int32_t bin_shift,
                               double* coarse, void* stream);

/* Lifting profiles of the three moments (Section 3.2 lifting, zero details): coarse[3][n_coarse]
 * is synthesised to the nodes as in pe_refine; n is clamped at 0 and rescaled to keep its sum,
 * u = nV / n and T = max(S / n - u^2, 0) where n > 1e-12 max n (u = T = 0 elsewhere). Writes
 * prof_n, prof_u, prof_T (float[ncell] each). ncell <= 4096 (four FP64 rows in shared memory). */
PE_API int pe_refine_pressure(const double* coarse, int32_t n_coarse, int32_t wavelet, int32_t ncell,
                              float* prof_n, float* prof_u, float* prof_T, void* stream);

/* pe_quiet_start at a local temperature: the same cells, offsets, weights, quantiles and
 * storage order, with V = u(X) + sqrt(T(X)) Phi^-1(b_h), T linear between the nodes like n and
 * u (prof_T >= 0; a uniform T = v_th^2 gives pe_quiet_start's particles). */
PE_API int pe_quiet_start_thermal(int32_t* cell, float* theta, float* v, float* w, int64_t n,
                                  int32_t ncell, const float* prof_n, const float* prof_u,
                                  const float* prof_T, uint64_t seed, int32_t s_w, int64_t* rho_fx,
                                  uint32_t* status, void* stream);

/* Quiet-start loading with equal weights on a bounded grid (Appendix C's loading, with the
 * particle count of each cell in proportion to its mass, as for Section 4.2's slab whose
 * vacuum cells hold no ions). The nodal density profile (prof_n, its wall nodes multiplied by
 * wall_factor: 1 when prof_n holds densities, 2 when it holds deposits) is linear inside each
 * of the ncell-1 cells between the walls: cell mass m_c = (n_c + n_{c+1}) / 2, cumulative mass
 * C_c = m_0 + ... + m_{c-1}, total M. Particle i (storage slot i) sits at the quantile
 * (i + 1/2) M / n of the cumulative mass: in the cell c with C_c <= (i + 1/2) M / n < C_{c+1},
 * at the offset t solving t + sigma (t^2 - t) = r, r the fraction of m_c below it and
 * sigma = (n_{c+1} - n_c) / (n_{c+1} + n_c). w = M / n for every particle;
 * V = u(X) + v_th Phi^-1(b_i) with b_i of pe_quiet_start. Storage: inside every full
 * aligned block of 4096 slots, slot s holds point i = s with its low 12 bits reversed (the
 * block's points, within 4096 mass quantiles of each other, in ascending velocity quantile:
 * co-moving targets then vary smoothly along the array); the ragged tail holds i = s. Cells
 * are non-decreasing from block to block.
 * scratch: PE_EQ_SCRATCH_BYTES(ncell) bytes of device memory, 16-byte aligned. A profile of
 * zero (or non-finite) mass sets PE_FLAG_RANGE and gives weight-0 particles in cell 0.
 * If rho_fx != NULL it is overwritten with the charge deposit of the new particles. */
#define PE_EQ_SCRATCH_BYTES(ncell) (16 * (size_t)(ncell) + 16)
PE_API int pe_quiet_start_equal(int32_t* cell, float* theta, float* v, float* w, int64_t n,
                                int32_t ncell, const float* prof_n, const float* prof_u,
                                float wall_factor, float v_th, uint64_t seed, int32_t s_w,
                                void* scratch, int64_t* rho_fx, uint32_t* status, void* stream);

/* Sort by cell (counting sort), used by the plain PIC path to keep the deposit's
 * per-block grids local. Reads (cell, theta, v, w), writes the permuted particles to
 * the out_* arrays (which must not alias the inputs). scratch: int32[2*ncell + 64].
 * The order of particles inside a cell is not specified; the multiset is exact. */
PE_API int pe_sort(const int32_t* cell, const float* theta, const float* v, const float* w,
                   int64_t n, int32_t ncell, int32_t* out_cell, float* out_theta, float* out_v,
                   float* out_w, int32_t* scratch, uint32_t* status, void* stream);

/* Allocation-free variant of pe_sort (the paper has no counterpart; this is a library
 * service). Some callers cannot allocate device memory at the point where they sort:
 * code running inside a host framework that owns all device allocations, real-time
 * loops that must not take cudaMalloc's implicit device synchronisation, or plugins
 * handed only the particle buffers. This entry point therefore takes no scratch
 * argument: its two counter arrays live in a statically sized device array of this
 * library (2 * PE_SORT_STATIC_MAX_CELLS + 64 int32, 66 KB), which every GPU that loads
 * the library keeps until the process exits. It calls no cudaMalloc, cudaFree or any
 * allocating routine.
 * - ncell must not exceed PE_SORT_STATIC_MAX_CELLS; larger grids return PE_EINVAL.
 * - Each call looks up the array's device address in the current context (no allocation),
 *   so it follows the device and context that are current when it is made; the first call
 *   in a process may load the library's device code, so make it before any stream capture.
 * - All calls share the one array (the counters are cleared at the start of each call):
 *   calls that may overlap on the GPU (different streams, or different threads without
 *   ordering) race and give wrong results. Serialise them.
 * Arguments and results are those of pe_sort. */
#define PE_SORT_STATIC_MAX_CELLS 8192
PE_API int pe_sort_noalloc(const int32_t* cell, const float* theta, const float* v, const float* w,
                           int64_t n, int32_t ncell, int32_t* out_cell, float* out_theta,
                           float* out_v, float* out_w, uint32_t* status, void* stream);

/* Diagnostics of a particle state (Section 4's conservation checks and the particle
 * CFL number). Velocities are taken at integer time, Vbar = v + (kick - 1/2) qm_dt E(X)
 * with E(X) the CIC gather of Ef (kick = 1/2 when v is already at integer time, 1 when
 * it is at half-integer time and Ef is the field of the current positions). Each
 * particle carries charge w dx. The electron free energy is sum (phi e^phi - e^phi + 1) dx
 * for PE_POISSON_BOLTZMANN and sum phi^2 dx / 2 for PE_POISSON_LINEARIZED: with the ion
 * kinetic and the field energy it makes the energy that the continuous ion /
 * Boltzmann-electron system conserves. phi and E (FP64 [ncell]) may be NULL (their
 * energies are then 0). A particle with cell outside [0, ncell), theta outside [0, 1] or
 * a non-finite v or w is counted in `invalid`, left out of every sum, and sets
 * PE_FLAG_RANGE. scratch: PE_MOMENTS_SCRATCH_BYTES of device memory (16-byte aligned);
 * out: one pe_moments in device memory, written on the stream. Floating-point sums use a
 * fixed partition for a given n, so repeated calls return identical bits. */
#define PE_MOMENTS_SCRATCH_BYTES 65536
typedef struct pe_moments {
    int64_t charge_fx;          /* sum_p rn(w 2^s_w) 2^24: equals the sum of the deposit (modulo 2^64:
                                   the total wraps beyond 2^63, e.g. 2^25 ions near the weight cap) */
    int64_t invalid;            /* particles left out (see above) */
    double charge_fixed_point;  /* charge_fx 2^-(s_w+24) dx */
    double charge;              /* sum w dx */
    double momentum;            /* sum w Vbar dx */
    double kinetic;             /* sum w Vbar^2 dx / 2 */
    double field_energy;        /* sum E_j^2 dx / 2 */
    double electron_energy;     /* see above */
    double total_energy;        /* kinetic + field + electron */
    double max_speed;           /* max |Vbar| */
    double cfl;                 /* max_speed dt / dx */
    int64_t charge_wq;          /* sum_p rn(w 2^s_w): the exact charge in weight units (no wrap up
                                   to 2^40 ions) */
} pe_moments;
PE_API int pe_compute_moments(const int32_t* cell, const float* theta, const float* v, const float* w, int64_t n,
                      const float* Ef, const double* phi, const double* E, int32_t ncell, double dx, double dt,
                      float qm_dt, float kick, int32_t s_w, int32_t mode, void* scratch, pe_moments* out,
                      uint32_t* status, void* stream);

/* Kinetic energy sum w Vbar^2 dx / 2 of one species (Vbar = v + (kick - 1/2) qm_dt E(X) at
 * integer time, E gathered from Ef), into out (device double): the global active variable of
 * Section 4.2 for the kinetic electrons. FP32 per-thread sums over a fixed grid-stride partition,
 * FP64 beyond (about 1e-6 relative; reproducible). scratch: device, double[1024]. An
 * out-of-range cell is skipped and sets PE_FLAG_RANGE. */
PE_API int pe_kinetic_energy(const int32_t* cell, const float* theta, const float* v, const float* w, int64_t n,
                             const float* Ef, int32_t ncell, double dx, float qm_dt, float kick, double* scratch,
                             double* out, uint32_t* status, void* stream);

/* Error measure of Section 4.1.1 between two coarse states (or any FP64 vectors):
 * out = sqrt( sum_i (a_i - b_i)^2 / sum_i (a_i^2 + b_i^2) ), 0 when both vanish. a, b, out
 * in device memory; one block, fixed summation order. */
PE_API int pe_rel_l2(const double* a, const double* b, int64_t n, double* out, void* stream);

/* ---- Phase-space coarse variable (Section 3.3 "A wavelet-based equation-free scheme",
 * Appendices B and C), Haar reading: the active variables are the masses H[i][j] of the
 * phase-space cells, coarse x-bin i of 2^b nodes times velocity cell j = [v_min + j dv,
 * v_min + (j+1) dv) (the Haar scaling coefficients of the histogram, up to one constant).
 * The co-moving sample is pe_push / pe_sample with pe_sample_args.n_v > 0. */

/* Fixed-point phase-space samples int64[nsamples][ncoef] -> FP64 masses (x 2^-(s_w+24))
 * into coarse[nsamples][ncoef]. */
PE_API int pe_ps_coarsen(const int64_t* sample_fx, int32_t nsamples, int64_t ncoef, int32_t s_w, double* coarse,
                         void* stream);

/* Projective step of the phase-space masses (Section 3.3, Eqs. extrapolation2 and
 * leastsquares) with the least-squares slope filtered before the leap: with filter bit 0 the
 * slope of every x-bin is smoothed along v by (1/4, 1/2, 1/4) (zero beyond the velocity range),
 * with bit 1 every velocity cell along x (periodic; with bit 2 as well, reflecting at the walls
 * of a bounded grid: the edge bin's slope stands in beyond it). The filter keeps the slope's sum (charge)
 * and, along v, its first moment (momentum); it damps the grid-scale structure of the slope,
 * which the leap multiplies by (dT - K dt) / (K dt / 2). samples[(K+1)][nxc][n_v]; work, out and
 * slope [nxc][n_v] (work: the unfiltered slope; slope: the filtered one; none may alias
 * samples or each other). filter = 0 gives pe_ls_project's result. */
PE_API int pe_ps_project(const double* samples, int32_t K, int32_t nxc, int32_t n_v, double dt, double dT,
                         int32_t filter, double* work, double* out, double* slope, void* stream);

/* Lifting tables of H[nxc][n_v] (FP64, device): mass[nxc] = sum_j H[i][j] with negative
 * masses clamped to 0 and the rest rescaled to keep the total (the clamp of Section 3.3's
 * remark on negative values); cdf[nxc][n_v + 1] the normalised CDF of each bin over its
 * velocity cells after the momentum-conserving reconstruction of Appendix C (edge
 * reconstruction below 0 and above 1, interior reconstruction from both ends, averaged;
 * where no admissible ramp exists the entry is clamped / filled by a running max and
 * flags[0] (device, may be NULL) is set to 1). Bins of non-positive raw mass get a uniform
 * CDF. FP64 without contraction, so mass and cdf equal a host evaluation of the same steps
 * bit for bit. table[nxc][3 n_v + 1] (FP32) is the sampling form used by pe_ps_quiet_start:
 * the CDF row, the inverse cell masses 1 / p_k (p_k = F[k+1] - F[k]; 0 for an empty cell),
 * and the cells' relative density slopes sigma_k = (p_{k+1} - p_{k-1}) / (4 p_k) clamped to
 * [-1, 1].
 * scratch: not used (may be NULL); the reconstruction works in shared memory. */
PE_API int pe_ps_lift_tables(const double* H, int32_t nxc, int32_t n_v, double* mass, double* cdf, float* table,
                             double* scratch, int32_t* flags, void* stream);

/* Particle loading of Appendix C on the tables: the Hammersley points, quantiles b and
 * storage order of pe_quiet_start. The lifted f(x, v) is linear in x between neighbouring
 * bin centres (Section 3.3's linear interpolation): with phi the particle's distance from the
 * centre of the bin b0 at or left of it, in bin widths, b1 = b0 + 1 (periodic),
 * w = ((1 - phi) mass[b0] + phi mass[b1]) 2^-b / ppc and V = (1 - phi) G_b0(b) + phi G_b1(b),
 * G the inverse of a bin's CDF: G(b) = v_min + dv (k + t), k the first index with
 * F[k+1] > b and t in [0, 1] where t + sigma_k (t^2 - t) = (b - F[k]) / p_k, i.e. the density
 * inside a velocity cell is linear, 1 + sigma_k (2t - 1), following its neighbours (uniform
 * cells would add dv^2/12 to the temperature at every lift). FP32 on the sampling table of
 * pe_ps_lift_tables. rho_fx (may be NULL) gets the
 * charge deposit. */
PE_API int pe_ps_quiet_start(int32_t* cell, float* theta, float* v, float* w, int64_t n, int32_t ncell,
                             int32_t bin_shift, const double* mass, const float* table, int32_t n_v, double v_min,
                             double dv, uint64_t seed, int32_t s_w, int64_t* rho_fx, uint32_t* status,
                             void* stream);

/* The phase-space loading on a bounded grid (walls at nodes 0 and ncell-1), with equal
 * weights placed by mass. Bin i sums the CIC charge of its 2^b nodes, x/dx in
 * [i 2^b - 1/2, (i+1) 2^b - 1/2) cut to the domain [0, ncell-1] (the first and last bins are
 * half a node narrower); the lifted density in x is linear between the bins' span midpoints,
 * with value mass_i / width_i there, and constant beyond the first and last midpoints. Its
 * nodal values are loaded by pe_quiet_start_equal's rule (positions by mass quantile, storage in
 * velocity-ordered blocks of 4096); every ion gets w = (sum of the bin masses) / n, so lifting
 * keeps the charge; V = (1 - f) G_b0(b) + f G_b1(b) blends the inverse CDFs of the two bins
 * whose midpoints bracket the ion, with b the ion's Hammersley quantile, G as in
 * pe_ps_quiet_start, and f = phi d1 / ((1 - phi) d0 + phi d1) bin b1's share of the density at
 * the ion (phi the fraction of the way from b0's midpoint, d the bin densities): a bin without
 * ions, next to the expansion front, then lends no velocities. scratch: PE_PS_EQ_SCRATCH_BYTES(ncell)
 * bytes of device memory, 16-byte aligned. */
#define PE_PS_EQ_SCRATCH_BYTES(ncell) (28 * (size_t)(ncell) + 64)
PE_API int pe_ps_quiet_start_equal(int32_t* cell, float* theta, float* v, float* w, int64_t n, int32_t ncell,
                                   int32_t bin_shift, const double* mass, const float* table, int32_t n_v,
                                   double v_min, double dv, uint64_t seed, int32_t s_w, void* scratch,
                                   int64_t* rho_fx, uint32_t* status, void* stream);

/* ---- Phase-space coarse variable, wavelet form: Section 3.3 as the paper states it. The
 * active variables are the coarse scaling coefficients C[i][m] of the phase-space histogram:
 * coarse node i (fine node i 2^b) of Eq. (restriction) applied b times in x, scaling
 * coefficient m of the periodized DWT in v (Appendix A) at n_vc of the n_vf fine velocity cells.
 * Restriction: pe_push / pe_sample with n_v = n_vf and x_tent = 1 (the hat rows), then
 * pe_ps_coarsen_v. Lifting: pe_ps_refine_v, pe_ps_lift_tables on the n_vf-cell rows (Appendix
 * C's reconstruction per coarse node, which the Appendix's Remark allows before the lift in
 * space), pe_ps_node_tables (Eq. interpolation to the fine nodes) and
 * pe_ps_quiet_start_nodes. */

/* Rows sample_fx[nrows][n_vf] (int64, fixed point with shift s_w, hat rows of pe_sample's
 * x_tent = 1 with bin_shift b) -> coarse[nrows][n_vc] (FP64): row values x 2^-(s_w + 24 + b)
 * (the averaged values of Eq. restriction), then L = log2(n_vf / n_vc) levels of the
 * periodized analysis filter of `wavelet` (PE_WAVELET_*) along v with the details discarded,
 * times 2^(L/2), so that a row's coefficients sum to its mass (Haar: sums of 2^L cells).
 * n_vf and n_vc powers of two, n_vc <= n_vf <= 4096. One block per row. */
PE_API int pe_ps_coarsen_v(const int64_t* sample_fx, int64_t nrows, int32_t n_vf, int32_t s_w, int32_t bin_shift,
                           int32_t wavelet, int32_t n_vc, double* coarse, void* stream);

/* The inverse of pe_ps_coarsen_v on its range: coarse[nrows][n_vc] -> hist[nrows][n_vf] by
 * L levels of periodized synthesis with zero details, times 2^(-L/2) (FP64, device). */
PE_API int pe_ps_refine_v(const double* coarse, int64_t nrows, int32_t n_vc, int32_t wavelet, int32_t n_vf,
                          double* hist, void* stream);

/* Eq. (interpolation) of the coarse-node tables of pe_ps_lift_tables (mass[nxc], cdf[nxc][n_v + 1],
 * FP64, device) to the ncell fine nodes: fine node j is phi = (j mod 2^b) / 2^b of the way from
 * coarse node i0 = j >> b to i1 = i0 + 1 (periodic, 2^b = ncell / nxc); its histogram is the
 * linear interpolation of the two coarse nodes' reconstructed histograms, so
 * node_dens[j] = (1 - phi) mass[i0] + phi mass[i1] and its CDF is the mixture
 * ((1 - phi) mass[i0] F_i0 + phi mass[i1] F_i1) / node_dens[j] (uniform if node_dens[j] <= 0).
 * node_table[ncell][3 n_v + 1] (FP32, evaluated in FP64) is the sampling row of
 * pe_ps_quiet_start with zero density slopes: the density is uniform inside a velocity cell
 * (Appendix C: the inverse by lookup and linear interpolation). */
PE_API int pe_ps_node_tables(const double* mass, const double* cdf, int32_t nxc, int32_t ncell, int32_t n_v,
                             float* node_table, float* node_dens, void* stream);

/* Appendix C loading of the wavelet form on the fine-node tables of pe_ps_node_tables: the
 * Hammersley points, quantiles b and storage order of pe_quiet_start; a particle in cell c at
 * offset theta gets w = ((1 - theta) node_dens[c] + theta node_dens[c+1]) / ppc and
 * V = (1 - theta) G_c(b) + theta G_{c+1}(b), G_j the inverse of node j's CDF (values linearly
 * interpolated between the two closest fine nodes). FP32. rho_fx (may be NULL) gets the charge
 * deposit. */
PE_API int pe_ps_quiet_start_nodes(int32_t* cell, float* theta, float* v, float* w, int64_t n, int32_t ncell,
                                   const float* node_table, const float* node_dens, int32_t n_v, double v_min,
                                   double dv, uint64_t seed, int32_t s_w, int64_t* rho_fx, uint32_t* status,
                                   void* stream);

/* =================================================================== context
 * One realisation of the projective-integration cycle (Section 3.1, Figure
 * efpicycle): lift -> N_e fine steps with restriction after each -> least-squares
 * slope -> forward-Euler leap of the coarse variables.
 */
typedef struct pe_config {
    int32_t ncell;        /* fine cells, power of two */
    int32_t n_coarse;     /* coarse coefficients per moment, power of two dividing ncell */
    int32_t wavelet;      /* PE_WAVELET_* */
    int32_t K;            /* burst length N_e (fine steps per macro step) */
    int64_t nparticles;   /* ppc * ncell */
    double L;             /* domain length */
    double dt;            /* fine step delta t */
    double dT;            /* macro step Delta t (>= K dt) */
    double qm;            /* ion charge-to-mass ratio */
    double v_th;          /* ion thermal speed used by lifting */
    int32_t comoving;     /* 1: restriction along approximate characteristics (App. B) */
    int32_t poisson;      /* PE_POISSON_* */
    double newton_tol;    /* max |Newton update| to stop (e.g. 1e-10) */
    int32_t newton_maxit; /* e.g. 30 */
    int32_t sort_every;   /* plain PIC: sort every this many steps (0 = never) */
    uint64_t seed;        /* lifting shift seeds: splitmix64(seed + macro step) */
    double w_cap;         /* largest particle weight (fixed-point range); 0 = 8 ncell / N */
    double v_cap;         /* largest |V~| in restriction samples; 0 = 32 */
    int32_t coarse_kind;  /* PE_COARSE_MOMENTS, PE_COARSE_PHASE_SPACE or PE_COARSE_MOMENTS_PRESSURE
                             (the last: periodic grids, Boltzmann electrons, ncell <= 4096; nodal
                             samples of three moments, lifting at the local temperature; the
                             coarse state is [3][n_coarse]) */
    int32_t n_v;          /* phase space: velocity cells (2..256) */
    double v_max;         /* phase space: velocity range [-v_max, v_max) */
    int32_t ps_filter;    /* phase space: 1-2-1 filter of the projected slope; bit 0 in v, bit 1 in x */
    int32_t boundary;     /* PE_BOUNDARY_*; absorbing grids lift with pe_quiet_start_equal
                             (moments) or pe_ps_quiet_start_equal (phase space) */
    int32_t electrons;    /* PE_ELECTRONS_*: Boltzmann fluid (0) or kinetic particles (1) */
    int32_t reset_every;  /* kinetic electrons, plain PIC: reload the electrons in Boltzmann
                             equilibrium with the ions every this many steps (0 = never) */
    double qm_e;          /* kinetic electrons: charge-to-mass ratio (0 = -1800, the paper's value) */
    double v_th_e;        /* kinetic electrons: thermal speed (0 = sqrt(-qm_e), i.e. T_e = 1) */
    int32_t n_v_coarse;   /* phase space: 0 = the Haar-bin form (n_coarse bins x n_v cells);
                             > 0 = the wavelet form of Section 3.3 (periodic, Boltzmann electrons,
                             ps_filter 0): hat rows at n_coarse nodes (Eq. restriction), n_v fine
                             velocity cells (power of two, <= 1024) reduced by the DWT of
                             `wavelet` to n_v_coarse coefficients (power of two, 2..n_v); the
                             coarse state is [n_coarse][n_v_coarse] */
    int32_t te_active;    /* kinetic electrons: 1 projects the electrons' total kinetic energy as a
                             global active variable (Section 4.2): sampled at every burst step,
                             least-squares leap, and each lift loads the Boltzmann electrons at
                             T_e / T_e0 = projected energy / energy at the initial load (their
                             Poisson-Boltzmann potential with n_e = exp(phi / T_e), thermal speed
                             v_th_e sqrt(T_e)); 0 keeps T_e = T_e0 */
} pe_config;

typedef struct pe_ctx pe_ctx;

/* Named regions of the caller-allocated device arena. */
enum pe_buffer {
    PE_BUF_PARTICLES_A = 0, /* cell i32[N] | theta f32[N] | v f32[N] | w f32[N] */
    PE_BUF_PARTICLES_B,     /* second bank (sort target) */
    PE_BUF_RHO,             /* int64[ncell] charge deposit */
    PE_BUF_PHI,             /* f64[ncell] potential (Newton warm start) */
    PE_BUF_E,               /* f64[ncell] field */
    PE_BUF_EF,              /* f32[ncell] field copy for the particle kernels */
    PE_BUF_E0F,             /* f32[ncell] field at burst start */
    PE_BUF_SAMPLES_FX,      /* int64[K+2][row] restriction samples (row: 2 bins, 3 ncell nodes with
                               the pressure, or n_coarse n_v) */
    PE_BUF_COARSE_SAMPLES,  /* f64[K+2][ncoef] */
    PE_BUF_COARSE,          /* f64[ncoef] current coarse state: [2][n_coarse], [3][n_coarse] (pressure)
                               or [n_coarse][n_v] */
    PE_BUF_SLOPE,           /* f64[ncoef] last least-squares slope */
    PE_BUF_PROFILE,         /* f32[2][ncell] lifting profiles (n, u); [3][ncell] (n, u, T) with the
                               pressure */
    PE_BUF_SORT,            /* int32[2 ncell + 64] sort scratch */
    PE_BUF_STATUS,          /* uint32[4] status word; int32[4] Newton diag after it */
    PE_BUF_DIAG,            /* pe_moments scratch + one pe_moments result */
    PE_BUF_SURROGATE,       /* f64[2][n_coarse] surrogate slope + gate result */
    PE_BUF_PHASE,           /* phase space: f64 bin masses, CDF tables, reconstruction scratch, flag;
                               absorbing grids: the equal-weight loading scratch */
    PE_BUF_ELECTRONS_A,     /* kinetic electrons: cell | theta | v | w, as the ion banks (else empty) */
    PE_BUF_ELECTRONS_B,     /* kinetic electrons: second bank (sort target) */
    PE_BUF_RHO_E,           /* kinetic electrons: int64[ncell] electron deposit, then int64[2][ncell]
                               ion moments for the electrons' drift */
    PE_NBUF
};

typedef struct pe_layout {
    size_t total_bytes;     /* size of the arena the caller must allocate */
    size_t offset[PE_NBUF]; /* 256-byte aligned offsets into the arena */
    size_t bytes[PE_NBUF];
} pe_layout;

typedef struct pe_diag {
    int64_t macro_steps;    /* completed projective steps */
    int64_t fine_steps;     /* fine PIC steps run (bursts + plain PIC) */
    double time;            /* simulated time */
    int32_t particle_bank;  /* 0 or 1: which PE_BUF_PARTICLES_* holds the particles */
    int32_t v_at_integer;   /* 1 if stored v is at integer time (after load/lift) */
    int32_t s_w, s_p;       /* fixed-point shifts in use */
    int32_t newton_iters;   /* iterations of the last field solve (after sync) */
    uint32_t status;        /* device status word (after sync) */
    int32_t electron_bank;  /* kinetic electrons: which PE_BUF_ELECTRONS_* holds them */
    int32_t e_v_at_integer; /* kinetic electrons: 1 if their stored v is at integer time */
    double T_e;             /* kinetic electrons: T_e / T_e0 of the last lift (1 unless te_active) */
    double W_e;             /* te_active: the electrons' projected kinetic energy of the last leap */
} pe_diag;

/* Validates cfg and fills the arena layout. PE_EINVAL on a bad configuration. */
PE_API int pe_layout_for(const pe_config* cfg, pe_layout* out);

/* Binds a context to a caller-allocated device arena of at least
 * layout.total_bytes (256-byte aligned) and a stream. No device allocation.
 * The context (host memory) is owned by the library: free it with pe_destroy. */
PE_API int pe_create(const pe_config* cfg, void* arena, size_t arena_bytes, void* stream,
                     pe_ctx** out);
PE_API void pe_destroy(pe_ctx* ctx);

/* Initial state at t = 0 from an analytic nodal profile (PE_PROFILE_SINE with the
 * given amplitude, or PE_PROFILE_SLAB, amplitude unused) by the quiet start (periodic grids:
 * pe_quiet_start; absorbing grids: pe_quiet_start_equal); also computes the initial coarse
 * state. Kinetic electrons start in Boltzmann equilibrium with these ions. */
PE_API int pe_load_initial(pe_ctx* ctx, int32_t profile, double amplitude);

/* Micro-scale evolution (Section 3.1): K fine steps from the current particles with
 * the co-moving restriction sample of each of the K+1 instants (Appendix B). With kinetic
 * electrons every fine step pushes both species in the field of the net charge; the
 * samples are the ions'. */
PE_API int pe_burst(pe_ctx* ctx);
/* Coarsening of the K+1 samples (pe_coarsen into PE_BUF_COARSE_SAMPLES). */
PE_API int pe_restrict(pe_ctx* ctx);
/* Least-squares slope and forward-Euler leap to t + Delta t (pe_ls_project). */
PE_API int pe_project(pe_ctx* ctx);
/* Lifting (Section 3.3 + Appendix C): coarse state -> profiles -> quiet start; kinetic
 * electrons are then placed in Boltzmann equilibrium with the lifted ions. */
PE_API int pe_lift(pe_ctx* ctx);
/* One projective macro step: lift (unless the particles are fresh), burst,
 * restrict, project. Advances time by Delta t. */
PE_API int pe_step(pe_ctx* ctx);
/* Plain (resolved) PIC: nsteps leapfrog steps with deposit + Newton each step (kinetic
 * electrons: both species, Poisson field), sorting every sort_every steps; with kinetic
 * electrons and reset_every > 0 the electrons are reloaded in Boltzmann equilibrium with the
 * ions every reset_every steps (Section 4.1's reset runs). Advances time by nsteps dt. */
PE_API int pe_pic_steps(pe_ctx* ctx, int32_t nsteps);
/* Coarse state of the current particles (restriction at integer time, no frame
 * shift) into host or device memory out[2][n_coarse]. */
PE_API int pe_measure(pe_ctx* ctx, double* out, int32_t out_on_device);

/* Least-squares slope (f64[2][n_coarse]) of the last macro step (or the accepted surrogate
 * slope), into host or device memory. */
PE_API int pe_get_slope(pe_ctx* ctx, double* out, int32_t out_on_device);
/* Copy the coarse state (f64[2][n_coarse]) out of / into the context. */
PE_API int pe_get_coarse(pe_ctx* ctx, double* out, int32_t out_on_device);
PE_API int pe_set_coarse(pe_ctx* ctx, const double* in, int32_t in_on_device);

/* Checkpoint and resume between macro steps. Projective integration's state is the coarse
 * state: with the clock (macro and fine step counts, time, the next Delta t), which seeds the
 * next lifting, and the potential that starts its first Newton solve, it determines every later
 * step, so a context restored from a checkpoint continues bit for bit as the original would.
 * Valid after a projection (the next step lifts; a context whose particles are current, just
 * loaded or advanced by plain PIC, returns PE_ESTATE). pe_checkpoint_bytes gives the size of
 * the host buffer; the image holds a header (with the context's pe_config: a restore into a
 * context of another configuration, seed included, returns PE_EINVAL), the coarse state, the
 * last slope and phi with its Newton history. Synchronises. */
PE_API int pe_checkpoint_bytes(const pe_ctx* ctx, size_t* bytes);
PE_API int pe_checkpoint_save(pe_ctx* ctx, void* host_buf, size_t bytes);
PE_API int pe_checkpoint_restore(pe_ctx* ctx, const void* host_buf, size_t bytes);

/* Synchronises the context's stream and returns PE_OK or the first device fault
 * (PE_ETIMEOUT, PE_ERANGE, PE_EOVERFLOW, PE_ENOCONV); clears the status word. */
PE_API int pe_sync_status(pe_ctx* ctx);
/* Conserved quantities of the current particles at the current time (pe_compute_moments
 * with the field of the current positions; deposits and solves it first, which also
 * refreshes the Newton warm start, as pe_measure does). With kinetic electrons the charge
 * entries are the ions', electron_energy is the electrons' kinetic energy (mass w / |q_e/m_e|
 * per unit weight), momentum and the speed and CFL maxima cover both species, and
 * total_energy = ion kinetic + field + electron kinetic energy, what the two-species system
 * conserves. out: host (synchronises) or device memory. */
PE_API int pe_state_moments(pe_ctx* ctx, pe_moments* out, int32_t out_on_device);
/* Host-side counters (no synchronisation except for newton_iters/status, which are
 * read after a stream synchronise). */
PE_API int pe_diagnostics(pe_ctx* ctx, pe_diag* out);

/* Kernel timing for measurement: while enabled, the context records a pair of CUDA
 * events on its stream around every particle-kernel launch and every field solve it
 * issues, pooled by launch kind:
 *   PE_PROF_PUSH_SAMPLE     fused push + deposit + moment restriction sample (a burst step)
 *   PE_PROF_PUSH            push + deposit without a sample (plain PIC, kinetic electrons)
 *   PE_PROF_SAMPLE          restriction sample alone (the last sample of a burst)
 *   PE_PROF_DEPOSIT         charge deposit alone
 *   PE_PROF_LOAD            quiet-start loading and lifting (deposit fused)
 *   PE_PROF_PUSH_SAMPLE_PS  fused push + deposit + phase-space restriction sample
 *   PE_PROF_FIELD           field solve (Newton, or the kinetic-electron Poisson solve)
 * pe_profile_read synchronises, returns the summed elapsed milliseconds and launch counts
 * since the last read (push_* = every kind but PE_PROF_FIELD, field_* = PE_PROF_FIELD) and
 * resets them. pe_profile_read_kinds returns the same per kind (ms[PE_PROF_NKINDS],
 * launches[PE_PROF_NKINDS], host arrays) and resets them. Events are host resources created
 * on first use. pe_profile(ctx, 1) times every kind; pe_profile_mask(ctx, kinds) only the
 * kinds whose bit (1 << PE_PROF_*) is set (0 turns timing off; PE_EINVAL for unknown bits):
 * each event pair costs a few microseconds of stream time, so a measurement of whole steps
 * times only the kernels it reports. */
enum {
    PE_PROF_PUSH_SAMPLE = 0,
    PE_PROF_PUSH = 1,
    PE_PROF_SAMPLE = 2,
    PE_PROF_DEPOSIT = 3,
    PE_PROF_LOAD = 4,
    PE_PROF_PUSH_SAMPLE_PS = 5,
    PE_PROF_FIELD = 6,
    PE_PROF_NKINDS = 7
};
PE_API int pe_profile(pe_ctx* ctx, int32_t enable);
PE_API int pe_profile_mask(pe_ctx* ctx, int32_t kinds);
PE_API int pe_profile_read(pe_ctx* ctx, double* push_ms, int64_t* push_launches, double* field_ms,
                           int64_t* field_launches);
PE_API int pe_profile_read_kinds(pe_ctx* ctx, double* ms, int64_t* launches);

/* =================================================================== tensor-core GEMM
 * C[M][N] (FP32, row stride ldc) = A[M][K] B[N][K]^T for BF16 A and B stored with K contiguous
 * (row strides lda, ldb elements; 16-byte aligned bases, lda and ldb multiples of 8): tcgen05.mma
 * with the accumulator in tensor memory, operands staged by TMA in the 128-byte swizzle layout,
 * tiles of 128 x 128 (N % 128 == 0) or 128 x 64 (N % 64 == 0), four stages of K = 64; M and K
 * may be ragged (zero fill). The GEMM engine of the surrogate's training and inference. A
 * device-side wait that exceeds its budget sets PE_FLAG_TIMEOUT in status[0] (device) and
 * skips the product. */
PE_API int pe_tc_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int32_t M,
                           int32_t N, int32_t K, uint32_t* status, void* stream);

/* =================================================================== batch
 * Ensemble of independent realisations advanced together (the same burst length, fine
 * and macro steps; any grid of at least 64 cells, any particle count, Haar wavelet, moment
 * coarse variables and Boltzmann electrons: other contexts make it PE_EINVAL).
 * Each fine step of the whole ensemble is one persistent particle launch over a shared
 * work list of particle chunks plus one launch of field-solve clusters (one per
 * realisation); from the second pe_batch_step on, the burst, restriction and
 * projection of every realisation replay as one captured CUDA graph. Lifting takes one
 * launch for every realisation's profile and one loading launch per realisation. Each
 * context keeps its own arena; the batch needs caller-owned
 * device scratch of pe_batch_scratch_bytes (256-byte aligned) for its descriptors, work
 * list and the ensemble's charge, field-copy and sample grids. Each realisation follows
 * pe_step on its context alone: the same particle arithmetic; its field solve may partition
 * the linear solve differently (ensembles use fewer SMs per solve), so states agree to the
 * Newton tolerance rather than bit for bit. The batch's stream waits for work
 * queued on each context's stream, and each context's stream waits for the batch. Graph
 * capture needs a created stream: on the legacy default stream every step runs eagerly. */
typedef struct pe_batch pe_batch;
PE_API int pe_batch_scratch_bytes(pe_ctx* const* ctxs, int32_t n, size_t* bytes);
PE_API int pe_batch_create(pe_ctx* const* ctxs, int32_t n, void* scratch, size_t scratch_bytes, void* stream,
                           pe_batch** out);
/* One projective macro step of every realisation (all must have been loaded, or all
 * advanced by the batch: PE_ESTATE otherwise). */
PE_API int pe_batch_step(pe_batch* b);
/* Autotuner: times the batched particle pass for every launch shape (particle chunks of
 * 16384, 32768 or 65536 per work item; blocks of 128, 256 or 512 threads; the charge deposit
 * through a shared-memory window or straight to the global grid): the burst's fused pass (push,
 * deposit, binned sample) run with a frozen step (dt/dx = 0, kick 0), which rewrites every
 * particle unchanged and leaves its deposit in the batch's charge grid (the current particles'
 * deposit) and its sample in a row that each burst clears; it keeps the fastest and returns its
 * chunk in *chunk. The
 * choice is cached for the process by the ensemble's composition (every realisation's ncell and
 * particle count, in order, and the device): a later batch of the same composition reuses it
 * without timing. pe_batch_tuned reports the shape in use. */
PE_API int pe_batch_tune(pe_batch* b, int64_t* chunk);
PE_API int pe_batch_tuned(const pe_batch* b, int64_t* chunk, int32_t* block, int32_t* privatised);
/* Mean of the coarse states (Section 3.3's coarse density and momentum coefficients) of a group
 * of realisations of the batch: members[nmembers] (1 <= nmembers <= 128) index the contexts
 * given to pe_batch_create, all with the same n_coarse; out (device, double[2 n_coarse]) gets
 * the component-wise mean, summed in the order given (repeatable bits), on the batch stream. */
PE_API int pe_batch_group_mean(pe_batch* b, const int32_t* members, int32_t nmembers, double* out);
PE_API void pe_batch_destroy(pe_batch* b);

/* =================================================================== learned surrogate
 * A multilayer perceptron that predicts the least-squares slope of the coarse variables
 * (Section 3.3, Eq. (leastsquares)) from the coarse state at the start of a burst, so that
 * a gated macro step (pe_step_surrogate) can replace most of the resolved burst. Linear
 * layers W_l [d_{l+1}][d_l] with bias, GELU (erf form, GELU(z) = z Phi(z)) after every
 * layer but the last. Inputs and targets are z-scored per component (pe_mlp_fit_norm).
 * Arithmetic: BF16 weights and activations on the tensor cores with FP32 accumulation,
 * FP32 bias, activation, loss and Adam state (master weights FP32, mirrored to BF16 after
 * every update). Training: mean squared error of the normalised outputs, Adam with bias
 * correction. All dims must be multiples of 64 (64..4096); training batches a multiple of
 * 32. Like the context API, the network lives in a caller-owned device arena (no
 * allocation) and runs on the stream given at creation. */
#define PE_MLP_MAX_LAYERS 8
enum pe_mlp_buffer {
    PE_MLP_PARAMS = 0,  /* f32[nparams]: W_1, b_1, W_2, b_2, ... (flat) */
    PE_MLP_PARAMS_BF16, /* bf16 mirror of the parameters [nparams], then its per-layer transposes
                           (W_l^T [d_l][d_{l+1}] at W_l's offset + nparams; the data-gradient
                           GEMMs read them with K contiguous) */
    PE_MLP_GRADS,       /* f32[nparams] gradients of the last pe_mlp_grad / training step */
    PE_MLP_ADAM_M,      /* f32[nparams] first moments */
    PE_MLP_ADAM_V,      /* f32[nparams] second moments */
    PE_MLP_NORM,        /* f32[4][dmax] mu_in, sd_in, mu_out, sd_out; statistics scratch; step, loss */
    PE_MLP_WORK,        /* batch workspace for max_batch rows: activations and gradients, and their
                           transposes (the weight-gradient GEMMs contract over the batch) */
    PE_MLP_NBUF
};
typedef struct pe_mlp_layout {
    size_t total_bytes;
    size_t offset[PE_MLP_NBUF];
    size_t bytes[PE_MLP_NBUF];
    int64_t nparams;
} pe_mlp_layout;
typedef struct pe_mlp pe_mlp;
/* dims[0..nlayers]: widths (input, hidden..., output); max_batch: largest batch. */
PE_API int pe_mlp_layout_for(int32_t nlayers, const int32_t* dims, int32_t max_batch, pe_mlp_layout* out);
PE_API int pe_mlp_create(int32_t nlayers, const int32_t* dims, int32_t max_batch, void* arena, size_t arena_bytes,
                         void* stream, pe_mlp** out);
PE_API void pe_mlp_destroy(pe_mlp* net);
/* Weights W = (2u - 1) a from the splitmix64 sequence of seed (u = (s_i >> 40) 2^-24, i the
 * flat parameter index), a = sqrt(6 / d_in) (hidden) or sqrt(3 / d_in) (last layer);
 * biases, Adam moments and the step counter 0; identity normalisation. Synchronises. */
PE_API int pe_mlp_init(pe_mlp* net, uint64_t seed);
/* z-score statistics of the training set X [npairs][d_0], Y [npairs][d_L] (FP32, device):
 * population mean and deviation per component, deviations floored at 1e-6 of their
 * largest; with period P > 0 the statistics are pooled over each block of P consecutive
 * components (for data that is augmented by circular shifts within such blocks). */
PE_API int pe_mlp_fit_norm(pe_mlp* net, const float* X, const float* Y, int64_t npairs, int32_t period);
/* Inference: y = net(x) for B rows (1 <= B <= max_batch): x raw [B][d_0] (FP32, or FP64 if
 * x_is_f64), normalised inside; y de-normalised [B][d_L] (FP32 or FP64). Device pointers. */
PE_API int pe_mlp_forward(pe_mlp* net, const void* x, int32_t x_is_f64, int32_t B, void* y, int32_t y_is_f64);
/* Gradients of the MSE loss over the batch rows[0..B) of (X, Y) (rows NULL: rows 0..B-1)
 * into PE_MLP_GRADS; loss (device f32, may be NULL) gets the loss. No update. */
PE_API int pe_mlp_grad(pe_mlp* net, const float* X, const float* Y, int64_t npairs, const int32_t* rows, int32_t B,
                       float* loss);
/* One Adam update from PE_MLP_GRADS (step counter on the device, advanced by one). */
PE_API int pe_mlp_adam(pe_mlp* net, double lr, double beta1, double beta2, double eps);
/* nsteps training steps: each draws B rows of (X, Y) and, with shift_period P > 0, one
 * circular shift per row inside every block of P components (the same for input and
 * target), from the splitmix64 sequence of (seed, step); gradients; Adam (0.9, 0.999, 1e-8).
 * The step is captured once as a CUDA graph and replayed (eagerly on the legacy default
 * stream). loss (device f32, may be NULL) gets the last step's loss. */
PE_API int pe_mlp_train(pe_mlp* net, const float* X, const float* Y, int64_t npairs, int32_t B, int32_t shift_period,
                        uint64_t seed, int32_t nsteps, float lr, float* loss);
/* Loads the FP32 parameter vector params[nparams] (device; layout of PE_MLP_PARAMS) and
 * rewrites the BF16 mirror. */
PE_API int pe_mlp_set_params(pe_mlp* net, const float* params);
/* Parameter count and device addresses of the step counter, parameters and gradients. */
PE_API int pe_mlp_info(const pe_mlp* net, int64_t* nparams, int64_t* steps_device_ptr, void** params, void** grads);
/* Every product of the network (forward, data and weight gradients) runs on the tensor-core
 * GEMM of pe_tc_gemm_bf16 with the bias, GELU, loss or GELU' factor fused into its epilogue.
 * pe_mlp_sync_status synchronises the network's stream, reads and clears its device status
 * word: PE_ETIMEOUT if a GEMM's bounded wait expired since the last call (its product was
 * skipped), else PE_OK. */
PE_API int pe_mlp_sync_status(pe_mlp* net);

/* Gated surrogate macro step (the a-posteriori check of the learned slope). From the coarse
 * state c at the start of the step: s_mlp = net(c); lift (unless fresh); a probe burst of
 * K_probe fine steps with co-moving samples c_0..c_Kp; probe slope s_p and its standard
 * error sigma_i (from the residuals of the line fit; K_probe >= 2). The estimated error of
 * the step is the relative change the slope difference makes to the projected state,
 * e = leap ||s_mlp - s_p|| / ||c_Kp|| with leap = Delta t - K_probe delta t; the prediction
 * is accepted when e <= max(tol, noise_sigmas leap ||sigma|| / ||c_Kp||): then
 * c <- c_Kp + leap s_mlp. Otherwise the burst continues to K steps and the step ends as
 * pe_step does (the probe is the burst's first K_probe steps, so nothing is recomputed).
 * The network must map 2 n_coarse inputs to 2 n_coarse outputs; it runs on the context's
 * stream. Synchronises once (the decision). */
typedef struct pe_gate_cfg {
    int32_t K_probe;     /* probe burst length, 2 <= K_probe < K */
    double tol;          /* tolerance on the estimated relative state error, e.g. 1e-3 */
    double noise_sigmas; /* multiple of the probe slope's standard error, e.g. 3 */
} pe_gate_cfg;
typedef struct pe_gate_stats {
    int32_t accepted;   /* 1 if the surrogate slope was used */
    int32_t fine_steps; /* fine steps run in this macro step */
    double err;         /* estimated relative state error e */
    double floor;       /* max(tol, noise floor) */
    double norm;        /* ||s_p|| */
    double sigma;       /* ||sigma|| */
} pe_gate_stats;
PE_API int pe_step_surrogate(pe_ctx* ctx, pe_mlp* net, const pe_gate_cfg* gate, pe_gate_stats* out);
/* The gate of pe_step_surrogate on its own: probe samples[(K_probe+1)][ncoef] at t_p = p dt,
 * slope s_p_i = sum_p (t_p - tbar)(c_p,i - cbar_i) / sum_p (t_p - tbar)^2, standard error
 * sigma_i^2 = sum_p r_p,i^2 / (K_probe - 1) / sum_p (t_p - tbar)^2 (r the fit residuals);
 * decision as above (result: err = e, floor, norm = ||s_p||, sigma = ||sigma||); on acceptance
 * coarse <- c_{K_probe} + (dT - K_probe dt) s_mlp and slope <- s_mlp (both [ncoef], untouched
 * otherwise). result: one pe_gate_result in device memory. One block, fixed summation order. */
typedef struct pe_gate_result {
    double err, floor, norm, sigma;
    int32_t accepted, pad;
} pe_gate_result;
PE_API int pe_gate(const double* samples, int32_t K_probe, int32_t ncoef, double dt, double dT, const double* s_mlp,
                   double tol, double noise_sigmas, double* coarse, double* slope, pe_gate_result* result,
                   void* stream);
/* =================================================================== adaptive macro step
 * The paper keeps Delta t fixed and names error estimators that adapt the projective time
 * step as the goal (Section 3.1's remark); this is one such estimator and controller.
 *
 * pe_leap_curvature: per coarse component i the quadratic least-squares coefficient q_i of
 * a burst's samples[(K+1)][ncoef] at t_p = p dt (c ~ a + b t + q t^2) and its sampling
 * variance var_i (the fit's residual variance, K - 2 degrees of freedom, over the sum of the
 * squared quadratic basis); out[0] = sqrt(max(0, ||q||^2 - sum var_i)), the curvature with the
 * particle noise's bias removed, out[1] = ||c_K||_2, out[2] = sqrt(sum var_i), out[3] =
 * sqrt(sum s_i^2 / sum_p (t_p - tbar)^2) the norm of the least-squares slopes' standard errors
 * (s_i^2 the same residual variance) (device, double[4]). On a quadratic trajectory the
 * least-squares slope is the derivative at the burst's midpoint, so the forward-Euler leap of
 * length L from c_K errs by exactly q L (L + K dt): e(L) = out[0] L (L + K dt) / out[1]
 * estimates the relative error of a leap, and L out[3] / out[1] the part the slope's noise
 * adds. K >= 2 (K = 2 leaves no residual: no noise terms). scratch: device, double[4 * 1024]
 * (per-block partial sums). Every sum in a fixed order: repeated calls give identical bits. */
PE_API int pe_leap_curvature(const double* samples, int32_t K, int32_t ncoef, double dt, double* scratch,
                             double* out, void* stream);

/* pe_step_adaptive: one macro step whose Delta t is a whole number M of bursts, M K dt, chosen
 * from the estimate e of the previous step: lift (unless fresh), burst and restriction with
 * the current Delta t (the co-moving frame depends on it, so it is fixed before the burst),
 * then e(L) with L = Delta t - K dt. If e > tol and M > M_min the burst is rejected: the
 * coarse state is lifted again (same seed) and the step rerun with the M of the tolerance
 * (at most M - 1). Otherwise the step is projected, and the next step takes
 * M = floor((K dt + safety L_tol) / (K dt)) bursts, L_tol the leap with e(L_tol) = tol,
 * clamped to [M_min, min(M_max, floor(grow M))]. Synchronises once per burst (the decision).
 * Adaptive burst length (K_max > 0): the burst length K itself (at most the configured K,
 * which sizes the sample buffers) is chosen for the next step as the smallest K' in
 * [K_min, K_max] whose slope noise, scaled from the measured out[3] at K by the least-squares
 * law var ~ 1 / (K (K+1) (K+2)), moves the leap just taken by at most noise_frac tol relative to
 * ||c_K||; the next Delta t is then M' K' dt with M' from the curvature rule in units of K' dt.
 * K_max = 0 keeps the burst length. */
typedef struct pe_adapt_cfg {
    double tol;      /* bound on the estimated relative error of one leap, e.g. 1e-4 */
    int32_t M_min;   /* smallest macro step in bursts (>= 1; 1 means no leap) */
    int32_t M_max;   /* largest macro step in bursts */
    double safety;   /* fraction of L_tol taken for the next step, in (0, 1] */
    double grow;     /* the next M is at most grow times the current one (>= 1) */
    int32_t K_min;   /* adaptive burst length: shortest burst (>= 3) */
    int32_t K_max;   /* adaptive burst length: longest burst (<= the configured K); 0: fixed K */
    double noise_frac; /* share of tol granted to the slope noise (in (0, 1]; 0 means 0.5) */
} pe_adapt_cfg;
typedef struct pe_adapt_stats {
    double dT;        /* the macro step taken */
    double err;       /* its estimated relative leap error */
    double dT_next;   /* the next macro step */
    int32_t rejected; /* bursts rejected and rerun in this step */
    int32_t fine_steps; /* fine steps run in this step */
    double noise;     /* the slope noise's estimated relative effect on the leap taken */
    int32_t K;        /* the burst length of this step */
    int32_t K_next;   /* the burst length of the next step */
} pe_adapt_stats;
PE_API int pe_step_adaptive(pe_ctx* ctx, const pe_adapt_cfg* cfg, pe_adapt_stats* out);
/* Delta t of the next macro steps (>= K dt, K the current burst length); the configured dT until
 * set. Bursts, projections, pe_step and pe_step_surrogate use it; a batch refuses contexts whose
 * Delta t or burst length was changed. */
PE_API int pe_set_macro_step(pe_ctx* ctx, double dT);

/* FP32 copy of the coarse state (what = 0) or of the last slope (what = 1) into out[2 n_coarse]
 * (device), e.g. one row of a surrogate training set. */
PE_API int pe_export_f32(pe_ctx* ctx, int32_t what, float* out);

/* Number of kernels this library has launched in the process so far. */
PE_API int64_t pe_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* PEPIC_H */
