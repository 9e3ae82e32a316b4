// Coarse-variable kernels (FP64): restriction of the fine moment samples to wavelet
// scaling coefficients, the least-squares projective leap, and the lifting profile.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "pe_common.cuh"
#include "pe_internal.h"

namespace pe {

// Orthonormal scaling filter (sum h = sqrt 2); the wavelet filter is
// g_m = (-1)^m h_{len-1-m} and is not needed: details are discarded.
struct Filter {
    double h[12];
    int len;
};

// Order-4 coiflet (Appendix A: the wavelet has four vanishing moments and the scaling
// function vanishing moments 1..3), taps h_k for k = -4..7 stored from k = -4. Its taps are
// the solution of 14 equations in 12 unknowns:
//   sum h_k = sqrt 2;  sum k^p h_k = 0 (p = 1..3);  sum (-1)^k k^p h_k = 0 (p = 0..3);
//   sum_k h_k h_{k+2m} = delta_m (m = 0..5),
// solved here on the host by Gauss-Newton on the normal equations (analytic Jacobian). The
// system has a few real solutions; the coiflet is the one concentrated at k = 0 (largest
// central tap h_0), Daubechies' choice. Which root a Newton path reaches depends on rounding
// (fused multiply-adds differ between hosts), so several starts are tried and the converged
// solution with the largest h_0 is kept.
static void coif4_residual(const double* h, double* r, double J[14][12])
{
    int e = 0;
    double s = 0.0;
    for (int i = 0; i < 12; ++i) s += h[i];
    r[e] = s - sqrt(2.0);
    for (int i = 0; i < 12; ++i) J[e][i] = 1.0;
    ++e;
    for (int p = 1; p <= 3; ++p, ++e) {
        r[e] = 0.0;
        for (int i = 0; i < 12; ++i) {
            const double k = i - 4, kp = pow(k, p);
            r[e] += kp * h[i];
            J[e][i] = kp;
        }
    }
    for (int p = 0; p <= 3; ++p, ++e) {
        r[e] = 0.0;
        for (int i = 0; i < 12; ++i) {
            const double k = i - 4, sg = ((i - 4) & 1) ? -1.0 : 1.0, kp = sg * (p ? pow(k, p) : 1.0);
            r[e] += kp * h[i];
            J[e][i] = kp;
        }
    }
    for (int m = 0; m < 6; ++m, ++e) {
        r[e] = (m == 0) ? -1.0 : 0.0;
        for (int i = 0; i < 12; ++i) J[e][i] = 0.0;
        for (int i = 0; i + 2 * m < 12; ++i) {
            r[e] += h[i] * h[i + 2 * m];
            J[e][i] += h[i + 2 * m];
            J[e][i + 2 * m] += h[i];
        }
    }
}

// Levenberg-Marquardt iteration on the normal equations from h; true if it converges to a
// root (max residual below 1e-13).
static bool coif4_newton(double* h)
{
    double r[14], J[14][12], mu = 1e-3;
    for (int it = 0; it < 400; ++it) {
        coif4_residual(h, r, J);
        double nr = 0.0, n0 = 0.0;
        for (int e = 0; e < 14; ++e) {
            nr = fmax(nr, fabs(r[e]));
            n0 += r[e] * r[e];
        }
        if (nr < 1e-15) return true;
        double A[12][13];
        for (int i = 0; i < 12; ++i) {
            for (int j = 0; j < 12; ++j) {
                double a = 0.0;
                for (int e = 0; e < 14; ++e) a += J[e][i] * J[e][j];
                A[i][j] = a + (i == j ? mu : 0.0);
            }
            double c = 0.0;
            for (int e = 0; e < 14; ++e) c -= J[e][i] * r[e];
            A[i][12] = c;
        }
        for (int c = 0; c < 12; ++c) {  // Gaussian elimination with partial pivoting
            int piv = c;
            for (int i = c + 1; i < 12; ++i)
                if (fabs(A[i][c]) > fabs(A[piv][c])) piv = i;
            if (fabs(A[piv][c]) < 1e-300) return false;
            for (int j = 0; j <= 12; ++j) {
                const double t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
            for (int i = c + 1; i < 12; ++i) {
                const double f = A[i][c] / A[c][c];
                for (int j = c; j <= 12; ++j) A[i][j] -= f * A[c][j];
            }
        }
        double d[12], hn[12], rn[14], Jn[14][12];
        for (int i = 11; i >= 0; --i) {
            double v = A[i][12];
            for (int j = i + 1; j < 12; ++j) v -= A[i][j] * d[j];
            d[i] = v / A[i][i];
        }
        for (int i = 0; i < 12; ++i) hn[i] = h[i] + d[i];
        coif4_residual(hn, rn, Jn);
        double nn = 0.0;
        for (int e = 0; e < 14; ++e) nn += rn[e] * rn[e];
        if (nn < n0) {  // accept, trust the quadratic model more
            for (int i = 0; i < 12; ++i) h[i] = hn[i];
            mu = fmax(mu * 0.1, 1e-15);
        } else {
            mu *= 10.0;
            if (mu > 1e10) break;
        }
    }
    coif4_residual(h, r, J);
    double nr = 0.0;
    for (int e = 0; e < 14; ++e) nr = fmax(nr, fabs(r[e]));
    return nr < 1e-13;
}

static bool coif4_solve(double* best)
{
    // starts: filters centred on k = 0 (B-spline hat, delta, Haar pair, shifted hats), then
    // pseudo-random ones (splitmix64); the root with the largest central tap is kept
    const double r2 = sqrt(2.0);
    const double centred[5][3] = {{0.5, 1.0, 0.5}, {0.0, 2.0, 0.0}, {0.0, 1.0, 1.0}, {1.0, 0.5, 0.0}, {0.0, 0.5, 1.0}};
    bool found = false;
    uint64_t z = 0x5EEDC01F;
    for (int s = 0; s < 64; ++s) {
        double h[12] = {0.0};
        if (s < 5) {
            for (int j = 0; j < 3; ++j) h[3 + j] = centred[s][j] / r2;
        } else {
            for (int i = 0; i < 12; ++i) {
                z += 0x9E3779B97F4A7C15ULL;
                uint64_t x = z;
                x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
                x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
                x ^= x >> 31;
                h[i] = ((double)(x >> 11) * 0x1.0p-53 - 0.5);
            }
        }
        if (!coif4_newton(h)) continue;
        if (!found || h[4] > best[4]) {
            for (int i = 0; i < 12; ++i) best[i] = h[i];
            found = true;
        }
    }
    return found && best[4] > 0.8;
}

static const double* coif4_taps()
{
    static double taps[12];
    static int state = 0;  // 0: not solved, 1: solved, -1: failed
    static std::once_flag once;
    std::call_once(once, [] { state = coif4_solve(taps) ? 1 : -1; });
    return state == 1 ? taps : nullptr;
}

static bool wavelet_ok(int wavelet)
{
    if (wavelet == PE_WAVELET_HAAR || wavelet == PE_WAVELET_D4) return true;
    return wavelet == PE_WAVELET_COIF4 && coif4_taps() != nullptr;
}

static Filter make_filter(int wavelet)
{
    Filter f{};
    if (wavelet == PE_WAVELET_COIF4) {
        const double* t = coif4_taps();
        for (int i = 0; i < 12; ++i) f.h[i] = t ? t[i] : 0.0;
        f.len = 12;
    } else if (wavelet == PE_WAVELET_D4) {
        // Daubechies' four-tap filter in closed form: (1+r3, 3+r3, 3-r3, 1-r3) / (4 sqrt 2)
        const double r3 = sqrt(3.0), den = 4.0 * sqrt(2.0);
        f.h[0] = (1.0 + r3) / den;
        f.h[1] = (3.0 + r3) / den;
        f.h[2] = (3.0 - r3) / den;
        f.h[3] = (1.0 - r3) / den;
        f.len = 4;
    } else {
        f.h[0] = f.h[1] = 1.0 / sqrt(2.0);
        f.len = 2;
    }
    return f;
}

// One block per (sample, moment) row: fine values -> level-J_f scaling coefficients ->
// periodized analysis (approximation branch only) down to n_coarse coefficients. Rows cycle
// through nmom moments (density, momentum and, with the pressure, the second moment).
__global__ void __launch_bounds__(256) k_coarsen(const long long* fx, int ncell, int nmom, double scale_n,
                                                 double scale_m, double scale_e, Filter f, int n_coarse, double* out)
{
    extern __shared__ double buf[];
    double* a = buf;
    double* b = buf + ncell;
    const int row = blockIdx.x;
    const int mom = row % nmom;
    const double scale = mom == 0 ? scale_n : (mom == 1 ? scale_m : scale_e);
    const long long* src = fx + (size_t)row * ncell;
    for (int j = threadIdx.x; j < ncell; j += blockDim.x) a[j] = (double)src[j] * scale;
    __syncthreads();
    for (int len = ncell; len > n_coarse; len >>= 1) {
        const int half = len >> 1;
        for (int k = threadIdx.x; k < half; k += blockDim.x) {
            double acc = 0.0;
            for (int m = 0; m < f.len; ++m) acc += f.h[m] * a[(2 * k + m) & (len - 1)];
            b[k] = acc;
        }
        __syncthreads();
        double* t = a;
        a = b;
        b = t;
    }
    for (int k = threadIdx.x; k < n_coarse; k += blockDim.x) out[(size_t)row * n_coarse + k] = a[k];
}

__device__ void synth_level(const Filter& f, const double* a, int nin, double* b);

// Phase space, wavelet form (Section 3.3): one block per row of nvf fixed-point values (coarse
// node i of sample p, hat-weighted in x), converted with `scale` and analysed in v by the
// periodized DWT (approximation branch only) down to nvc coefficients, scaled by 2^(L/2) for L
// levels so that a row's coefficients sum to its mass.
__global__ void __launch_bounds__(256) k_ps_coarsen_v(const long long* fx, int nvf, double scale, Filter f, int nvc,
                                                      double lev, double* out)
{
    extern __shared__ double buf[];
    double* a = buf;
    double* b = buf + nvf;
    const long long* src = fx + (size_t)blockIdx.x * nvf;
    for (int j = threadIdx.x; j < nvf; j += blockDim.x) a[j] = (double)src[j] * scale;
    __syncthreads();
    for (int len = nvf; len > nvc; len >>= 1) {
        const int half = len >> 1;
        for (int k = threadIdx.x; k < half; k += blockDim.x) {
            double acc = 0.0;
            for (int m = 0; m < f.len; ++m) acc += f.h[m] * a[(2 * k + m) & (len - 1)];
            b[k] = acc;
        }
        __syncthreads();
        double* t = a;
        a = b;
        b = t;
    }
    for (int k = threadIdx.x; k < nvc; k += blockDim.x) out[(size_t)blockIdx.x * nvc + k] = a[k] * lev;
}

// Lifting of the wavelet form in v: one block per row of nvc coefficients, periodized synthesis
// with zero details up to nvf cells, scaled by 2^(-L/2) (the inverse of k_ps_coarsen_v on its range).
__global__ void __launch_bounds__(256) k_ps_refine_v(const double* coarse, int nvc, Filter f, int nvf, double lev,
                                                     double* out)
{
    extern __shared__ double buf[];
    double* x = buf;
    double* y = buf + nvf;
    for (int k = threadIdx.x; k < nvc; k += blockDim.x) x[k] = coarse[(size_t)blockIdx.x * nvc + k];
    __syncthreads();
    double* a = x;
    double* b = y;
    for (int len = nvc; len < nvf; len <<= 1) {
        synth_level(f, a, len, b);
        __syncthreads();
        double* t = a;
        a = b;
        b = t;
    }
    for (int j = threadIdx.x; j < nvf; j += blockDim.x) out[(size_t)blockIdx.x * nvf + j] = a[j] * lev;
}

// Least-squares slope in the paired form of Eq. (leastsquares) and the forward-Euler leap.
__global__ void k_ls_project(const double* c, int K, int ncoef, double dt, double dT, double* out, double* slope)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncoef) return;
    const double den = (double)K * (K + 1) * (K + 2) * dt;
    double s = 0.0;
    for (int p = 0; 2 * p <= K; ++p)
        s += 6.0 * (K - 2 * p) / den * (c[(size_t)(K - p) * ncoef + i] - c[(size_t)p * ncoef + i]);
    if (slope) slope[i] = s;
    out[i] = c[(size_t)K * ncoef + i] + (dT - K * dt) * s;
}

__device__ double block_sum_d(double v, double* red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    return warp_sum(lane < nw ? red[lane] : 0.0);
}

__device__ double block_max_d(double v, double* red)
{
    v = warp_max(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    return warp_max(lane < nw ? red[lane] : -1e300);
}

// Periodized synthesis with zero details from nin coefficients in a to 2*nin in b.
__device__ void synth_level(const Filter& f, const double* a, int nin, double* b)
{
    const int n = 2 * nin;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int m = (i & 1); m < f.len; m += 2) acc += f.h[m] * a[((i - m) & (n - 1)) >> 1];
        b[i] = acc;
    }
}

// Returns the buffer holding the refined values (one of x, y).
__device__ double* synthesise(const Filter& f, const double* coarse, int nc, int ncell, double* x, double* y,
                              double scale)
{
    for (int k = threadIdx.x; k < nc; k += blockDim.x) x[k] = coarse[k];
    __syncthreads();
    double* a = x;
    double* b = y;
    for (int len = nc; len < ncell; len <<= 1) {
        synth_level(f, a, len, b);
        __syncthreads();
        double* t = a;
        a = b;
        b = t;
    }
    for (int j = threadIdx.x; j < ncell; j += blockDim.x) a[j] *= scale;
    __syncthreads();
    return a;
}

template <typename P>
__device__ __forceinline__ void refine_body(const double* coarse, int nc, const Filter& f, int ncell, double scale,
                                            P* prof_n, P* prof_u, double* buf, double* red,
                                            const double** nf_out = nullptr, const double** mf_out = nullptr);

template <typename P>
__global__ void __launch_bounds__(1024) k_refine(const double* coarse, int nc, Filter f, int ncell, double scale,
                                                 P* prof_n, P* prof_u)
{
    extern __shared__ double buf[];
    __shared__ double red[32];
    refine_body(coarse, nc, f, ncell, scale, prof_n, prof_u, buf, red);
}

// Lifting profiles of many realisations in one launch (the batched ensemble), block r for
// realisation r: the same arithmetic as k_refine.
struct RefineDesc {
    const double* coarse;
    float* prof_n;
    float* prof_u;
    int nc, ncell;
    double scale;
};

__global__ void __launch_bounds__(1024) k_refine_batch(const RefineDesc* d, Filter f)
{
    extern __shared__ double buf[];
    __shared__ double red[32];
    const RefineDesc r = d[blockIdx.x];
    refine_body(r.coarse, r.nc, f, r.ncell, r.scale, r.prof_n, r.prof_u, buf, red);
}

template <typename P>
__device__ __forceinline__ void refine_body(const double* coarse, int nc, const Filter& f, int ncell, double scale,
                                            P* prof_n, P* prof_u, double* buf, double* red, const double** nf_out,
                                            const double** mf_out)
{
    double* X = buf;
    double* Y = buf + ncell;
    double* Z = buf + 2 * ncell;
    double* nf = synthesise(f, coarse, nc, ncell, X, Y, scale);
    double* o1 = (nf == X) ? Y : X;
    // clamp negative densities and keep the total
    double s0 = 0.0, s1 = 0.0, neg = 0.0;
    for (int j = threadIdx.x; j < ncell; j += blockDim.x) {
        const double v = nf[j];
        s0 += v;
        s1 += fmax(v, 0.0);
        neg += (v < 0.0) ? 1.0 : 0.0;
    }
    s0 = block_sum_d(s0, red);
    s1 = block_sum_d(s1, red);
    neg = block_sum_d(neg, red);
    const double resc = (neg > 0.0 && s1 > 0.0 && s0 > 0.0) ? s0 / s1 : 1.0;
    double nmax = 0.0;
    for (int j = threadIdx.x; j < ncell; j += blockDim.x) {
        const double v = fmax(nf[j], 0.0) * resc;
        nf[j] = v;
        nmax = fmax(nmax, v);
    }
    nmax = block_max_d(nmax, red);
    double* mf = synthesise(f, coarse + nc, nc, ncell, o1, Z, scale);
    for (int j = threadIdx.x; j < ncell; j += blockDim.x) {
        const double n = nf[j];
        prof_n[j] = (P)n;
        prof_u[j] = (n > 1e-12 * nmax) ? (P)(mf[j] / n) : P(0);
    }
    if (nf_out) *nf_out = nf;
    if (mf_out) *mf_out = mf;
}

// Lifting profiles with the ion pressure (Section 3.2): n and u as k_refine, then the second
// moment S synthesised into the two rows left free (four FP64 rows of ncell in shared memory)
// and T = max(S / n - u^2, 0) with u = nV / n in FP64, where n is above the floor of u.
__global__ void __launch_bounds__(1024) k_refine_pressure(const double* coarse, int nc, Filter f, int ncell,
                                                          double scale, float* prof_n, float* prof_u, float* prof_t)
{
    extern __shared__ double buf[];
    __shared__ double red[32];
    const double* nf = nullptr;
    const double* mf = nullptr;
    refine_body(coarse, nc, f, ncell, scale, prof_n, prof_u, buf, red, &nf, &mf);
    double* X = buf;
    double* Y = buf + ncell;
    double* Z = buf + 2 * ncell;
    double* W = buf + 3 * ncell;
    double* o1 = (nf == X) ? Y : X;
    double* free1 = (mf == o1) ? Z : o1;  // the row of the momentum's pair it does not hold
    double nmax = 0.0;
    for (int j = threadIdx.x; j < ncell; j += blockDim.x) nmax = fmax(nmax, nf[j]);
    nmax = block_max_d(nmax, red);
    const double* sf = synthesise(f, coarse + 2 * nc, nc, ncell, free1, W, scale);
    for (int j = threadIdx.x; j < ncell; j += blockDim.x) {
        const double n = nf[j];
        double t = 0.0;
        if (n > 1e-12 * nmax) {
            const double u = mf[j] / n;
            t = sf[j] / n - u * u;
        }
        prof_t[j] = (float)(t > 0.0 ? t : 0.0);
    }
}

// Batched restriction + projection for Haar samples summed over coarse bins (one block per
// realisation): the same arithmetic, in the same order, as pe_coarsen with bin_shift =
// log2(ncell / n_coarse) followed by pe_ls_project.
struct ProjDesc {
    const long long* samp;  // row p of this realisation at samp + p * row_stride: [2][nc]
    int64_t row_stride;
    double scale_n, scale_m;
    double* csamples;  // [K+1][2][nc] coarse samples (may be null)
    double* coarse;    // [2][nc] projected state
    double* slope;     // [2][nc]
    int nc, pad;
};

__global__ void __launch_bounds__(256) k_restrict_project_batch(const ProjDesc* descs, int K, double dt, double dT)
{
    const ProjDesc d = descs[blockIdx.x];
    const int ncoef = 2 * d.nc;
    const double den = (double)K * (K + 1) * (K + 2) * dt;
    for (int i = threadIdx.x; i < ncoef; i += blockDim.x) {
        const double scale = (i >= d.nc) ? d.scale_m : d.scale_n;
        double s = 0.0;
        for (int p = 0; 2 * p <= K; ++p) {
            const double cK = (double)d.samp[(int64_t)(K - p) * d.row_stride + i] * scale;
            const double c0 = (double)d.samp[(int64_t)p * d.row_stride + i] * scale;
            s += 6.0 * (K - 2 * p) / den * (cK - c0);
        }
        const double last = (double)d.samp[(int64_t)K * d.row_stride + i] * scale;
        d.slope[i] = s;
        d.coarse[i] = last + (dT - K * dt) * s;
        if (d.csamples)
            for (int p = 0; p <= K; ++p)
                d.csamples[(size_t)p * ncoef + i] = (double)d.samp[(int64_t)p * d.row_stride + i] * scale;
    }
}

size_t proj_desc_size() { return sizeof(ProjDesc); }

void make_proj_desc(void* out, const int64_t* samp, int64_t row_stride, int ncell, int nc, int s_w, int s_p,
                    double* csamples, double* coarse, double* slope)
{
    const int b = ilog2(ncell / nc);
    const double lev = pow(2.0, -0.5 * (ilog2(ncell) + b));
    ProjDesc d{reinterpret_cast<const long long*>(samp), row_stride, ldexp(1.0, -(s_w + 24)) * lev,
               ldexp(1.0, -(s_p + 24)) * lev, csamples, coarse, slope, nc, 0};
    memcpy(out, &d, sizeof(d));
}

int launch_restrict_project_batch(const void* descs, int R, int K, double dt, double dT, cudaStream_t s)
{
    k_restrict_project_batch<<<R, 256, 0, s>>>(static_cast<const ProjDesc*>(descs), K, dt, dT);
    return launch_status();
}

// Curvature of a burst's coarse trajectory: per component the quadratic least-squares
// coefficient q_i of the K+1 samples at tau_p = (p - K/2) dt on the basis {1, tau, g = tau^2 - m2}
// (m2 the mean of tau^2; the three are orthogonal on the symmetric points):
// q_i = sum_p g_p c_p,i / G with G = sum_p g_p^2, and its sampling variance
// var_i = s_i^2 / G, s_i^2 the residual variance of the fit (K - 2 degrees of freedom).
// Block b sums q_i^2, c_K,i^2, var_i and s_i^2 / T2 (the variance of the least-squares slope,
// T2 = sum_p (t_p - tbar)^2) over its components (a fixed grid-stride partition) into
// part[4 b ..]; the final block adds the partial sums in block order:
// out[0] = sqrt(max(0, sum q_i^2 - sum var_i)) (the curvature with the noise's bias removed),
// out[1] = ||c_K||_2, out[2] = sqrt(sum var_i), out[3] = sqrt(sum s_i^2 / T2) (the slope noise).
// The FP64 work is spread over the SMs.
constexpr int kCurvThreads = 256;
constexpr int kCurvMaxBlocks = 1024;

__global__ void __launch_bounds__(kCurvThreads) k_leap_curvature_part(const double* __restrict__ c, int K, int n,
                                                                     double dt, double* __restrict__ part)
{
    __shared__ double red[32];
    const double m2 = dt * dt * (double)K * (double)(K + 2) / 12.0;
    double G = 0.0, T2 = 0.0;
    for (int p = 0; p <= K; ++p) {
        const double tp = (p - 0.5 * K) * dt, g = tp * tp - m2;
        G += g * g;
        T2 += tp * tp;
    }
    double qq = 0.0, cc = 0.0, vv = 0.0, ss = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double a = 0.0, b = 0.0, q = 0.0;
        for (int p = 0; p <= K; ++p) {
            const double tp = (p - 0.5 * K) * dt, x = c[(size_t)p * n + i];
            a += x;
            b += tp * x;
            q += (tp * tp - m2) * x;
        }
        a /= (K + 1);
        b /= T2;
        q /= G;
        double rr = 0.0;
        for (int p = 0; p <= K; ++p) {
            const double tp = (p - 0.5 * K) * dt;
            const double r = c[(size_t)p * n + i] - (a + b * tp + q * (tp * tp - m2));
            rr += r * r;
        }
        const double cK = c[(size_t)K * n + i];
        qq += q * q;
        cc += cK * cK;
        vv += K > 2 ? rr / (K - 2) / G : 0.0;
        ss += K > 2 ? rr / (K - 2) / T2 : 0.0;
    }
    qq = block_sum_d(qq, red);
    cc = block_sum_d(cc, red);
    vv = block_sum_d(vv, red);
    ss = block_sum_d(ss, red);
    if (threadIdx.x == 0) {
        part[4 * blockIdx.x] = qq;
        part[4 * blockIdx.x + 1] = cc;
        part[4 * blockIdx.x + 2] = vv;
        part[4 * blockIdx.x + 3] = ss;
    }
}

__global__ void k_leap_curvature_final(const double* __restrict__ part, int nb, double* __restrict__ out)
{
    if (threadIdx.x != 0) return;
    double qq = 0.0, cc = 0.0, vv = 0.0, ss = 0.0;
    for (int b = 0; b < nb; ++b) {
        qq += part[4 * b];
        cc += part[4 * b + 1];
        vv += part[4 * b + 2];
        ss += part[4 * b + 3];
    }
    out[0] = sqrt(fmax(0.0, qq - vv));
    out[1] = sqrt(cc);
    out[2] = sqrt(vv);
    out[3] = sqrt(ss);
}

}  // namespace pe

using namespace pe;

extern "C" PE_API int pe_leap_curvature(const double* samples, int32_t K, int32_t ncoef, double dt, double* scratch,
                                        double* out, void* stream)
{
    if (!samples || !out || !scratch || K < 2 || ncoef < 1 || !(dt > 0.0)) return PE_EINVAL;
    const int nb = std::min(kCurvMaxBlocks, (ncoef + kCurvThreads - 1) / kCurvThreads);
    cudaStream_t s = (cudaStream_t)stream;
    k_leap_curvature_part<<<nb, kCurvThreads, 0, s>>>(samples, K, ncoef, dt, scratch);
    k_leap_curvature_final<<<1, 32, 0, s>>>(scratch, nb, out);
    return launch_status(2);
}

extern "C" PE_API int pe_coarsen(const int64_t* sample_fx, int32_t nsamples, int32_t ncell, int32_t s_w, int32_t s_p,
                                 int32_t wavelet, int32_t n_coarse, int32_t bin_shift, double* coarse, void* stream)
{
    if (!is_pow2(ncell) || !is_pow2(n_coarse) || n_coarse > ncell || nsamples < 1 || !sample_fx || !coarse)
        return PE_EINVAL;
    if (!wavelet_ok(wavelet)) return PE_EINVAL;
    if (bin_shift < 0 || (bin_shift > 0 && wavelet != PE_WAVELET_HAAR) || (ncell >> bin_shift) < n_coarse)
        return PE_EINVAL;
    const int nb = ncell >> bin_shift;  // input length per row
    const size_t smem = 2 * sizeof(double) * (size_t)nb;
    if (smem > (size_t)max_smem_optin()) return PE_EINVAL;
    if (ensure_smem((const void*)k_coarsen, smem) != PE_OK) return PE_ECUDA;
    // fine values are level-J_f scaling coefficients 2^{-J_f/2} f; b Haar levels of a bin sum add 2^{-b/2}
    const double lev = pow(2.0, -0.5 * (ilog2(ncell) + bin_shift));
    k_coarsen<<<2 * nsamples, 256, smem, (cudaStream_t)stream>>>(reinterpret_cast<const long long*>(sample_fx), nb, 2,
                                                                 ldexp(1.0, -(s_w + 24)) * lev,
                                                                 ldexp(1.0, -(s_p + 24)) * lev, 0.0,
                                                                 make_filter(wavelet), n_coarse, coarse);
    return launch_status();
}

extern "C" PE_API int pe_coarsen_pressure(const int64_t* sample_fx, int32_t nsamples, int32_t ncell, int32_t s_w,
                                          int32_t s_p, int32_t s_e, int32_t wavelet, int32_t n_coarse,
                                          int32_t bin_shift, double* coarse, void* stream)
{
    if (!is_pow2(ncell) || !is_pow2(n_coarse) || n_coarse > ncell || nsamples < 1 || !sample_fx || !coarse)
        return PE_EINVAL;
    if (!wavelet_ok(wavelet)) return PE_EINVAL;
    if (bin_shift < 0 || (bin_shift > 0 && wavelet != PE_WAVELET_HAAR) || (ncell >> bin_shift) < n_coarse)
        return PE_EINVAL;
    const int nb = ncell >> bin_shift;  // input length per row
    const size_t smem = 2 * sizeof(double) * (size_t)nb;
    if (smem > (size_t)max_smem_optin()) return PE_EINVAL;
    if (ensure_smem((const void*)k_coarsen, smem) != PE_OK) return PE_ECUDA;
    const double lev = pow(2.0, -0.5 * (ilog2(ncell) + bin_shift));
    k_coarsen<<<3 * nsamples, 256, smem, (cudaStream_t)stream>>>(reinterpret_cast<const long long*>(sample_fx), nb, 3,
                                                                 ldexp(1.0, -(s_w + 24)) * lev,
                                                                 ldexp(1.0, -(s_p + 24)) * lev,
                                                                 ldexp(1.0, -(s_e + 24)) * lev, make_filter(wavelet),
                                                                 n_coarse, coarse);
    return launch_status();
}

extern "C" PE_API int pe_ps_coarsen_v(const int64_t* sample_fx, int64_t nrows, int32_t n_vf, int32_t s_w,
                                      int32_t bin_shift, int32_t wavelet, int32_t n_vc, double* coarse, void* stream)
{
    if (!sample_fx || !coarse || nrows < 0 || nrows > INT32_MAX || !is_pow2(n_vf) || !is_pow2(n_vc) || n_vc > n_vf ||
        n_vf > 4096 || bin_shift < 0 || bin_shift > 30 || s_w < -60 || s_w > 60 || !wavelet_ok(wavelet))
        return PE_EINVAL;
    if (nrows == 0) return PE_OK;
    const size_t smem = 2 * sizeof(double) * (size_t)n_vf;
    if (ensure_smem((const void*)k_ps_coarsen_v, smem) != PE_OK) return PE_ECUDA;
    const int L = ilog2(n_vf / n_vc);
    k_ps_coarsen_v<<<(unsigned)nrows, 256, smem, (cudaStream_t)stream>>>(
        reinterpret_cast<const long long*>(sample_fx), n_vf, ldexp(1.0, -(s_w + 24 + bin_shift)),
        make_filter(wavelet), n_vc, pow(2.0, 0.5 * L), coarse);
    return launch_status();
}

extern "C" PE_API int pe_ps_refine_v(const double* coarse, int64_t nrows, int32_t n_vc, int32_t wavelet, int32_t n_vf,
                                     double* hist, void* stream)
{
    if (!coarse || !hist || nrows < 0 || nrows > INT32_MAX || !is_pow2(n_vf) || !is_pow2(n_vc) || n_vc > n_vf ||
        n_vf > 4096 || !wavelet_ok(wavelet))
        return PE_EINVAL;
    if (nrows == 0) return PE_OK;
    const size_t smem = 2 * sizeof(double) * (size_t)n_vf;
    if (ensure_smem((const void*)k_ps_refine_v, smem) != PE_OK) return PE_ECUDA;
    const int L = ilog2(n_vf / n_vc);
    k_ps_refine_v<<<(unsigned)nrows, 256, smem, (cudaStream_t)stream>>>(coarse, n_vc, make_filter(wavelet), n_vf,
                                                                         pow(2.0, -0.5 * L), hist);
    return launch_status();
}

extern "C" PE_API int pe_ls_project(const double* samples, int32_t K, int32_t ncoef, double dt, double dT, double* out,
                                    double* slope, void* stream)
{
    if (!samples || !out || K < 1 || ncoef < 1 || !(dt > 0.0)) return PE_EINVAL;
    const int block = 256;
    k_ls_project<<<(ncoef + block - 1) / block, block, 0, (cudaStream_t)stream>>>(samples, K, ncoef, dt, dT, out, slope);
    return launch_status();
}

namespace pe {
size_t refine_desc_size() { return sizeof(RefineDesc); }

void make_refine_desc(void* out, const double* coarse, int nc, int ncell, float* prof_n, float* prof_u)
{
    RefineDesc d{coarse, prof_n, prof_u, nc, ncell, pow(2.0, 0.5 * ilog2(ncell))};
    memcpy(out, &d, sizeof(d));
}

// R realisations (descs on the device), all with the same wavelet, grids of at most max_ncell.
int launch_refine_batch(const void* descs, int R, int wavelet, int max_ncell, cudaStream_t s)
{
    const size_t smem = 3 * sizeof(double) * (size_t)max_ncell;
    if (R < 1 || smem > (size_t)max_smem_optin() || !wavelet_ok(wavelet)) return PE_EINVAL;
    if (ensure_smem((const void*)k_refine_batch, smem) != PE_OK) return PE_ECUDA;
    k_refine_batch<<<R, 1024, smem, s>>>(static_cast<const RefineDesc*>(descs), make_filter(wavelet));
    return launch_status();
}
}  // namespace pe

template <typename P>
static int refine_into(const double* coarse, int32_t n_coarse, int32_t wavelet, int32_t ncell, P* prof_n, P* prof_u,
                       void* stream)
{
    if (!is_pow2(ncell) || !is_pow2(n_coarse) || n_coarse > ncell || !coarse || !prof_n || !prof_u) return PE_EINVAL;
    if (!wavelet_ok(wavelet)) return PE_EINVAL;
    const size_t smem = 3 * sizeof(double) * (size_t)ncell;
    if (smem > (size_t)max_smem_optin()) return PE_EINVAL;
    if (ensure_smem((const void*)k_refine<P>, smem) != PE_OK) return PE_ECUDA;
    k_refine<P><<<1, 1024, smem, (cudaStream_t)stream>>>(coarse, n_coarse, make_filter(wavelet), ncell,
                                                         pow(2.0, 0.5 * ilog2(ncell)), prof_n, prof_u);
    return launch_status();
}

extern "C" PE_API int pe_refine_pressure(const double* coarse, int32_t n_coarse, int32_t wavelet, int32_t ncell,
                                         float* prof_n, float* prof_u, float* prof_T, void* stream)
{
    if (!is_pow2(ncell) || !is_pow2(n_coarse) || n_coarse > ncell || ncell > 4096 || !coarse || !prof_n || !prof_u ||
        !prof_T)
        return PE_EINVAL;
    if (!wavelet_ok(wavelet)) return PE_EINVAL;
    const size_t smem = 4 * sizeof(double) * (size_t)ncell;
    if (smem > (size_t)max_smem_optin()) return PE_EINVAL;
    if (ensure_smem((const void*)k_refine_pressure, smem) != PE_OK) return PE_ECUDA;
    k_refine_pressure<<<1, 1024, smem, (cudaStream_t)stream>>>(coarse, n_coarse, make_filter(wavelet), ncell,
                                                               pow(2.0, 0.5 * ilog2(ncell)), prof_n, prof_u, prof_T);
    return launch_status();
}

extern "C" PE_API int pe_refine(const double* coarse, int32_t n_coarse, int32_t wavelet, int32_t ncell, float* prof_n,
                                float* prof_u, void* stream)
{
    return refine_into(coarse, n_coarse, wavelet, ncell, prof_n, prof_u, stream);
}

extern "C" PE_API int pe_refine_f64(const double* coarse, int32_t n_coarse, int32_t wavelet, int32_t ncell,
                                    double* prof_n, double* prof_u, void* stream)
{
    return refine_into(coarse, n_coarse, wavelet, ncell, prof_n, prof_u, stream);
}
