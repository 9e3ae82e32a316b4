// FP64 particles: the same method as the FP32 particle pass (Appendix C loading, Section 2.2
// leapfrog with CIC gather, Appendix B co-moving restriction sample, the fixed-point charge
// deposit), with (theta, v, w) stored in double precision. The small workload of the method
// (128 cells, 2^17 ions) runs both ways, so that the error of a run against the FP64 oracle
// separates into the FP32 particles' precision and the method itself.
//
// One particle per thread; the fixed-point sums go straight to the global int64 grids with
// 64-bit atomics (exact, so the order does not matter). The FP64 path is latency-bound at the
// sizes it serves; throughput is the FP32 path's job.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pe_common.cuh"
#include "pe_internal.h"

namespace pe {

constexpr int kThreads64 = 256;
constexpr double kThetaOneD = 16777216.0;  // 2^24

// Fixed-point CIC split of one FP64 particle: theta_q = rn(theta 2^24), the same rule as the
// FP32 particles (theta 2^24 is exact in FP64 too; round half to even).
__device__ __forceinline__ void fx_add64(unsigned long long* g, int c, int c1, long long q, double theta)
{
    const long long tq = __double2ll_rn(theta * kThetaOneD);
    const long long r = q * tq;
    const long long l = q * (long long)(1 << 24) - r;
    atomicAdd(g + c, (unsigned long long)l);
    atomicAdd(g + c1, (unsigned long long)r);
}

__device__ __forceinline__ long long fx_q64(double x, double scale, uint32_t* status)
{
    const long long q = __double2ll_rn(x * scale);
    if (q > (1ll << 23) || q < -(1ll << 23)) raise_flag(status, PE_FLAG_OVERFLOW);
    return q;
}

// Drift by s cells: theta + s = k + theta', theta' in [0, 1) (a rounding to 1 moves to the next cell).
__device__ __forceinline__ void drift64(int& c, double& th, double s, int mask)
{
    const double x = th + s;
    double k = floor(x);
    double t = x - k;
    if (t >= 1.0) {
        t = 0.0;
        k += 1.0;
    }
    c = (c + (int)k) & mask;
    th = t;
}

struct Push64 {
    int32_t* cell;
    double* theta;
    double* v;
    const double* w;
    int64_t n;
    const double* E;
    int ncell, mask;
    double dt_dx, qm_dt, kick, wscale;
    unsigned long long* rho;  // deposit of the pushed particles (push) or of the current ones
    const double* E0;         // restriction sample at the start of the pass (nullptr: none)
    double tau_dx, qm_tau, pscale;
    unsigned long long* samp;  // [2][ncell]: density then momentum
    int push;
    uint32_t* status;
};

// One thread per particle: the co-moving sample of the current state (Appendix B: target
// X + tau Vbar, velocity Vbar + qm tau E0(X), Vbar the integer-time velocity), then the kick
// and drift, then the charge deposit of the new position.
__global__ void __launch_bounds__(kThreads64) k_particles64(Push64 P)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    int c = P.cell[i];
    if ((unsigned)c >= (unsigned)P.ncell) {
        raise_flag(P.status, PE_FLAG_RANGE);
        return;
    }
    double th = P.theta[i], vv = P.v[i];
    const double ww = P.w[i];
    const int c1 = (c + 1) & P.mask;
    const double Ep = (1.0 - th) * P.E[c] + th * P.E[c1];
    const long long wq = fx_q64(ww, P.wscale, P.status);
    if (P.E0) {
        const double vbar = vv + (P.kick - 0.5) * P.qm_dt * Ep;
        const double E0p = (1.0 - th) * P.E0[c] + th * P.E0[c1];
        int cs = c;
        double ts = th;
        drift64(cs, ts, P.tau_dx * vbar, P.mask);
        const double vt = vbar + P.qm_tau * E0p;
        const long long mq = fx_q64(ww * vt, P.pscale, P.status);
        const int cs1 = (cs + 1) & P.mask;
        fx_add64(P.samp, cs, cs1, wq, ts);
        fx_add64(P.samp + P.ncell, cs, cs1, mq, ts);
    }
    if (P.push) {
        vv += P.kick * P.qm_dt * Ep;
        drift64(c, th, vv * P.dt_dx, P.mask);
        P.cell[i] = c;
        P.theta[i] = th;
        P.v[i] = vv;
    }
    if (P.rho) fx_add64(P.rho, c, (c + 1) & P.mask, wq, th);
}

struct Load64 {
    int32_t* cell;
    double* theta;
    double* v;
    double* w;
    int64_t n;
    uint32_t ppc;
    int log2ppc, ncell, mask;
    const double* prof_n;
    const double* prof_u;
    double v_th, wscale;
    uint32_t half, shift;
    unsigned long long* rho;
    uint32_t* status;
};

// Appendix C: storage slot s holds the Hammersley point h (h = s, or with ppc = 2^m its low m
// bits reversed: the cell's points in ascending velocity quantile), cell h / ppc, offset
// (2 (h mod ppc) + 1) / (2 ppc), weight n(X) / ppc, V = u(X) + v_th Phi^-1(b_h) with
// b_h = (B_h + 1/2) 2^-32, B_h = brev32(h) + floor(2^31 / n) + shift (mod 2^32).
__global__ void __launch_bounds__(kThreads64) k_quiet_start64(Load64 P)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.n) return;
    uint32_t h = (uint32_t)s;
    if (P.log2ppc > 0) {
        const uint32_t k = h & (P.ppc - 1u);
        h = (h & ~(P.ppc - 1u)) | (__brev(k) >> (32 - P.log2ppc));
    }
    const int c = (int)(h / P.ppc);
    const double th = (2.0 * (double)(h % P.ppc) + 1.0) / (2.0 * (double)P.ppc);
    const int c1 = (c + 1) & P.mask;
    const double nX = (1.0 - th) * P.prof_n[c] + th * P.prof_n[c1];
    const double uX = (1.0 - th) * P.prof_u[c] + th * P.prof_u[c1];
    const uint32_t B = __brev(h) + P.half + P.shift;
    const double b = ((double)B + 0.5) * 2.3283064365386963e-10;
    const double ww = nX / (double)P.ppc;
    P.cell[s] = c;
    P.theta[s] = th;
    P.w[s] = ww;
    P.v[s] = uX + P.v_th * normcdfinv(b);
    if (P.rho) fx_add64(P.rho, c, c1, fx_q64(ww, P.wscale, P.status), th);
}

static bool ok64(const void* a, const void* b, const void* c, const void* d, int64_t n)
{
    return n >= 0 && n < (int64_t(1) << 32) && (n == 0 || (a && b && c && d));
}

static int blocks64(int64_t n) { return (int)((n + kThreads64 - 1) / kThreads64); }

}  // namespace pe

using namespace pe;

extern "C" PE_API int pe_push_f64(int32_t* cell, double* theta, double* v, const double* w, int64_t n,
                                  const double* E, int32_t ncell, double dt_over_dx, double qm_dt, double kick,
                                  int32_t s_w, int64_t* rho_fx, const double* E0, double tau_over_dx, double qm_tau,
                                  int32_t s_p, int64_t* sample_fx, uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !E || !ok64(cell, theta, v, w, n) || (E0 && !sample_fx)) return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Push64 P{cell, theta, v, w, n, E, ncell, ncell - 1, dt_over_dx, qm_dt, kick, ldexp(1.0, s_w),
             reinterpret_cast<unsigned long long*>(rho_fx), E0, tau_over_dx, qm_tau, ldexp(1.0, s_p),
             reinterpret_cast<unsigned long long*>(sample_fx), 1, status};
    if (rho_fx && cudaMemsetAsync(rho_fx, 0, sizeof(int64_t) * (size_t)ncell, s) != cudaSuccess) return PE_ECUDA;
    if (E0 && cudaMemsetAsync(sample_fx, 0, 2 * sizeof(int64_t) * (size_t)ncell, s) != cudaSuccess) return PE_ECUDA;
    if (n == 0) return PE_OK;
    k_particles64<<<blocks64(n), kThreads64, 0, s>>>(P);
    return launch_status();
}

extern "C" PE_API int pe_sample_f64(const int32_t* cell, const double* theta, const double* v, const double* w,
                                    int64_t n, const double* E, int32_t ncell, double qm_dt, double kick, int32_t s_w,
                                    const double* E0, double tau_over_dx, double qm_tau, int32_t s_p,
                                    int64_t* sample_fx, uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !E || !E0 || !sample_fx || !ok64(cell, theta, v, w, n)) return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Push64 P{const_cast<int32_t*>(cell), const_cast<double*>(theta), const_cast<double*>(v), w, n, E, ncell,
             ncell - 1, 0.0, qm_dt, kick, ldexp(1.0, s_w), nullptr, E0, tau_over_dx, qm_tau, ldexp(1.0, s_p),
             reinterpret_cast<unsigned long long*>(sample_fx), 0, status};
    if (cudaMemsetAsync(sample_fx, 0, 2 * sizeof(int64_t) * (size_t)ncell, s) != cudaSuccess) return PE_ECUDA;
    if (n == 0) return PE_OK;
    k_particles64<<<blocks64(n), kThreads64, 0, s>>>(P);
    return launch_status();
}

extern "C" PE_API int pe_quiet_start_f64(int32_t* cell, double* theta, double* v, double* w, int64_t n, int32_t ncell,
                                         const double* prof_n, const double* prof_u, double v_th, uint64_t seed,
                                         int32_t s_w, int64_t* rho_fx, uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !prof_n || !prof_u || !ok64(cell, theta, v, w, n)) return PE_EINVAL;
    if (n == 0 || n % ncell != 0) return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Load64 P{};
    P.cell = cell;
    P.theta = theta;
    P.v = v;
    P.w = w;
    P.n = n;
    P.ppc = (uint32_t)(n / ncell);
    P.log2ppc = is_pow2(P.ppc) ? ilog2(P.ppc) : -1;
    P.ncell = ncell;
    P.mask = ncell - 1;
    P.prof_n = prof_n;
    P.prof_u = prof_u;
    P.v_th = v_th;
    P.wscale = ldexp(1.0, s_w);
    P.half = (uint32_t)(2147483648.0 / (double)n);
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL;  // splitmix64 of the seed: the shift is its upper half
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    P.shift = (uint32_t)(z >> 32);
    P.rho = reinterpret_cast<unsigned long long*>(rho_fx);
    P.status = status;
    if (rho_fx && cudaMemsetAsync(rho_fx, 0, sizeof(int64_t) * (size_t)ncell, s) != cudaSuccess) return PE_ECUDA;
    k_quiet_start64<<<blocks64(n), kThreads64, 0, s>>>(P);
    return launch_status();
}
