// Diagnostics of a particle state (Section 4: the charge, momentum and energy checks of
// the resolved and projective runs; the particle Courant number max|V| dt / dx of the
// fine step, the particle-level counterpart of the macroscopic condition Eq. (CFL)) and the
// coarse-variable error measure of Section 4.1.1.
//
// Two launches: a particle pass (grid-stride, fixed grid for a given n, so the
// floating-point sums are reproduced bit for bit) writes one partial per block; a
// single 1024-thread block adds the partials in a fixed tree and the grid energies.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pe_common.cuh"
#include "pe_internal.h"
#include "pepic.h"

namespace pe {
namespace {

constexpr int kDiagThreads = 256;
constexpr int kDiagMaxBlocks = 1024;
constexpr int kFinalThreads = 1024;

struct DiagScratch {
    long long charge[kDiagMaxBlocks];
    long long wq[kDiagMaxBlocks];
    long long invalid[kDiagMaxBlocks];
    double mom[kDiagMaxBlocks];
    double kin[kDiagMaxBlocks];
    double wsum[kDiagMaxBlocks];
    float vmax[kDiagMaxBlocks];
};
static_assert(sizeof(DiagScratch) <= PE_MOMENTS_SCRATCH_BYTES, "scratch size");

__device__ __forceinline__ long long warp_sum_i64(long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_maxf(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Particle pass. Vbar = v + (kick - 1/2) qm dt E(X) is the integer-time velocity; a
// particle with a cell outside [0, ncell), a non-finite offset or velocity, or an offset
// outside [0, 1] is counted as invalid, sets PE_FLAG_RANGE and is left out of the sums.
__global__ void __launch_bounds__(kDiagThreads) k_moments_particles(
    const int32_t* __restrict__ cell, const float* __restrict__ theta, const float* __restrict__ v,
    const float* __restrict__ w, int64_t n, const float* __restrict__ Ef, int ncell, float hk, float wscale,
    DiagScratch* __restrict__ out, uint32_t* status)
{
    long long q = 0, bad = 0, qw = 0;
    double mom = 0.0, kin = 0.0, ws = 0.0;
    float vmax = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int c = cell[i];
        const float th = theta[i], vv = v[i], ww = w[i];
        if ((unsigned)c >= (unsigned)ncell || !isfinite(vv) || !isfinite(ww) || !(th >= 0.0f && th <= 1.0f)) {
            ++bad;
            continue;
        }
        const int c1 = (c + 1 == ncell) ? 0 : c + 1;
        const float Ec = __ldg(Ef + c), Ec1 = __ldg(Ef + c1);
        const float vb = fmaf(hk, fmaf(th, Ec1 - Ec, Ec), vv);
        const long long wqi = (long long)__float2int_rn(ww * wscale);
        q += wqi * (long long)kThetaOne;
        qw += wqi;
        const double wd = (double)ww, vd = (double)vb;
        mom += wd * vd;
        kin += 0.5 * wd * vd * vd;
        ws += wd;
        vmax = fmaxf(vmax, fabsf(vb));
    }
    __shared__ long long sq[kDiagThreads / 32], sb[kDiagThreads / 32], sqw[kDiagThreads / 32];
    __shared__ double sm[kDiagThreads / 32], sk[kDiagThreads / 32], sw[kDiagThreads / 32];
    __shared__ float sv[kDiagThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    q = warp_sum_i64(q);
    bad = warp_sum_i64(bad);
    qw = warp_sum_i64(qw);
    mom = warp_sum(mom);
    kin = warp_sum(kin);
    ws = warp_sum(ws);
    vmax = warp_maxf(vmax);
    if (lane == 0) {
        sq[wid] = q;
        sb[wid] = bad;
        sqw[wid] = qw;
        sm[wid] = mom;
        sk[wid] = kin;
        sw[wid] = ws;
        sv[wid] = vmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kDiagThreads / 32; ++k) {
            q += sq[k];
            bad += sb[k];
            qw += sqw[k];
            mom += sm[k];
            kin += sk[k];
            ws += sw[k];
            vmax = fmaxf(vmax, sv[k]);
        }
        out->charge[blockIdx.x] = q;
        out->invalid[blockIdx.x] = bad;
        out->wq[blockIdx.x] = qw;
        out->mom[blockIdx.x] = mom;
        out->kin[blockIdx.x] = kin;
        out->wsum[blockIdx.x] = ws;
        out->vmax[blockIdx.x] = vmax;
        if (bad) raise_flag(status, PE_FLAG_RANGE);
    }
}

template <typename T, typename Op>
__device__ T block_reduce(T x, T* red, Op op)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) x = op(x, __shfl_xor_sync(0xffffffffu, x, o));
    __syncthreads();
    if (lane == 0) red[wid] = x;
    __syncthreads();
    if (wid == 0) {
        x = red[lane];  // 32 warps of 32 threads
        for (int o = 16; o > 0; o >>= 1) x = op(x, __shfl_xor_sync(0xffffffffu, x, o));
    }
    return x;  // valid in warp 0
}

// Final pass: sums of the block partials (fixed order) and of the nodal energies.
__global__ void __launch_bounds__(kFinalThreads) k_moments_final(
    const DiagScratch* __restrict__ part, int nblocks, const double* __restrict__ phi, const double* __restrict__ E,
    int ncell, double dx, double dt, double charge_scale, int mode, pe_moments* out)
{
    __shared__ double rd[32];
    __shared__ long long ri[32];
    __shared__ float rf[32];
    const int t = threadIdx.x;
    const bool have = t < nblocks;
    long long q = have ? part->charge[t] : 0, bad = have ? part->invalid[t] : 0, qw = have ? part->wq[t] : 0;
    double mom = have ? part->mom[t] : 0.0, kin = have ? part->kin[t] : 0.0, ws = have ? part->wsum[t] : 0.0;
    float vmax = have ? part->vmax[t] : 0.0f;
    double fe = 0.0, ee = 0.0;
    for (int j = t; j < ncell; j += kFinalThreads) {
        const double e = E ? E[j] : 0.0;
        fe += 0.5 * e * e;
        if (phi) {
            const double p = phi[j];
            ee += (mode == PE_POISSON_BOLTZMANN) ? (p * exp(p) - exp(p) + 1.0) : 0.5 * p * p;
        }
    }
    auto add_i = [](long long a, long long b) { return a + b; };
    auto add_d = [](double a, double b) { return a + b; };
    auto max_f = [](float a, float b) { return fmaxf(a, b); };
    q = block_reduce(q, ri, add_i);
    const long long qs = q;
    bad = block_reduce(bad, ri, add_i);
    const long long bads = bad;
    qw = block_reduce(qw, ri, add_i);
    mom = block_reduce(mom, rd, add_d);
    const double moms = mom;
    kin = block_reduce(kin, rd, add_d);
    const double kins = kin;
    ws = block_reduce(ws, rd, add_d);
    const double wss = ws;
    fe = block_reduce(fe, rd, add_d);
    const double fes = fe;
    ee = block_reduce(ee, rd, add_d);
    vmax = block_reduce(vmax, rf, max_f);
    if (t == 0) {
        pe_moments m;
        m.charge_fx = qs;
        m.invalid = bads;
        m.charge_wq = qw;
        m.charge_fixed_point = (double)qs * charge_scale * dx;
        m.charge = wss * dx;
        m.momentum = moms * dx;
        m.kinetic = kins * dx;
        m.field_energy = fes * dx;
        m.electron_energy = ee * dx;
        m.total_energy = m.kinetic + m.field_energy + m.electron_energy;
        m.max_speed = (double)vmax;
        m.cfl = (double)vmax * dt / dx;
        *out = m;
    }
}

__global__ void __launch_bounds__(kFinalThreads) k_rel_l2(const double* __restrict__ a, const double* __restrict__ b,
                                                           int64_t n, double* out)
{
    __shared__ double rd[32];
    double num = 0.0, den = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kFinalThreads) {
        const double x = a[i], y = b[i];
        num += (x - y) * (x - y);
        den += x * x + y * y;
    }
    auto add_d = [](double u, double v) { return u + v; };
    num = block_reduce(num, rd, add_d);
    const double nums = num;
    den = block_reduce(den, rd, add_d);
    if (threadIdx.x == 0) *out = den > 0.0 ? sqrt(nums / den) : 0.0;
}

}  // namespace

int moments_blocks(int64_t n)
{
    const int64_t per = (int64_t)kDiagThreads * 16;
    int64_t b = (n + per - 1) / per;
    if (b < 1) b = 1;
    if (b > kDiagMaxBlocks) b = kDiagMaxBlocks;
    return (int)b;
}

}  // namespace pe

using namespace pe;

namespace pe {
namespace {
// Kinetic energy sum w Vbar^2 dx / 2 of one species: FP32 per-thread sums over a fixed
// grid-stride partition, FP64 from the warp sums on (the FP64 pipe is narrow on this part), block
// partials folded in block order by one thread: reproducible.
constexpr int kEnergyBlocks = 1024;

__global__ void __launch_bounds__(kDiagThreads) k_energy_part(const int32_t* __restrict__ cell,
                                                              const float* __restrict__ theta,
                                                              const float* __restrict__ v, const float* __restrict__ w,
                                                              int64_t n, const float* __restrict__ Ef, int ncell,
                                                              float hk, double* __restrict__ part,
                                                              uint32_t* __restrict__ status)
{
    float k = 0.0f;
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int c = cell[i];
        if ((unsigned)c >= (unsigned)ncell) {
            bad = true;
            continue;
        }
        const int c1 = (c + 1 == ncell) ? 0 : c + 1;
        const float Ec = __ldg(Ef + c), Ec1 = __ldg(Ef + c1);
        const float vb = fmaf(hk, fmaf(theta[i], Ec1 - Ec, Ec), v[i]);
        k = fmaf(w[i] * vb, vb, k);
    }
    if (bad) raise_flag(status, PE_FLAG_RANGE);
    __shared__ double sk[kDiagThreads / 32];
    const double kw = warp_sum((double)k);
    if ((threadIdx.x & 31) == 0) sk[threadIdx.x >> 5] = kw;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < kDiagThreads / 32; ++j) t += sk[j];
        part[blockIdx.x] = t;
    }
}

__global__ void k_energy_final(const double* __restrict__ part, int nb, double half_dx, double* __restrict__ out)
{
    if (threadIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[b];
    *out = t * half_dx;
}
}  // namespace
}  // namespace pe

extern "C" PE_API int pe_kinetic_energy(const int32_t* cell, const float* theta, const float* v, const float* w,
                                        int64_t n, const float* Ef, int32_t ncell, double dx, float qm_dt, float kick,
                                        double* scratch, double* out, uint32_t* status, void* stream)
{
    if (n < 0 || ncell < 2 || !(dx > 0.0) || !scratch || !out || !status) return PE_EINVAL;
    if (n > 0 && (!cell || !theta || !v || !w || !Ef)) return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)std::min<int64_t>(kEnergyBlocks, std::max<int64_t>(1, (n + 4095) / 4096));
    k_energy_part<<<nb, kDiagThreads, 0, s>>>(cell, theta, v, w, n, Ef, ncell, (kick - 0.5f) * qm_dt, scratch,
                                              status);
    k_energy_final<<<1, 32, 0, s>>>(scratch, nb, 0.5 * dx, out);
    return launch_status(2);
}

extern "C" PE_API int pe_compute_moments(const int32_t* cell, const float* theta, const float* v, const float* w, int64_t n,
                                 const float* Ef, const double* phi, const double* E, int32_t ncell, double dx,
                                 double dt, float qm_dt, float kick, int32_t s_w, int32_t mode, void* scratch,
                                 pe_moments* out, uint32_t* status, void* stream)
{
    if (n < 0 || ncell < 2 || !(dx > 0.0) || !(dt >= 0.0) || !scratch || !out) return PE_EINVAL;
    if (n > 0 && (!cell || !theta || !v || !w || !Ef)) return PE_EINVAL;
    if (((uintptr_t)scratch & 15u) || ((uintptr_t)out & 7u)) return PE_EINVAL;
    if (mode != PE_POISSON_BOLTZMANN && mode != PE_POISSON_LINEARIZED) return PE_EINVAL;
    if (s_w < -60 || s_w > 60) return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = moments_blocks(n);
    DiagScratch* part = (DiagScratch*)scratch;
    const float wscale = ldexpf(1.0f, s_w);
    const float hk = (kick - 0.5f) * qm_dt;
    k_moments_particles<<<nb, kDiagThreads, 0, s>>>(cell, theta, v, w, n, Ef, ncell, hk, wscale, part, status);
    k_moments_final<<<1, kFinalThreads, 0, s>>>(part, nb, phi, E, ncell, dx, dt, ldexp(1.0, -(s_w + 24)), mode, out);
    return launch_status(2);
}

namespace pe {

// Kinetic electrons: the ions' moments (out) absorb the electrons' (e, velocities of the
// electron pass, mass w / |q_e/m_e| per particle): electron_energy = the electrons' kinetic
// energy, momentum of both species, the larger speed and CFL number, total = kinetic of the
// ions + field + electrons.
__global__ void k_moments_kinetic(pe_moments* out, const pe_moments* e, double inv_mass_ratio)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    out->electron_energy = e->kinetic * inv_mass_ratio;
    out->momentum += e->momentum * inv_mass_ratio;
    out->total_energy = out->kinetic + out->field_energy + out->electron_energy;
    out->max_speed = fmax(out->max_speed, e->max_speed);
    out->cfl = fmax(out->cfl, e->cfl);
    out->invalid += e->invalid;
}

int combine_kinetic_moments(pe_moments* out, const pe_moments* electrons, double qm_e, cudaStream_t s)
{
    if (!(qm_e < 0.0)) return PE_EINVAL;
    k_moments_kinetic<<<1, 32, 0, s>>>(out, electrons, 1.0 / -qm_e);
    return launch_status(1);
}

}  // namespace pe

extern "C" PE_API int pe_rel_l2(const double* a, const double* b, int64_t n, double* out, void* stream)
{
    if (n < 0 || !out || (n > 0 && (!a || !b))) return PE_EINVAL;
    k_rel_l2<<<1, kFinalThreads, 0, (cudaStream_t)stream>>>(a, b, n, out);
    return launch_status(1);
}
