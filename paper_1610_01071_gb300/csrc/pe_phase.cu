// Phase-space coarse variable (Section 3.3, "A wavelet-based equation-free scheme", with
// Appendices B and C), Haar reading: the active variables are the masses H[i][j] of the
// phase-space cells (coarse x-bin i of 2^b nodes, velocity cell j of width dv from v_min).
// The co-moving restriction sample itself is a mode of the fused particle pass
// (pe_push / pe_sample with n_v > 0); this file holds the rest of the cycle:
//   - pe_ps_coarsen: fixed-point samples -> FP64 masses;
//   - pe_ps_lift_tables: per bin the mass and the momentum-conserving reconstruction of the
//     velocity CDF (Appendix C), one warp per bin, in FP64 with every operation rounded
//     separately (no contraction) so the tables are reproducible bit for bit;
//   - pe_ps_quiet_start: the Hammersley loading of Appendix C on those tables, with the
//     charge deposit of the new particles fused;
//   - pe_ps_quiet_start_equal: the same on a bounded grid, with equal weights placed by the
//     mass of the bins (the equal-weight loader of pe_eq.cuh).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "pe_common.cuh"
#include "pe_eq.cuh"
#include "pe_internal.h"
#include "pepic.h"

namespace pe {
namespace {

// Fixed-point weight rn(x 2^s) of the deposit rule; records whether |q| left 2^23.
__device__ __forceinline__ int32_t fx_weight_q(float x, float scale, bool* ovf)
{
    const int32_t q = __float2int_rn(x * scale);
    *ovf |= (q > (1 << 23)) | (q < -(1 << 23));
    return q;
}

// FP64 arithmetic without fused multiply-add, so that the device reproduces a host
// evaluation of the same expressions in the same order.
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double div_(double a, double b) { return __ddiv_rn(a, b); }

// Reconstruction of a CDF row F[0..N] (Appendix C) by one warp, the row in shared memory. Each
// step tests candidate ranges in a fixed order and keeps the first that passes; the warp tests
// up to 32 candidates at once, each with exactly the operations (each rounded separately) of
// the serial test, and keeps the first passing one in the serial order, so the result is that
// of the serial procedure bit for bit. The sums S that the tests need are running sums, left to
// right; lane 0 extends them one candidate at a time into the warp's slots Sc[0..31].
constexpr unsigned kFull = 0xffffffffu;

// Smallest k in [from, to) with F[k] >= x, or to.
__device__ __forceinline__ int warp_first_geq(const double* F, int from, int to, double x, int lane)
{
    for (int base = from; base < to; base += 32) {
        const int k = base + lane;
        const unsigned m = __ballot_sync(kFull, k < to && F[k] >= x);
        if (m) return base + __ffs(m) - 1;
    }
    return to;
}

// Largest k in [0, top] with F[k] <= x, or -1.
__device__ __forceinline__ int warp_last_leq(const double* F, int top, double x, int lane)
{
    for (; top >= 0; top -= 32) {
        const int k = top - lane;
        const unsigned m = __ballot_sync(kFull, k >= 0 && F[k] <= x);
        if (m) return top - (__ffs(m) - 1);
    }
    return -1;
}

// Largest k in [0, top] with F[k] < 0, or -1.
__device__ __forceinline__ int warp_last_negative(const double* F, int top, int lane)
{
    for (; top >= 0; top -= 32) {
        const int k = top - lane;
        const unsigned m = __ballot_sync(kFull, k >= 0 && F[k] < 0.0);
        if (m) return top - (__ffs(m) - 1);
    }
    return -1;
}

// Smallest k in [from, N) with F[k] > F[k + 1], or -1.
__device__ __forceinline__ int warp_first_descent(const double* F, int from, int N, int lane)
{
    for (int base = from; base < N; base += 32) {
        const int k = base + lane;
        const unsigned m = __ballot_sync(kFull, k < N && F[k] > F[k + 1]);
        if (m) return base + __ffs(m) - 1;
    }
    return -1;
}

// First index of the minimum of F over [from, to].
__device__ __forceinline__ int warp_argmin(const double* F, int from, int to, int lane)
{
    int best = -1;
    double bv = 0.0;
    for (int k = from + lane; k <= to; k += 32) {
        const double f = F[k];
        if (best < 0 || f < bv) {
            best = k;
            bv = f;
        }
    }
    for (int o = 16; o; o >>= 1) {
        const int ob = __shfl_xor_sync(kFull, best, o);
        const double ov = __shfl_xor_sync(kFull, bv, o);
        if (ob >= 0 && (best < 0 || ov < bv || (ov == bv && ob < best))) {
            best = ob;
            bv = ov;
        }
    }
    return best;
}

// Lane 0 extends the running sum S = F[s_k] + F[s_k + 1] + ... (left to right) up to each of the
// cnt candidates k_+ = base, base + 1, ..., storing the sum below each in Sc[l].
__device__ __forceinline__ void running_sums(const double* F, int base, int cnt, double& S, int& s_k, double* Sc,
                                             int lane)
{
    if (lane == 0)
        for (int l = 0; l < cnt; ++l) {
            for (; s_k < base + l; ++s_k) S = add_(S, F[s_k]);
            Sc[l] = S;
        }
    __syncwarp();
}

// Edge reconstruction of the entries below 0 of F (Appendix C): with k0 the largest index where
// F < 0, a ramp (k - k_-) dF on [k_-, k_+) (zero below) whose slope keeps the sum of F below
// k_+ (the histogram's first moment); the range grows (k_- down from k0 - 1 to 0, then k_+ up
// with k_- back at k0 - 1) until 0 <= (k_+ - k_- - 1) dF <= F[k_+]. Returns 1 (on every lane)
// if none exists.
// The test's top (L - 1) dF is 2 S / L up to rounding (L = k_+ - k_-, S the sum below k_+),
// smallest at k_- = 0: where it clearly exceeds F[k_+] there (relative margin 1e-12, far
// beyond the rounding) no k_- passes, and that k_+ is skipped without its scan.
__device__ int edge_low_warp(int N, double* F, double* Sc, int lane)
{
    const int k0 = warp_last_negative(F, N, lane);
    if (k0 < 0) return 0;
    const int hi = k0 - 1;  // first k_- of each scan
    if (hi < 0) return 1;
    auto top_of = [](double S, int km, int kp, double& dF) {
        const double L = (double)(kp - km);
        dF = div_(mul_(2.0, S), mul_(L, sub_(L, 1.0)));
        return mul_(sub_(L, 1.0), dF);
    };
    double S = 0.0;  // lane 0: F[0] + ... + F[s_k - 1]
    int s_k = 0;
    for (int base = k0 + 1; base <= N; base += 32) {
        const int cnt = min(32, N + 1 - base);
        running_sums(F, base, cnt, S, s_k, Sc, lane);
        // candidates k_+ = base + lane: can any k_- pass?
        bool cand = false;
        if (lane < cnt) {
            const int kp = base + lane;
            const double s = Sc[lane];
            double dF;
            if (s > 0.0) {
                const double t0 = top_of(s, 0, kp, dF);
                cand = (t0 >= 0.0 && t0 <= F[kp]) || !(t0 > F[kp] * (1.0 + 1e-12) + 1e-300);
            } else if (s == 0.0) {
                const double t = top_of(s, hi, kp, dF);
                cand = t >= 0.0 && t <= F[kp];
            }
        }
        unsigned m = __ballot_sync(kFull, cand);
        while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1;
            const int kp = base + l;
            const double s = Sc[l];
            // the scan k_- = hi, hi - 1, ..., 0: the first that passes
            int km = -1;
            for (int top = hi; top >= 0 && km < 0; top -= 32) {
                const int k = top - lane;
                bool ok = false;
                if (k >= 0) {
                    double dF;
                    const double t = top_of(s, k, kp, dF);
                    ok = t >= 0.0 && t <= F[kp];
                }
                const unsigned mk = __ballot_sync(kFull, ok);
                if (mk) km = top - (__ffs(mk) - 1);
            }
            if (km >= 0) {
                double dF;
                top_of(s, km, kp, dF);
                for (int k = lane; k < kp; k += 32) F[k] = k < km ? 0.0 : mul_((double)(k - km), dF);
                __syncwarp();
                return 0;
            }
        }
        __syncwarp();  // Sc is rewritten by the next chunk
    }
    return 1;
}

// Interior reconstruction from the low indices (Appendix C), descent after descent: at the
// first descent k0 (F[k0] > F[k0 + 1]; the search resumes at the previous k_-), k1 is the first
// later index with F[k1] >= F[k0] (or N), k_+ the first minimum on (k0, k1], k_- the last
// earlier index with F <= F[k_+] (or 0); a ramp F[k_-] + (k - k_-) dF on (k_-, k_+) keeps the
// sum of F over [k_-, k_+); k_+ grows until dF >= 0 and the ramp ends at or below F[k_+]. A
// descent with no admissible range is filled by a running max and 1 is returned (on every lane).
__device__ int interior_fwd_warp(int N, double* F, double* Sc, int lane)
{
    int bad = 0, start = 0;
    for (;;) {
        const int k0 = warp_first_descent(F, start, N, lane);
        if (k0 < 0) return bad;
        const int k1 = warp_first_geq(F, k0 + 1, N, F[k0], lane);
        const int kmin = warp_argmin(F, k0 + 1, k1, lane);
        const int kl = warp_last_leq(F, k0 - 1, F[kmin], lane);
        const int km = kl < 0 ? 0 : kl;
        const double Fkm = F[km];
        double S = 0.0;  // lane 0: F[km] + ... + F[s_k - 1]
        int s_k = km;
        int found = -1;
        double dF_found = 0.0;
        for (int base = kmin, chunk = 8; base <= N && found < 0; base += chunk, chunk = 32) {
            const int cnt = min(chunk, N + 1 - base);
            running_sums(F, base, cnt, S, s_k, Sc, lane);
            bool ok = false;
            double dF = 0.0;
            if (lane < cnt) {
                const int kp = base + lane;
                const double L = (double)(kp - km);
                dF = mul_(div_(2.0, sub_(L, 1.0)), sub_(div_(Sc[lane], L), Fkm));
                const double end = add_(Fkm, mul_(sub_(L, 1.0), dF));
                ok = dF >= 0.0 && end <= F[kp];
            }
            const unsigned m = __ballot_sync(kFull, ok);
            if (m) {
                const int l = __ffs(m) - 1;
                found = base + l;
                dF_found = __shfl_sync(kFull, dF, l);
            }
            __syncwarp();  // Sc is rewritten by the next chunk
        }
        if (found >= 0) {
            for (int k = km + 1 + lane; k < found; k += 32) F[k] = add_(Fkm, mul_((double)(k - km), dF_found));
        } else {
            bad = 1;
            if (lane == 0)
                for (int k = k0 + 1; k <= N; ++k)
                    if (F[k] < F[k - 1]) F[k] = F[k - 1];
        }
        __syncwarp();
        start = km;
    }
}

// G[k] = 1 - F[N - k] over the warp.
__device__ __forceinline__ void mirror_warp(int N, const double* F, double* G, int lane)
{
    for (int k = lane; k <= N; k += 32) G[k] = sub_(1.0, F[N - k]);
    __syncwarp();
}

}  // namespace
}  // namespace pe

namespace pe {
namespace {

// Synchronises the two warps of bin slot q of the block (named barrier 1 + q, 64 threads).
__device__ __forceinline__ void pair_sync(int q)
{
    asm volatile("bar.sync %0, 64;" ::"r"(1 + q) : "memory");
}

// Lifting tables, two warps per bin: the raw mass, the reconstructed FP64 CDF row (uniform
// where the raw mass is not positive), and the FP32 sampling row used by the particle loader:
// F[0..nv], the inverse cell masses 1 / (F[k+1] - F[k]) (0 for an empty cell) and the cells'
// relative density slopes sigma_k = (p_{k+1} - p_{k-1}) / (4 p_k) clamped to [-1, 1].
// The reconstruction (Appendix C) works on three rows per bin in shared memory (plus 32 slots
// of running sums per warp): the running sum of the masses is one serial chain (lane 0 of the
// first warp, left to right) and the edges are fixed by the first warp; the two interior
// passes (on P and on the mirror G) run one per warp; the divisions, mirrors, searches,
// candidate tests and stores are spread over the lanes. Every element gets the FP64 operations
// (each rounded separately) of a serial host evaluation, so the CDF rows are reproducible bit
// for bit.
__global__ void __launch_bounds__(256) k_ps_cdf(const double* __restrict__ H, int nxc, int nv,
                                               double* __restrict__ mass, double* __restrict__ cdf,
                                               float* __restrict__ table, int32_t* __restrict__ flags)
{
    extern __shared__ double rows[];
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 6, half = (threadIdx.x >> 5) & 1;
    const int t64 = threadIdx.x & 63;
    const int i = blockIdx.x * (blockDim.x >> 6) + q;
    if (i >= nxc) return;  // whole pairs of warps
    const int N = nv;
    double* F = rows + (size_t)q * (3 * (N + 1) + 66);
    double* G = F + N + 1;
    double* P = G + N + 1;
    double* Sc = P + N + 1 + 32 * half;        // this warp's running sums
    double* shared_s = P + N + 1 + 64;         // the mass, for the second warp
    int* shared_bad = reinterpret_cast<int*>(shared_s + 1);
    const double* h = H + (size_t)i * nv;
    for (int j = t64; j < nv; j += 64) P[j] = h[j];
    if (t64 == 0) *shared_bad = 0;
    pair_sync(q);
    // running sum r_j = h_0 + ... + h_j from 0.0, left to right; its last value is the mass
    if (t64 == 0) {
        double r = 0.0;
        for (int j = 0; j < nv; ++j) {
            r = add_(r, P[j]);
            F[j + 1] = r;
        }
        *shared_s = r;
        mass[i] = r;
    }
    pair_sync(q);
    const double s = *shared_s;
    if (s > 0.0) {
        for (int k = t64; k <= N; k += 64) F[k] = k == 0 ? 0.0 : (k == N ? 1.0 : div_(F[k], s));
        pair_sync(q);
        if (half == 0) {
            // edges: the low one, then the high one as the low edge of the mirror
            int bad = edge_low_warp(N, F, Sc, lane);
            mirror_warp(N, F, G, lane);
            bad |= edge_low_warp(N, G, Sc, lane);
            mirror_warp(N, G, F, lane);
            for (int k = lane; k <= N; k += 32) {
                double f = F[k];
                if (bad) f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
                F[k] = f;
                P[k] = f;
            }
            __syncwarp();
            mirror_warp(N, F, G, lane);
            if (bad && lane == 0) *shared_bad = 1;
        }
        pair_sync(q);
        // interior: forward on P (first warp) and on the mirror G (the high indices, second warp)
        const int bad = interior_fwd_warp(N, half == 0 ? P : G, Sc, lane);
        if (bad && lane == 0) atomicOr(shared_bad, 1);
        pair_sync(q);
        for (int k = t64; k <= N; k += 64) F[k] = mul_(0.5, add_(P[k], sub_(1.0, G[N - k])));
        if (t64 == 0 && *shared_bad && flags) atomicOr(flags, 1);
    } else {
        for (int k = t64; k <= N; k += 64) F[k] = div_((double)k, (double)nv);
    }
    pair_sync(q);
    double* out = cdf + (size_t)i * (nv + 1);
    float* T = table + (size_t)i * (3 * nv + 1);
    for (int k = t64; k <= N; k += 64) {
        out[k] = F[k];
        T[k] = (float)F[k];
    }
    // sampling rows: one FP64 reciprocal per cell (the slope's division by 4 p_k as a product
    // with it; both are rounded to FP32)
    for (int k = t64; k < nv; k += 64) {
        const double p = F[k + 1] - F[k];
        const double pl = k > 0 ? F[k] - F[k - 1] : 0.0, pr = k + 1 < nv ? F[k + 2] - F[k + 1] : 0.0;
        const double r = p > 0.0 ? 1.0 / p : 0.0;
        const double sg = (pr - pl) * (0.25 * r);
        T[nv + 1 + k] = (float)r;
        T[2 * nv + 1 + k] = (float)(sg > 1.0 ? 1.0 : (sg < -1.0 ? -1.0 : sg));
    }
}

// Negative masses clamped to 0, the others rescaled to keep the total (summed by one thread
// in bin order, as the host evaluation does). The masses are staged in shared memory a block
// at a time, so the serial sums wait on FP64 adds only, not on global loads.
__global__ void __launch_bounds__(1024) k_ps_mass(int nxc, double* __restrict__ mass)
{
    __shared__ double stage[1024];
    __shared__ double sscale;
    double tot = 0.0, pos = 0.0;
    for (int i0 = 0; i0 < nxc; i0 += blockDim.x) {
        const int n = min((int)blockDim.x, nxc - i0);
        if ((int)threadIdx.x < n) stage[threadIdx.x] = mass[i0 + threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 0; i < n; ++i) {
                const double m = stage[i];
                tot = add_(tot, m);
                pos = add_(pos, m > 0.0 ? m : 0.0);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) sscale = pos > 0.0 ? div_(tot, pos) : 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < nxc; i += blockDim.x) mass[i] = mass[i] > 0.0 ? mul_(mass[i], sscale) : 0.0;
}

struct PSLoad {
    int32_t* cell;
    float* theta;
    float* v;
    float* w;
    int64_t n, chunk;
    uint32_t ppc;
    int log2ppc, ncell, mask, bin_shift, nv;
    float per_node, vmin, dv, inv_ppc, two_ppc, inv_two_ppc;
    const double* mass;
    const float* table;
    const float* node_dens;  // wavelet form: per fine node density and sampling row (else null)
    int stage_rows;          // wavelet form: fine-node rows staged in shared memory per block
    uint32_t half, shift;
    float wscale;
    unsigned long long* rho;
    int rho_width;
    uint32_t* status;
};

template <bool LDG>
__device__ __forceinline__ float ld_row(const float* p)
{
    if (LDG) return __ldg(p);
    return *p;
}

// First index k in [lo, nv - 1] with T[k + 1] > b (nv - 1 if none), for a row T[0..nv] that is
// non-decreasing, given that no index below lo qualifies (lo = 0 for a fresh search): the two
// indices from lo are tried first (consecutive quantiles of a velocity-ordered cell land in the
// same or the next cells), then the rest is bisected. The result is the full bisection's.
template <bool LDG>
__device__ __forceinline__ int cdf_search(const float* T, int nv, float b, int lo)
{
    int hi = nv - 1;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (lo < hi) {
            if (ld_row<LDG>(T + lo + 1) > b) return lo;
            ++lo;
        }
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ld_row<LDG>(T + mid + 1) > b)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// Search state of one lane across its particles: the rows last searched, the indices found
// and the quantile they were found for. A later search of the same row for a quantile at or
// above it starts from the index found (no lower index qualifies, the row being
// non-decreasing); any other search starts from 0.
struct SearchHint {
    const float* row0;
    const float* row1;
    int k0, k1;
    float b;

    __device__ __forceinline__ void reset()
    {
        row0 = row1 = nullptr;
        k0 = k1 = 0;
        b = 0.0f;
    }
    __device__ __forceinline__ int start(const float* T, float bq) const
    {
        if (bq < b) return 0;
        return T == row0 ? k0 : (T == row1 ? k1 : 0);
    }
};

// V = v_min + dv (k + t) on a bin's FP32 sampling row: k the first index with F[k+1] > b
// (nv - 1 if none; cdf_search from lo0), t the position inside the cell where the cell's
// linear density reaches the fraction r = (b - F[k]) / (F[k+1] - F[k]) of its mass.
__device__ __forceinline__ float cdf_inverse_f(const float* __restrict__ T, int nv, float b, float vmin, float dv,
                                               int lo0 = 0, int* found = nullptr)
{
    const int lo = cdf_search<true>(T, nv, b, lo0);
    if (found) *found = lo;
    const float f0 = __ldg(T + lo), sl = __ldg(T + nv + 1 + lo), sg = __ldg(T + 2 * nv + 1 + lo);
    const float r = sl > 0.0f ? fminf(fmaxf((b - f0) * sl, 0.0f), 1.0f) : 0.5f;
    // linear density 1 + sigma (2t - 1) inside the cell: t solves t + sigma (t^2 - t) = r
    const float om = 1.0f - sg;
    const float den = om + sqrtf(fmaxf(fmaf(om, om, 4.0f * sg * r), 0.0f));
    const float t = den > 0.0f ? fminf(2.0f * r / den, 1.0f) : 0.0f;  // den = 0 only for sigma = 1, r = 0
    return fmaf(dv, (float)lo + t, vmin);
}

// Appendix C loading of slot i: the Hammersley point and storage order of pe_quiet_start;
// the lifted f(x, v) is linear in x between neighbouring bin centres (Section 3.3's linear
// interpolation): weight n(X)/ppc and velocity quantile blended between the two bins around
// the particle. A piecewise-constant (Haar) lift would give the density steps at bin edges,
// and the field spikes there, multiplied by the co-moving time tau ~ Delta t, spread the next
// restriction sample in velocity. FP32 (the particle precision) on tables built in FP64.
// Inverse of a row with uniform density inside each cell (F[0..nv], then the inverse cell
// masses): v_min + dv (k + r), k the first index with F[k+1] > b, r = (b - F[k]) / p_k.
__device__ __forceinline__ float cdf_inverse_lin(const float* T, int nv, float b, float vmin, float dv, int lo0,
                                                 int* found)
{
    const int lo = cdf_search<false>(T, nv, b, lo0);
    *found = lo;
    const float f0 = T[lo], sl = T[nv + 1 + lo];
    const float r = sl > 0.0f ? fminf(fmaxf((b - f0) * sl, 0.0f), 1.0f) : 0.5f;
    return fmaf(dv, (float)lo + r, vmin);
}

// Fine-node rows of the block's cells staged in shared memory (rows c_stage .. c_stage + n - 1,
// 2 nv + 1 floats each); other nodes read the global table.
struct NodeStage {
    const float* rows;
    int c_stage, n;
};

__device__ __forceinline__ void ps_load_one(const PSLoad& P, const NodeStage& ns, SearchHint& hint, uint32_t i,
                                            int& c, float& th, float& vv, float& ww)
{
    if (P.log2ppc > 0) {
        const uint32_t k = i & (P.ppc - 1u);
        i = (i & ~(P.ppc - 1u)) | (__brev(k) >> (32 - P.log2ppc));
    }
    uint32_t j;
    if (P.log2ppc >= 0) {  // ppc = 2^m: shifts, and theta scaled by the exact 1 / (2 ppc)
        j = i & (P.ppc - 1u);
        c = (int)(i >> P.log2ppc);
        th = (float)(2u * j + 1u) * P.inv_two_ppc;
    } else {
        j = i % P.ppc;
        c = (int)(i / P.ppc);
        th = __fdiv_rn((float)(2u * j + 1u), P.two_ppc);
    }
    if (P.node_dens) {
        // wavelet form: the fine nodes c and c + 1 carry their own density and sampling row
        // (k_ps_node_tables); weight and velocity are linear in x between them
        const int c1 = (c + 1) & P.mask;
        const float d0 = __ldg(P.node_dens + c), d1 = __ldg(P.node_dens + c1);
        ww = fmaf(th, d1 - d0, d0) * P.inv_ppc;
        const uint32_t B = __brev(i) + P.half + P.shift;
        const float b = fmaf(__uint2float_rn(B), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
        const int row = 3 * P.nv + 1, srow = 2 * P.nv + 1;
        const int r0 = (c - ns.c_stage) & P.mask, r1 = (c1 - ns.c_stage) & P.mask;
        const float* T0 = r0 < ns.n ? ns.rows + r0 * srow : P.table + (size_t)c * row;
        const float* T1 = r1 < ns.n ? ns.rows + r1 * srow : P.table + (size_t)c1 * row;
        int k0, k1;
        const float v0 = cdf_inverse_lin(T0, P.nv, b, P.vmin, P.dv, hint.start(T0, b), &k0);
        const float v1 = cdf_inverse_lin(T1, P.nv, b, P.vmin, P.dv, hint.start(T1, b), &k1);
        hint = SearchHint{T0, T1, k0, k1, b};
        vv = fmaf(th, v1 - v0, v0);
        return;
    }
    // linear in x between neighbouring bin centres: phi is the distance from the centre of
    // bin b0 (at or left of the particle) in bin widths
    // (a bin sums the CIC charge of its 2^b nodes: it covers x/dx in [i 2^b - 1/2, (i+1) 2^b - 1/2))
    const int nxc_mask = ((P.mask + 1) >> P.bin_shift) - 1;
    float t = th + 0.5f;
    int cc = c;
    if (t >= 1.0f) {
        t -= 1.0f;
        cc = (c + 1) & P.mask;
    }
    const int bin = cc >> P.bin_shift;
    const float pos = ((float)(cc & ((1 << P.bin_shift) - 1)) + t) * P.per_node;
    int b0, b1;
    float phi;
    if (pos >= 0.5f) {
        b0 = bin;
        b1 = (bin + 1) & nxc_mask;
        phi = pos - 0.5f;
    } else {
        b0 = (bin - 1) & nxc_mask;
        b1 = bin;
        phi = pos + 0.5f;
    }
    const float n0 = (float)__ldg(P.mass + b0), n1 = (float)__ldg(P.mass + b1);
    ww = fmaf(phi, n1 - n0, n0) * P.per_node * P.inv_ppc;
    const uint32_t B = __brev(i) + P.half + P.shift;
    const float b = fmaf(__uint2float_rn(B), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const int row = 3 * P.nv + 1;
    const float* T0 = P.table + (size_t)b0 * row;
    const float* T1 = P.table + (size_t)b1 * row;
    int k0, k1;
    const float v0 = cdf_inverse_f(T0, P.nv, b, P.vmin, P.dv, hint.start(T0, b), &k0);
    float v1 = v0;
    k1 = k0;
    if (b1 != b0) v1 = cdf_inverse_f(T1, P.nv, b, P.vmin, P.dv, hint.start(T1, b), &k1);
    hint = SearchHint{T0, T1, k0, k1, b};
    vv = fmaf(phi, v1 - v0, v0);
}

__global__ void __launch_bounds__(256) k_ps_quiet_start(PSLoad P)
{
    extern __shared__ uint32_t smem[];
    int64_t begin, end;
    block_chunk(P.n, P.chunk, &begin, &end);
    const bool dep = P.rho != nullptr;
    const int c_first = (begin < end) ? (int)((uint64_t)begin / P.ppc) : 0;
    SmemGrid grho{};
    uint32_t* s = smem;
    if (dep) {
        s = grho.bind(s, P.rho, P.rho_width < P.ncell ? ((c_first - 64) & P.mask) : 0, P.rho_width, P.mask);
        grho.zero();
    }
    NodeStage ns{nullptr, 0, 0};
    if (P.node_dens && P.stage_rows > 0) {
        float* st = reinterpret_cast<float*>(s);
        const int rw = 2 * P.nv + 1;
        for (int i = threadIdx.x; i < P.stage_rows * rw; i += blockDim.x) {
            const int r = i / rw, k = i - r * rw;
            st[i] = __ldg(P.table + (size_t)((c_first + r) & P.mask) * (3 * P.nv + 1) + k);
        }
        ns = NodeStage{st, c_first, P.stage_rows};
    }
    __syncthreads();
    const int64_t gb0 = begin >> 2, gb1 = end >> 2;
    int64_t g0, g1;
    warp_groups(gb0, gb1, &g0, &g1);
    LaneWindow lw;
    lw.reset(((int)((uint64_t)(g0 << 2) / P.ppc) - 1) & P.mask);
    bool ovf = false;
    int4* cell4 = reinterpret_cast<int4*>(P.cell);
    float4* th4 = reinterpret_cast<float4*>(P.theta);
    float4* v4 = reinterpret_cast<float4*>(P.v);
    float4* w4 = reinterpret_cast<float4*>(P.w);
    SearchHint hint;
    hint.reset();
    for (int64_t g = g0 + (threadIdx.x & 31); g < g1; g += 32) {
        int4 c;
        float4 t, vv, ww;
        const uint32_t i0 = (uint32_t)(g << 2);
        ps_load_one(P, ns, hint, i0, c.x, t.x, vv.x, ww.x);
        ps_load_one(P, ns, hint, i0 + 1, c.y, t.y, vv.y, ww.y);
        ps_load_one(P, ns, hint, i0 + 2, c.z, t.z, vv.z, ww.z);
        ps_load_one(P, ns, hint, i0 + 3, c.w, t.w, vv.w, ww.w);
        cell4[g] = c;
        th4[g] = t;
        v4[g] = vv;
        w4[g] = ww;
        if (dep) {
            lw.add(c.x, fx_split(fx_weight_q(ww.x, P.wscale, &ovf), t.x), grho);
            lw.add(c.y, fx_split(fx_weight_q(ww.y, P.wscale, &ovf), t.y), grho);
            lw.add(c.z, fx_split(fx_weight_q(ww.z, P.wscale, &ovf), t.z), grho);
            lw.add(c.w, fx_split(fx_weight_q(ww.w, P.wscale, &ovf), t.w), grho);
        }
    }
    for (int64_t i = (gb1 << 2) + threadIdx.x; i < end; i += blockDim.x) {
        int c;
        float t, vv, ww;
        ps_load_one(P, ns, hint, (uint32_t)i, c, t, vv, ww);
        P.cell[i] = c;
        P.theta[i] = t;
        P.v[i] = vv;
        P.w[i] = ww;
        if (dep) lw.add(c, fx_split(fx_weight_q(ww, P.wscale, &ovf), t), grho);
    }
    if (dep) lw.flush(grho);
    if (ovf) raise_flag(P.status, PE_FLAG_OVERFLOW);
    __syncthreads();
    if (dep) grho.flush();
}

// Wavelet-form loading when ppc = 2^m, m >= 2: the same slots, values and deposit as
// k_ps_quiet_start on fine-node tables, with the work a lane's group of four slots shares done
// once. The four slots lie in one cell c (ppc a multiple of four), so they share the nodes'
// densities and sampling rows; their quantiles increase with the slot inside the cell (the
// slot's bit-reversed position index gives the Hammersley point), so each row's search resumes
// from the previous slot's index until the quantile wraps around.
__device__ __forceinline__ const float* node_row(const PSLoad& P, const NodeStage& ns, int c)
{
    const int r = (c - ns.c_stage) & P.mask;
    return r < ns.n ? ns.rows + r * (2 * P.nv + 1) : P.table + (size_t)c * (3 * P.nv + 1);
}

__global__ void __launch_bounds__(256) k_ps_quiet_start_nodes(PSLoad P)
{
    extern __shared__ uint32_t smem[];
    int64_t begin, end;
    block_chunk(P.n, P.chunk, &begin, &end);
    const int m = P.log2ppc;
    const int c_first = (begin < end) ? (int)((uint64_t)begin >> m) : 0;
    SmemGrid grho{};
    uint32_t* s = smem;
    const bool dep = P.rho != nullptr;
    if (dep) {
        s = grho.bind(s, P.rho, P.rho_width < P.ncell ? ((c_first - 64) & P.mask) : 0, P.rho_width, P.mask);
        grho.zero();
    }
    NodeStage ns{nullptr, 0, 0};
    if (P.stage_rows > 0) {
        float* st = reinterpret_cast<float*>(s);
        const int rw = 2 * P.nv + 1;
        for (int i = threadIdx.x; i < P.stage_rows * rw; i += blockDim.x) {
            const int r = i / rw, k = i - r * rw;
            st[i] = __ldg(P.table + (size_t)((c_first + r) & P.mask) * (3 * P.nv + 1) + k);
        }
        ns = NodeStage{st, c_first, P.stage_rows};
    }
    __syncthreads();
    const int64_t gb0 = begin >> 2, gb1 = end >> 2;  // ppc >= 4 divides n: no ragged tail
    int64_t g0, g1;
    warp_groups(gb0, gb1, &g0, &g1);
    LaneWindow lw;
    lw.reset(((int)((uint64_t)(g0 << 2) >> m) - 1) & P.mask);
    bool ovf = false;
    int c_prev = -1;
    int k0 = 0, k1 = 0;
    float b_prev = 2.0f;
    for (int64_t g = g0 + (threadIdx.x & 31); g < g1; g += 32) {
        const uint32_t i0 = (uint32_t)(g << 2);
        const int c = (int)(i0 >> m), c1 = (c + 1) & P.mask;
        const uint32_t kin = i0 & (P.ppc - 1u);
        const float d0 = __ldg(P.node_dens + c), d1 = __ldg(P.node_dens + c1);
        const float* T0 = node_row(P, ns, c);
        const float* T1 = node_row(P, ns, c1);
        if (c != c_prev) {  // a new cell: the searches start over
            c_prev = c;
            b_prev = 2.0f;
        }
        float th[4], vq[4], wq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t j = __brev(kin + (uint32_t)q) >> (32 - m);
            th[q] = (float)(2u * j + 1u) * P.inv_two_ppc;
            wq[q] = fmaf(th[q], d1 - d0, d0) * P.inv_ppc;
            const uint32_t B = __brev(((uint32_t)c << m) | j) + P.half + P.shift;
            const float b = fmaf(__uint2float_rn(B), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
            if (b < b_prev) k0 = k1 = 0;  // the quantile wrapped (or a new cell)
            b_prev = b;
            const float v0 = cdf_inverse_lin(T0, P.nv, b, P.vmin, P.dv, k0, &k0);
            const float v1 = cdf_inverse_lin(T1, P.nv, b, P.vmin, P.dv, k1, &k1);
            vq[q] = fmaf(th[q], v1 - v0, v0);
        }
        reinterpret_cast<int4*>(P.cell)[g] = make_int4(c, c, c, c);
        reinterpret_cast<float4*>(P.theta)[g] = make_float4(th[0], th[1], th[2], th[3]);
        reinterpret_cast<float4*>(P.v)[g] = make_float4(vq[0], vq[1], vq[2], vq[3]);
        reinterpret_cast<float4*>(P.w)[g] = make_float4(wq[0], wq[1], wq[2], wq[3]);
        if (dep) {
#pragma unroll
            for (int q = 0; q < 4; ++q) lw.add(c, fx_split(fx_weight_q(wq[q], P.wscale, &ovf), th[q]), grho);
        }
    }
    if (dep) lw.flush(grho);
    if (ovf) raise_flag(P.status, PE_FLAG_OVERFLOW);
    __syncthreads();
    if (dep) grho.flush();
}

// Wavelet form, lifting in x (Eq. interpolation) at the fine nodes: fine node j lies phi =
// (j mod 2^b) / 2^b of the way from coarse node i0 = j >> b to i1 = i0 + 1 (periodic); its
// histogram is the linear interpolation (1 - phi) H_i0 + phi H_i1 of the reconstructed
// coarse-node histograms, so its density is a0 + a1 (a0 = (1 - phi) mass[i0], a1 = phi
// mass[i1]) and its CDF the mixture (a0 F_i0 + a1 F_i1) / (a0 + a1). One block per fine node
// writes the FP32 sampling row of cdf_inverse_f (CDF, inverse cell masses, zero slopes: the
// density is uniform inside a velocity cell, Appendix C's lookup with linear interpolation),
// evaluated in FP64, and the node density. The mixture is scaled by one FP64 reciprocal of the
// density per node (FP64 divisions are slow on this GPU) and each CDF value is formed once, in
// shared memory, for both of its neighbouring cells; the inverse cell masses are FP32
// reciprocals of the FP64 differences (both roundings are below the FP32 table's resolution).
__global__ void __launch_bounds__(256) k_ps_node_tables(const double* __restrict__ mass, const double* __restrict__ cdf,
                                                        int nxc, int bin_shift, int nv, float* __restrict__ table,
                                                        float* __restrict__ dens)
{
    extern __shared__ double gs[];  // nv + 1 CDF values of this node
    const int j = blockIdx.x;
    const int i0 = j >> bin_shift, i1 = (i0 + 1) & (nxc - 1);
    const double phi = ldexp((double)(j & ((1 << bin_shift) - 1)), -bin_shift);
    const double a0 = (1.0 - phi) * mass[i0], a1 = phi * mass[i1], tot = a0 + a1;
    const double inv = tot > 0.0 ? 1.0 / tot : 0.0, inv_nv = 1.0 / (double)nv;
    const double* F0 = cdf + (size_t)i0 * (nv + 1);
    const double* F1 = cdf + (size_t)i1 * (nv + 1);
    float* T = table + (size_t)j * (3 * nv + 1);
    for (int k = threadIdx.x; k <= nv; k += blockDim.x) {
        const double g = tot > 0.0 ? (a0 * F0[k] + a1 * F1[k]) * inv : (double)k * inv_nv;
        gs[k] = g;
        T[k] = (float)g;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        const double d = gs[k + 1] - gs[k];
        T[nv + 1 + k] = d > 0.0 ? __frcp_rn((float)d) : 0.0f;
        T[2 * nv + 1 + k] = 0.0f;
    }
    if (threadIdx.x == 0) dens[j] = (float)tot;
}

// Least-squares slope of every phase-space cell (Eq. leastsquares), into raw[nxc][nv].
__global__ void k_ps_slope(const double* __restrict__ c, int K, int n, double dt, double* __restrict__ raw)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double den = (double)K * (K + 1) * (K + 2) * dt;
    double s = 0.0;
    for (int p = 0; 2 * p <= K; ++p) s += 6.0 * (K - 2 * p) / den * (c[(size_t)(K - p) * n + i] - c[(size_t)p * n + i]);
    raw[i] = s;
}

// Filtered slope (1/4, 1/2, 1/4 along v and/or x) and the leap c_K + (dT - K dt) slope.
__global__ void k_ps_leap(const double* __restrict__ c, const double* __restrict__ raw, int K, int nxc, int nv,
                          double leap, int filter, double* __restrict__ out, double* __restrict__ slope)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nxc * nv) return;
    const int i = idx / nv, j = idx - i * nv;
    auto at = [&](int ii, int jj) -> double {
        if (jj < 0 || jj >= nv) return 0.0;
        if (filter & 4)  // bounded grid: reflecting at the walls (keeps the sum)
            ii = ii < 0 ? 0 : (ii >= nxc ? nxc - 1 : ii);
        else
            ii = (ii + nxc) % nxc;
        return raw[(size_t)ii * nv + jj];
    };
    auto vfilt = [&](int ii) -> double {
        return (filter & 1) ? 0.25 * at(ii, j - 1) + 0.5 * at(ii, j) + 0.25 * at(ii, j + 1) : at(ii, j);
    };
    const double s = (filter & 2) ? 0.25 * vfilt(i - 1) + 0.5 * vfilt(i) + 0.25 * vfilt(i + 1) : vfilt(i);
    slope[idx] = s;
    out[idx] = c[(size_t)K * nxc * nv + idx] + leap * s;
}

__global__ void k_ps_scale(const long long* __restrict__ src, int64_t n, double scale, double* __restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i] * scale;
}

// ---- bounded grid: equal-weight loading of the phase-space tables
// Bin i sums the CIC charge of its 2^b nodes, x/dx in [i 2^b - 1/2, (i+1) 2^b - 1/2), cut to
// the domain [0, ncell - 1]: the first and last bins are half a node narrower. The lifted
// density in x is linear between the bins' span midpoints, mass_i / width_i there, constant
// beyond the first and last midpoints.
__device__ __forceinline__ double ps_mid(int i, int nxc, double width, int ncell)
{
    if (i == 0) return 0.5 * (width - 0.5);
    if (i == nxc - 1) return 0.5 * ((nxc - 1) * width - 0.5 + (double)(ncell - 1));
    return (i + 0.5) * width - 0.5;
}

// Bins b0 <= b1 whose midpoints bracket x (in nodes) and the fraction phi of the way.
__device__ __forceinline__ void ps_bracket(double x, int nxc, double width, int ncell, int& b0, int& b1, double& phi)
{
    if (nxc < 2 || x <= ps_mid(0, nxc, width, ncell)) {
        b0 = b1 = 0;
        phi = 0.0;
        return;
    }
    if (x >= ps_mid(nxc - 1, nxc, width, ncell)) {
        b0 = b1 = nxc - 1;
        phi = 0.0;
        return;
    }
    int i = (int)floor((x + 0.5) / width - 0.5);
    i = i < 0 ? 0 : (i > nxc - 2 ? nxc - 2 : i);
    while (i > 0 && x < ps_mid(i, nxc, width, ncell)) --i;
    while (i < nxc - 2 && x >= ps_mid(i + 1, nxc, width, ncell)) ++i;
    const double m0 = ps_mid(i, nxc, width, ncell), m1 = ps_mid(i + 1, nxc, width, ncell);
    b0 = i;
    b1 = i + 1;
    phi = (x - m0) / (m1 - m0);
}

// FP32 form of ps_bracket for the per-ion blend (the interior midpoints are a power-of-two
// width apart; the end midpoints are passed in).
__device__ __forceinline__ void ps_bracket_f(float x, int nxc, float width, float inv_width, float mid_first,
                                             float mid_last, int& b0, int& b1, float& phi)
{
    if (nxc < 2 || x <= mid_first) {
        b0 = b1 = 0;
        phi = 0.0f;
        return;
    }
    if (x >= mid_last) {
        b0 = b1 = nxc - 1;
        phi = 0.0f;
        return;
    }
    auto mid = [&](int i) {
        return i == 0 ? mid_first : (i == nxc - 1 ? mid_last : fmaf((float)i + 0.5f, width, -0.5f));
    };
    int i = (int)floorf(fmaf(x + 0.5f, inv_width, -0.5f));
    i = i < 0 ? 0 : (i > nxc - 2 ? nxc - 2 : i);
    if (i > 0 && x < mid(i)) --i;
    if (i < nxc - 2 && x >= mid(i + 1)) ++i;
    const float m0 = mid(i), m1 = mid(i + 1);
    b0 = i;
    b1 = i + 1;
    phi = fminf(fmaxf((x - m0) / (m1 - m0), 0.0f), 1.0f);
}

// One block: the nodal profile prof[ncell] (FP64) of the bin densities, total = sum of the bin
// masses (fixed-order tree), and for the per-ion blend the FP32 bin densities densf[nxc] and the
// ion weight total / n.
__global__ void __launch_bounds__(1024) k_ps_profile(const double* __restrict__ mass, int nxc, int bin_shift,
                                                     int ncell, int64_t n, double* __restrict__ prof, double* total,
                                                     float* __restrict__ densf, float* wn)
{
    __shared__ double red[32];
    const double width = ldexp(1.0, bin_shift);
    for (int j = threadIdx.x; j < ncell; j += blockDim.x) {
        int b0, b1;
        double phi;
        ps_bracket((double)j, nxc, width, ncell, b0, b1, phi);
        const double w0 = (b0 == 0 || b0 == nxc - 1) ? width - 0.5 : width;
        const double w1 = (b1 == 0 || b1 == nxc - 1) ? width - 0.5 : width;
        prof[j] = (1.0 - phi) * (mass[b0] / w0) + phi * (mass[b1] / w1);
    }
    for (int i = threadIdx.x; i < nxc; i += blockDim.x)
        densf[i] = (float)(mass[i] / ((i == 0 || i == nxc - 1) ? width - 0.5 : width));
    double acc = 0.0;
    for (int i = threadIdx.x; i < nxc; i += blockDim.x) acc += mass[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            *total = v;
            *wn = (float)(v / (double)n);
        }
    }
}

struct PSEqLoad {
    int32_t* cell;
    float* theta;
    float* v;
    float* w;
    int64_t n, chunk;
    int ncell, mask, bin_shift, nv, nxc;
    float vmin, dv;
    const double* prof;
    const float* densf;
    const float* wn;
    float width, inv_width, mid_first, mid_last;
    EqTable tab;
    const float* table;
    uint32_t half, shift;
    float wscale;
    unsigned long long* rho;
    int rho_width;
    uint32_t* status;
};

__device__ __forceinline__ void ps_eq_one(const PSEqLoad& P, uint32_t i, int& c, float& th, float& vv, float& ww,
                                          EqCellCache& cache)
{
    const float t = eq_position(P.tab, P.prof, 1.0f, P.ncell, i, c, cache);
    th = t;
    int b0, b1;
    float phi;
    ps_bracket_f((float)c + t, P.nxc, P.width, P.inv_width, P.mid_first, P.mid_last, b0, b1, phi);
    float r0 = (1.0f - phi) * __ldg(P.densf + b0), r1 = phi * __ldg(P.densf + b1);
    if (!(r0 + r1 > 0.0f)) {
        // the cell's linear profile reaches past the midpoint interpolation's zero (next to an
        // empty bin): take the velocities at the cell's denser node
        const float x = (__ldg(P.prof + c + 1) > __ldg(P.prof + c)) ? (float)(c + 1) : (float)c;
        ps_bracket_f(x, P.nxc, P.width, P.inv_width, P.mid_first, P.mid_last, b0, b1, phi);
        r0 = (1.0f - phi) * __ldg(P.densf + b0);
        r1 = phi * __ldg(P.densf + b1);
    }
    const uint32_t B = __brev(i) + P.half + P.shift;
    const float b = fmaf(__uint2float_rn(B), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const int row = 3 * P.nv + 1;
    const float v0 = cdf_inverse_f(P.table + (size_t)b0 * row, P.nv, b, P.vmin, P.dv);
    const float v1 = (b1 == b0) ? v0 : cdf_inverse_f(P.table + (size_t)b1 * row, P.nv, b, P.vmin, P.dv);
    // quantiles blended by each bin's share of the density at x: a bin without ions (whose
    // table is a placeholder) contributes nothing
    const float f = (r0 + r1 > 0.0f) ? r1 / (r0 + r1) : phi;
    vv = fmaf(f, v1 - v0, v0);
    ww = __ldg(P.wn);
}

__global__ void __launch_bounds__(256) k_ps_quiet_start_equal(PSEqLoad P)
{
    extern __shared__ uint32_t smem[];
    int64_t begin, end;
    block_chunk(P.n, P.chunk, &begin, &end);
    const bool dep = P.rho != nullptr;
    const int c_first = (begin < end) ? eq_cell_of(P.tab, P.ncell, eq_point_of_slot((uint32_t)begin, P.n)) : 0;
    SmemGrid grho{};
    if (dep) {
        grho.bind(smem, P.rho, P.rho_width < P.ncell ? ((c_first - 64) & P.mask) : 0, P.rho_width, P.mask);
        grho.zero();
    }
    __syncthreads();
    const int64_t gb0 = begin >> 2, gb1 = end >> 2;
    int64_t g0, g1;
    warp_groups(gb0, gb1, &g0, &g1);
    LaneWindow lw;
    lw.reset((c_first - 1) & P.mask);
    EqCellCache cache;
    cache.reset();
    bool ovf = false;
    int4* cell4 = reinterpret_cast<int4*>(P.cell);
    float4* th4 = reinterpret_cast<float4*>(P.theta);
    float4* v4 = reinterpret_cast<float4*>(P.v);
    float4* w4 = reinterpret_cast<float4*>(P.w);
    for (int64_t g = g0 + (threadIdx.x & 31); g < g1; g += 32) {
        int4 c;
        float4 t, vv, ww;
        const uint32_t s0 = (uint32_t)(g << 2);
        const uint32_t p0 = eq_point_of_slot(s0, P.n), p1 = eq_point_of_slot(s0 + 1, P.n),
                       p2 = eq_point_of_slot(s0 + 2, P.n), p3 = eq_point_of_slot(s0 + 3, P.n);
        const int cb = eq_cell_of(P.tab, P.ncell, min(min(p0, p1), min(p2, p3)));
        c.x = c.y = c.z = c.w = cb;
        ps_eq_one(P, p0, c.x, t.x, vv.x, ww.x, cache);
        ps_eq_one(P, p1, c.y, t.y, vv.y, ww.y, cache);
        ps_eq_one(P, p2, c.z, t.z, vv.z, ww.z, cache);
        ps_eq_one(P, p3, c.w, t.w, vv.w, ww.w, cache);
        cell4[g] = c;
        th4[g] = t;
        v4[g] = vv;
        w4[g] = ww;
        if (dep) {
            lw.add(c.x, fx_split(fx_weight_q(ww.x, P.wscale, &ovf), t.x), grho);
            lw.add(c.y, fx_split(fx_weight_q(ww.y, P.wscale, &ovf), t.y), grho);
            lw.add(c.z, fx_split(fx_weight_q(ww.z, P.wscale, &ovf), t.z), grho);
            lw.add(c.w, fx_split(fx_weight_q(ww.w, P.wscale, &ovf), t.w), grho);
        }
    }
    for (int64_t i = (gb1 << 2) + threadIdx.x; i < end; i += blockDim.x) {
        const uint32_t pi = eq_point_of_slot((uint32_t)i, P.n);
        int c = eq_cell_of(P.tab, P.ncell, pi);
        float t, vv, ww;
        ps_eq_one(P, pi, c, t, vv, ww, cache);
        P.cell[i] = c;
        P.theta[i] = t;
        P.v[i] = vv;
        P.w[i] = ww;
        if (dep) lw.add(c, fx_split(fx_weight_q(ww, P.wscale, &ovf), t), grho);
    }
    if (dep) lw.flush(grho);
    if (ovf) raise_flag(P.status, PE_FLAG_OVERFLOW);
    __syncthreads();
    if (dep) grho.flush();
}

}  // namespace
}  // namespace pe

using namespace pe;

extern "C" PE_API int pe_ps_coarsen(const int64_t* sample_fx, int32_t nsamples, int64_t ncoef, int32_t s_w,
                                    double* coarse, void* stream)
{
    if (nsamples < 0 || ncoef < 0 || !sample_fx || !coarse || s_w < -60 || s_w > 60) return PE_EINVAL;
    const int64_t n = (int64_t)nsamples * ncoef;
    if (n == 0) return PE_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * (int64_t)sm_count());
    k_ps_scale<<<grid, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const long long*>(sample_fx), n,
                                                       ldexp(1.0, -(s_w + 24)), coarse);
    return launch_status(1);
}

extern "C" PE_API int pe_ps_project(const double* samples, int32_t K, int32_t nxc, int32_t n_v, double dt, double dT,
                                    int32_t filter, double* work, double* out, double* slope, void* stream)
{
    if (!samples || !work || !out || !slope || K < 1 || nxc < 1 || n_v < 1 || !(dt > 0.0) || filter < 0 || filter > 7)
        return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = nxc * n_v;
    k_ps_slope<<<(n + 255) / 256, 256, 0, s>>>(samples, K, n, dt, work);
    k_ps_leap<<<(n + 255) / 256, 256, 0, s>>>(samples, work, K, nxc, n_v, dT - K * dt, filter, out, slope);
    return launch_status(2);
}

extern "C" PE_API int pe_ps_lift_tables(const double* H, int32_t nxc, int32_t n_v, double* mass, double* cdf,
                                        float* table, double* scratch, int32_t* flags, void* stream)
{
    (void)scratch;  // the rows live in shared memory
    if (!H || !mass || !cdf || !table || nxc < 1 || n_v < 1 || n_v > 1024) return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (flags && cudaMemsetAsync(flags, 0, sizeof(int32_t), s) != cudaSuccess) return PE_ECUDA;
    // three FP64 rows of n_v + 1, 2 x 32 running sums and the mass per bin, two warps per bin.
    // The serial chains (running sums) and the FP64 divisions set the time, so the bins spread
    // over all SMs: about one bin per SM, 1 to 4 per block (fewer for wide rows, <= 192 KB)
    const size_t row3 = sizeof(double) * (3 * ((size_t)n_v + 1) + 66);
    int per_block = std::max(1, std::min(4, nxc / sm_count()));
    per_block = (int)std::min<size_t>((size_t)per_block, (size_t)(192 * 1024) / row3);
    if (per_block < 1) return PE_EINVAL;
    const size_t smem = row3 * (size_t)per_block;
    if (ensure_smem((const void*)k_ps_cdf, smem) != PE_OK) return PE_ECUDA;
    k_ps_cdf<<<(nxc + per_block - 1) / per_block, 64 * per_block, smem, s>>>(H, nxc, n_v, mass, cdf, table, flags);
    k_ps_mass<<<1, 1024, 0, s>>>(nxc, mass);
    return launch_status(2);
}

namespace pe {
namespace {

// Mean velocity of the reconstructed distribution of bin b (cells of width dv from v_min,
// cell k holding F[k+1] - F[k] of the bin's mass), then linear between bin midpoints (periodic)
// at the nodes.
__device__ double ps_bin_mean(const double* cdf, int b, int nv, double vmin, double dv)
{
    const double* F = cdf + (size_t)b * (nv + 1);
    double m = 0.0;
    for (int k = 0; k < nv; ++k) m += (vmin + (k + 0.5) * dv) * (F[k + 1] - F[k]);
    return m;
}

// One block: the bin means into shared memory first (each bin once), then the nodes.
__global__ void __launch_bounds__(1024) k_ps_mean_velocity(const double* __restrict__ cdf, int nxc, int nv,
                                                           double vmin, double dv, int bin_shift, int ncell,
                                                           float* __restrict__ u)
{
    extern __shared__ double ub[];
    for (int b = threadIdx.x; b < nxc; b += blockDim.x) ub[b] = ps_bin_mean(cdf, b, nv, vmin, dv);
    __syncthreads();
    const double B = (double)(1 << bin_shift);
    for (int j = threadIdx.x; j < ncell; j += blockDim.x) {
        const double t = ((double)j - 0.5 * (B - 1.0)) / B;  // bin-midpoint coordinate of node j
        const double f0 = floor(t);
        const double f = t - f0;
        const int b0 = (((int)f0) % nxc + nxc) % nxc, b1 = (b0 + 1) % nxc;
        u[j] = (float)((1.0 - f) * ub[b0] + f * ub[b1]);
    }
}

}  // namespace
}  // namespace pe

extern "C" PE_API int pe_ps_mean_velocity(const double* cdf, int32_t nxc, int32_t n_v, double v_min, double dv,
                                          int32_t bin_shift, int32_t ncell, float* u_prof, void* stream)
{
    if (!cdf || !u_prof || nxc < 1 || n_v < 1 || !(dv > 0.0) || bin_shift < 0 || bin_shift > 13 || !is_pow2(ncell) ||
        ncell > kFullGridMax || ((int64_t)nxc << bin_shift) != ncell)
        return PE_EINVAL;
    const size_t smem = sizeof(double) * (size_t)nxc;
    if (ensure_smem((const void*)pe::k_ps_mean_velocity, smem) != PE_OK) return PE_ECUDA;
    pe::k_ps_mean_velocity<<<1, 1024, smem, (cudaStream_t)stream>>>(cdf, nxc, n_v, v_min, dv, bin_shift, ncell,
                                                                    u_prof);
    return launch_status(1);
}

extern "C" PE_API int pe_ps_quiet_start(int32_t* cell, float* theta, float* v, float* w, int64_t n, int32_t ncell,
                                        int32_t bin_shift, const double* mass, const float* table, int32_t n_v,
                                        double v_min, double dv, uint64_t seed, int32_t s_w, int64_t* rho_fx,
                                        uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !mass || !table || n_v < 1 || !(dv > 0.0)) return PE_EINVAL;
    if (bin_shift < 0 || (1 << bin_shift) > ncell) return PE_EINVAL;
    if (n <= 0 || n % ncell != 0 || n >= (int64_t(1) << 32)) return PE_EINVAL;
    if (!cell || !theta || !v || !w || !aligned16(cell) || !aligned16(theta) || !aligned16(v) || !aligned16(w))
        return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    PSLoad P{};
    P.cell = cell;
    P.theta = theta;
    P.v = v;
    P.w = w;
    P.n = n;
    P.ppc = (uint32_t)(n / ncell);
    P.log2ppc = is_pow2(P.ppc) ? ilog2(P.ppc) : -1;
    P.ncell = ncell;
    P.mask = ncell - 1;
    P.bin_shift = bin_shift;
    P.nv = n_v;
    P.per_node = ldexpf(1.0f, -bin_shift);
    P.vmin = (float)v_min;
    P.dv = (float)dv;
    P.inv_ppc = 1.0f / (float)P.ppc;
    P.two_ppc = 2.0f * (float)P.ppc;
    P.inv_two_ppc = 1.0f / P.two_ppc;
    P.mass = mass;
    P.table = table;
    P.half = (uint32_t)(2147483648.0 / (double)n);
    // splitmix64 (Steele, Lea, Flood 2014) of the seed; its upper half is the Cranley-Patterson shift
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    P.shift = (uint32_t)(z >> 32);
    P.wscale = ldexpf(1.0f, s_w);
    P.rho = reinterpret_cast<unsigned long long*>(rho_fx);
    P.rho_width = ncell <= kRhoWindowNodes ? ncell : kRhoWindowNodes;
    P.status = status;
    const size_t smem = rho_fx ? kSmemGridWords * sizeof(uint32_t) * (size_t)P.rho_width : 0;
    const void* k = (const void*)k_ps_quiet_start;
    if (ensure_smem(k, smem) != PE_OK) return PE_ECUDA;
    const int grid = particle_grid(k, 256, smem, n, &P.chunk);
    if (rho_fx && cudaMemsetAsync(rho_fx, 0, sizeof(int64_t) * (size_t)ncell, s) != cudaSuccess) return PE_ECUDA;
    k_ps_quiet_start<<<grid, 256, smem, s>>>(P);
    return launch_status(1);
}

extern "C" PE_API int pe_ps_node_tables(const double* mass, const double* cdf, int32_t nxc, int32_t ncell,
                                        int32_t n_v, float* node_table, float* node_dens, void* stream)
{
    if (!mass || !cdf || !node_table || !node_dens || !is_pow2(ncell) || !is_pow2(nxc) || nxc > ncell || n_v < 1 ||
        n_v > 4096)
        return PE_EINVAL;
    k_ps_node_tables<<<ncell, 256, sizeof(double) * ((size_t)n_v + 1), (cudaStream_t)stream>>>(mass, cdf, nxc, ilog2(ncell / nxc), n_v, node_table,
                                                              node_dens);
    return launch_status(1);
}

extern "C" PE_API int pe_ps_quiet_start_nodes(int32_t* cell, float* theta, float* v, float* w, int64_t n,
                                              int32_t ncell, const float* node_table, const float* node_dens,
                                              int32_t n_v, double v_min, double dv, uint64_t seed, int32_t s_w,
                                              int64_t* rho_fx, uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !node_table || !node_dens || n_v < 1 || n_v > 4096 || !(dv > 0.0))
        return PE_EINVAL;
    if (n <= 0 || n % ncell != 0 || n >= (int64_t(1) << 32)) return PE_EINVAL;
    if (!cell || !theta || !v || !w || !aligned16(cell) || !aligned16(theta) || !aligned16(v) || !aligned16(w))
        return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    PSLoad P{};
    P.cell = cell;
    P.theta = theta;
    P.v = v;
    P.w = w;
    P.n = n;
    P.ppc = (uint32_t)(n / ncell);
    P.log2ppc = is_pow2(P.ppc) ? ilog2(P.ppc) : -1;
    P.ncell = ncell;
    P.mask = ncell - 1;
    P.nv = n_v;
    P.vmin = (float)v_min;
    P.dv = (float)dv;
    P.inv_ppc = 1.0f / (float)P.ppc;
    P.two_ppc = 2.0f * (float)P.ppc;
    P.inv_two_ppc = 1.0f / P.two_ppc;
    P.table = node_table;
    P.node_dens = node_dens;
    // a block's cells (chunks of <= 65536 particles) and the next node, within 48 KB
    const int rw_bytes = 4 * (2 * n_v + 1);
    P.stage_rows = std::min<int64_t>({(int64_t)ncell, (48 * 1024) / rw_bytes, 65536 / (int64_t)P.ppc + 2});
    P.half = (uint32_t)(2147483648.0 / (double)n);
    // splitmix64 (Steele, Lea, Flood 2014) of the seed; its upper half is the Cranley-Patterson shift
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    P.shift = (uint32_t)(z >> 32);
    P.wscale = ldexpf(1.0f, s_w);
    P.rho = reinterpret_cast<unsigned long long*>(rho_fx);
    P.rho_width = ncell <= kRhoWindowNodes ? ncell : kRhoWindowNodes;
    P.status = status;
    const size_t smem = (rho_fx ? kSmemGridWords * sizeof(uint32_t) * (size_t)P.rho_width : 0) +
                        (size_t)P.stage_rows * (size_t)rw_bytes;
    const bool four = P.log2ppc >= 2;  // a lane's four slots in one cell
    const void* k = four ? (const void*)k_ps_quiet_start_nodes : (const void*)k_ps_quiet_start;
    if (ensure_smem(k, smem) != PE_OK) return PE_ECUDA;
    const int grid = particle_grid(k, 256, smem, n, &P.chunk);
    if (rho_fx && cudaMemsetAsync(rho_fx, 0, sizeof(int64_t) * (size_t)ncell, s) != cudaSuccess) return PE_ECUDA;
    if (four)
        k_ps_quiet_start_nodes<<<grid, 256, smem, s>>>(P);
    else
        k_ps_quiet_start<<<grid, 256, smem, s>>>(P);
    return launch_status(1);
}

extern "C" PE_API int pe_ps_quiet_start_equal(int32_t* cell, float* theta, float* v, float* w, int64_t n,
                                              int32_t ncell, int32_t bin_shift, const double* mass, const float* table,
                                              int32_t n_v, double v_min, double dv, uint64_t seed, int32_t s_w,
                                              void* scratch, int64_t* rho_fx, uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !mass || !table || !scratch || n_v < 1 || !(dv > 0.0)) return PE_EINVAL;
    if (bin_shift < 0 || (1 << bin_shift) > ncell) return PE_EINVAL;
    if (n <= 0 || n >= (int64_t(1) << 32) || ((uintptr_t)scratch & 15u)) return PE_EINVAL;
    if (!cell || !theta || !v || !w || !aligned16(cell) || !aligned16(theta) || !aligned16(v) || !aligned16(w))
        return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int nxc = ncell >> bin_shift, ncl = ncell - 1;
    double* prof = static_cast<double*>(scratch);                       // [ncell]
    double* C = prof + ncell;                                            // [ncl + 1]
    long long* first = reinterpret_cast<long long*>(C + ncl + 1);        // [ncl + 1]
    double* MoN = reinterpret_cast<double*>(first + ncl + 1);           // [1]
    double* total = MoN + 1;                                             // [1]
    float* densf = reinterpret_cast<float*>(total + 1);                  // [nxc]
    float* wn = densf + nxc;                                             // [1]
    k_ps_profile<<<1, 1024, 0, s>>>(mass, nxc, bin_shift, ncell, n, prof, total, densf, wn);
    k_eq_table<double><<<1, kEqThreads, 0, s>>>(prof, ncell, 1.0f, n, C, first, MoN, status);
    PSEqLoad P{};
    P.cell = cell;
    P.theta = theta;
    P.v = v;
    P.w = w;
    P.n = n;
    P.ncell = ncell;
    P.mask = ncell - 1;
    P.bin_shift = bin_shift;
    P.nv = n_v;
    P.nxc = nxc;
    P.vmin = (float)v_min;
    P.dv = (float)dv;
    P.prof = prof;
    P.densf = densf;
    P.wn = wn;
    P.width = ldexpf(1.0f, bin_shift);
    P.inv_width = ldexpf(1.0f, -bin_shift);
    P.mid_first = 0.5f * (P.width - 0.5f);
    P.mid_last = (float)(0.5 * ((nxc - 1) * (double)P.width - 0.5 + (double)(ncell - 1)));
    P.tab = EqTable{C, first, MoN};
    P.table = table;
    P.half = (uint32_t)(2147483648.0 / (double)n);
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL;  // splitmix64 of the seed: the shift is its upper half
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    P.shift = (uint32_t)(z >> 32);
    P.wscale = ldexpf(1.0f, s_w);
    P.rho = reinterpret_cast<unsigned long long*>(rho_fx);
    P.rho_width = ncell <= kRhoWindowNodes ? ncell : kRhoWindowNodes;
    P.status = status;
    const size_t smem = rho_fx ? kSmemGridWords * sizeof(uint32_t) * (size_t)P.rho_width : 0;
    const void* k = (const void*)k_ps_quiet_start_equal;
    if (ensure_smem(k, smem) != PE_OK) return PE_ECUDA;
    const int grid = particle_grid(k, 256, smem, n, &P.chunk);
    if (rho_fx && cudaMemsetAsync(rho_fx, 0, sizeof(int64_t) * (size_t)ncell, s) != cudaSuccess) return PE_ECUDA;
    k_ps_quiet_start_equal<<<grid, 256, smem, s>>>(P);
    return launch_status(3);
}
