// Equal-weight loading on a bounded grid (shared by the moment and phase-space loaders):
// the cumulative-mass table of a nodal density profile that is linear inside each of the
// ncell - 1 cells between the walls, the position of the point of quantile (i + 1/2) / n, and
// the storage order of the points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pe_common.cuh"

namespace pe {

// Scratch of the equal-weight loading: cumulative cell masses and first particle of each
// cell. Layout in the caller's scratch: double C[ncl + 1], int64 first[ncl + 1], double MoN.
struct EqTable {
    const double* C;
    const long long* first;
    const double* MoN;
};

constexpr int kEqThreads = 1024;

// One block: cell masses m_c = (n_c f_c + n_{c+1} f_{c+1}) / 2 of the linear profile over
// the ncl = ncell - 1 cells between the walls (f = wall_factor on the wall nodes, 1 inside),
// their cumulative sums C (each thread sums a contiguous run of cells, then an exclusive scan
// of the run totals in a fixed order), M = C[ncl], MoN = M / n and
// first[c] = ceil(C_c n / M - 1/2), the first particle i with (i + 1/2) M / n >= C_c.
// TP: the profile's type (FP32 profiles of the lifting, FP64 ones of the phase-space loader).
template <typename TP>
__global__ void __launch_bounds__(kEqThreads) k_eq_table(const TP* __restrict__ prof_n, int ncell, float wall_factor,
                                                        int64_t n, double* C, long long* first, double* MoN,
                                                        uint32_t* status)
{
    __shared__ double part[kEqThreads];
    const int ncl = ncell - 1;
    const int per = (ncl + kEqThreads - 1) / kEqThreads;
    const int t = threadIdx.x;
    const int c0 = t * per, c1 = (c0 + per < ncl) ? c0 + per : ncl;
    auto dens = [&](int j) {
        const double v = (double)prof_n[j];
        return (j == 0 || j == ncell - 1) ? v * (double)wall_factor : v;
    };
    double run = 0.0;
    for (int c = c0; c < c1; ++c) run += 0.5 * (dens(c) + dens(c + 1));
    // exclusive scan of the run totals: within each warp by shuffles, then over the warps' totals
    // (fixed order; a dependent FP64 add costs ~100 cycles here, so a serial scan of 1024 totals
    // took ~50 us)
    const int lane = t & 31, wid = t >> 5;
    double incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) part[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        double ws = (lane < kEqThreads / 32) ? part[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += y;
        }
        part[32 + lane] = ws;  // inclusive over warps
    }
    __syncthreads();
    double acc = (wid > 0 ? part[32 + wid - 1] : 0.0) + incl - run;
    for (int c = c0; c < c1; ++c) {
        C[c] = acc;
        acc += 0.5 * (dens(c) + dens(c + 1));
    }
    if (c1 == ncl && c0 < c1) C[ncl] = acc;
    __syncthreads();
    const double M = C[ncl];
    const bool ok = M > 0.0 && isfinite(M);
    if (t == 0) {
        *MoN = ok ? M / (double)n : 0.0;
        if (!ok) raise_flag(status, PE_FLAG_RANGE);
    }
    for (int c = t; c <= ncl; c += kEqThreads) {
        long long f;
        if (!ok) {
            f = (c == 0) ? 0 : n;  // no mass: every particle in cell 0 with weight 0
        } else {
            const double q = ceil(C[c] * ((double)n / M) - 0.5);
            f = q < 0.0 ? 0 : (q > (double)n ? n : (long long)q);
        }
        first[c] = (c == ncl) ? n : f;
    }
}

// Cell of particle i: the largest c in [0, ncl) with first[c] <= i (binary search; always
// in range whatever the table holds).
__device__ __forceinline__ int eq_cell_of(const EqTable& tab, int ncell, long long i)
{
    int lo = 0, hi = ncell - 1;  // first[lo] <= i < first[hi] on a valid table
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(tab.first + mid) <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Per-lane constants of the cell last visited by eq_position: the point's share of its cell's
// mass, r = ((i + 1/2) M/n - C_c) / m_c, is a_c + (i - first_c) s_c with
// a_c = ((first_c + 1/2) M/n - C_c) / m_c and s_c = (M/n) / m_c, formed once per cell in FP64
// and applied in FP32 (r within ~1e-7 of the FP64 quotient). A lane visits thousands of points
// of one cell in a row, and an FP64 division per point took most of the loaders' time.
struct EqCellCache {
    int c;          // cell of the constants; -1 before the first point
    long long i0;   // first[c]
    float a, s;

    __device__ __forceinline__ void reset() { c = -1; }
};

// Position of point i: c is walked forward from a cell at or before the point's; returns the
// offset t in [0, 1) at which the cell's linear density (the profile's two nodal values, wall
// nodes times wall_factor) holds the point's share r of the cell mass: t + sig (t^2 - t) = r.
template <typename TP>
__device__ __forceinline__ float eq_position(const EqTable& tab, const TP* __restrict__ prof, float wall_factor,
                                             int ncell, uint32_t i, int& c, EqCellCache& cache)
{
    while (c < ncell - 2 && __ldg(tab.first + c + 1) <= (long long)i) ++c;
    if (c != cache.c) {
        const double C0 = __ldg(tab.C + c), C1 = __ldg(tab.C + c + 1);
        const double MoN = __ldg(tab.MoN);
        const double mc = C1 - C0;
        const long long i0 = __ldg(tab.first + c);
        cache.c = c;
        cache.i0 = i0;
        if (mc > 0.0) {
            cache.a = (float)((((double)i0 + 0.5) * MoN - C0) / mc);
            cache.s = (float)(MoN / mc);
        } else {
            cache.a = 0.5f;
            cache.s = 0.0f;
        }
    }
    float r = fmaf((float)((long long)i - cache.i0), cache.s, cache.a);
    r = r < 0.0f ? 0.0f : (r > 1.0f ? 1.0f : r);
    float n0 = (float)__ldg(prof + c), n1 = (float)__ldg(prof + c + 1);
    if (c == 0) n0 *= wall_factor;
    if (c + 1 == ncell - 1) n1 *= wall_factor;
    const float sum = n0 + n1;
    const float sig = sum > 0.0f ? (n1 - n0) / sum : 0.0f;
    const float rf = r;
    const float om = 1.0f - sig;
    const float den = om + sqrtf(fmaxf(om * om + 4.0f * sig * rf, 0.0f));
    const float t = den > 0.0f ? 2.0f * rf / den : 0.0f;
    return fminf(fmaxf(t, 0.0f), 0.99999994f);  // stay inside the cell (largest float below 1)
}

// Storage order of the equal-weight loading: inside every full aligned block of 2^kEqBlockBits
// slots, slot s holds point i = s with its low kEqBlockBits bits reversed, so that the block's
// points (all within 2^kEqBlockBits mass quantiles of each other) are stored in ascending
// velocity quantile, as a power-of-two cell of pe_quiet_start stores its points: the 128
// slots a warp visits at once then span 1/32 of the velocity range and their co-moving
// targets stay together. The ragged tail keeps i = s. The reversal is its own inverse.
constexpr int kEqBlockBits = 12;
constexpr uint32_t kEqBlockMask = (1u << kEqBlockBits) - 1u;

__device__ __forceinline__ uint32_t eq_point_of_slot(uint32_t s, int64_t n)
{
    return ((int64_t)(s | kEqBlockMask) < n) ? ((s & ~kEqBlockMask) | (__brev(s & kEqBlockMask) >> (32 - kEqBlockBits)))
                                              : s;
}

}  // namespace pe
