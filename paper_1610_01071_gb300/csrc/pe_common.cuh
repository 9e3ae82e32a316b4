// Device helpers shared by the particle, field and coarse-variable kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pepic.h"

namespace pe {

constexpr float kThetaOneF = 16777216.0f;  // 2^24: offset resolution of the deposit rule
constexpr uint32_t kThetaOne = 1u << 24;

__device__ __forceinline__ void raise_flag(uint32_t* status, uint32_t bits)
{
    if (status) atomicOr(status, bits);
}

// Fixed-point CIC split of one particle: q (int32, w 2^s or w V 2^s) at offset theta.
// Left node gets q (2^24 - theta_q), right node q theta_q, both exact in 64 bits.
struct FxSplit {
    unsigned long long left, right;
};

__device__ __forceinline__ FxSplit fx_split(int32_t q, float theta)
{
    uint32_t tq = __float2uint_rn(theta * kThetaOneF);  // theta * 2^24 is exact in FP32
    long long r = (long long)q * (long long)tq;
    long long l = (long long)q * (long long)(kThetaOne - tq);
    return {(unsigned long long)l, (unsigned long long)r};
}

// Block-local copy of a nodal int64 grid in shared memory: either the full periodic
// grid (width == ncell, base == 0) or a window [base, base + width) of it; nodes
// outside the window go straight to the global grid with a 64-bit atomic.
//
// Each node's int64 sum is kept as three digit counters, value = d0 + d1 2^16 + d2 2^32,
// with every contribution v split as v mod 2^16, (v >> 16) mod 2^16 and v >> 32
// (arithmetic). The counters are updated with native 32-bit shared-memory reductions
// and cannot overflow while a block makes at most 65536 additions to a node whose
// absolute values sum to less than 2^62 (the launch keeps block chunks at or below
// 65536 particles, each adding to a node at most once, directly or through a lane
// window). The flush recombines them exactly: the same integer as a plain int64 sum.
constexpr int kMaxChunk = 65536;

struct SmemGrid {
    uint32_t* d0;
    uint32_t* d1;
    int32_t* d2;
    unsigned long long* g;
    int base, width, mask;

    // Carves three arrays of `width` counters from s; returns the next free word.
    __device__ __forceinline__ uint32_t* bind(uint32_t* s, unsigned long long* global, int b, int w, int m)
    {
        d0 = s;
        d1 = s + w;
        d2 = reinterpret_cast<int32_t*>(s + 2 * w);
        g = global;
        base = b;
        width = w;
        mask = m;
        return s + 3 * w;
    }

    __device__ __forceinline__ void add(int node, unsigned long long val) const
    {
        const int idx = (node - base) & mask;
        if (idx < width) {
            const uint32_t a = (uint32_t)val & 0xFFFFu, b = (uint32_t)(val >> 16) & 0xFFFFu;
            const int32_t c = (int32_t)((long long)val >> 32);
            if (a) atomicAdd(&d0[idx], a);
            if (b) atomicAdd(&d1[idx], b);
            if (c) atomicAdd(&d2[idx], c);
        } else {
            atomicAdd(&g[node], val);
        }
    }

    __device__ __forceinline__ void zero() const
    {
        for (int i = threadIdx.x; i < width; i += blockDim.x) {
            d0[i] = 0u;
            d1[i] = 0u;
            d2[i] = 0;
        }
    }

    // Adds the non-zero node sums to the global grid; call after __syncthreads().
    __device__ __forceinline__ void flush() const
    {
        for (int i = threadIdx.x; i < width; i += blockDim.x) {
            const long long v = (long long)d0[i] + ((long long)d1[i] << 16) + ((long long)d2[i] << 32);
            if (v) atomicAdd(&g[(base + i) & mask], (unsigned long long)v);
        }
    }
};

// Block-local phase-space restriction sample: a window of `width` coarse x-bins starting
// at `base` (mod nxc) times nv velocity cells, each an exact int64 sum kept as the three
// digit counters of SmemGrid (same bounds). Entries outside the window go to the global
// histogram g[nxc][nv] with a 64-bit atomic.
struct PSGrid {
    uint32_t* d0;
    uint32_t* d1;
    int32_t* d2;
    unsigned long long* g;
    int base, width, xmask, nv;

    __device__ __forceinline__ uint32_t* bind(uint32_t* s, unsigned long long* global, int b, int w, int nxc, int nvel)
    {
        const int n = w * nvel;
        d0 = s;
        d1 = s + n;
        d2 = reinterpret_cast<int32_t*>(s + 2 * n);
        g = global;
        base = b;
        width = w;
        xmask = nxc - 1;
        nv = nvel;
        return s + 3 * n;
    }

    __device__ __forceinline__ void add(int key, long long val) const
    {
        const int xb = key / nv, j = key - xb * nv;
        const int d = (xb - base) & xmask;
        if (d < width) {
            const int idx = d * nv + j;
            const uint32_t a = (uint32_t)val & 0xFFFFu, b = (uint32_t)(val >> 16) & 0xFFFFu;
            const int32_t c = (int32_t)(val >> 32);
            if (a) atomicAdd(&d0[idx], a);
            if (b) atomicAdd(&d1[idx], b);
            if (c) atomicAdd(&d2[idx], c);
        } else {
            atomicAdd(&g[key], (unsigned long long)val);
        }
    }

    __device__ __forceinline__ void zero() const
    {
        for (int i = threadIdx.x; i < width * nv; i += blockDim.x) {
            d0[i] = 0u;
            d1[i] = 0u;
            d2[i] = 0;
        }
    }

    __device__ __forceinline__ void flush() const
    {
        for (int i = threadIdx.x; i < width * nv; i += blockDim.x) {
            const long long v = (long long)d0[i] + ((long long)d1[i] << 16) + ((long long)d2[i] << 32);
            if (v) {
                const int d = i / nv, j = i - d * nv;
                atomicAdd(&g[(size_t)((base + d) & xmask) * nv + j], (unsigned long long)v);
            }
        }
    }
};

// Per-lane run of equal phase-space keys over consecutive particles of a lane (a lane's
// four particles of a 16-byte group are neighbours in a velocity-ordered cell, so they
// usually share their phase-space cell): adds accumulate while the key repeats; a new key
// sends the finished run to the grid directly.
struct PSAcc {
    int key;
    long long val;

    __device__ __forceinline__ void reset()
    {
        key = -1;
        val = 0;
    }
    __device__ __forceinline__ void add(int k, long long q, const PSGrid& gr)
    {
        if (k == key) {
            val += q;
        } else {
            if (key >= 0) gr.add(key, val);
            key = k;
            val = q;
        }
    }
};

// Adds (key, val) pairs of the active lanes to a PSGrid, summing runs of equal keys in
// consecutive lanes first (consecutive particles of a velocity-ordered cell share their
// phase-space cell): a segmented suffix sum over the run, added once by its first lane.
// key < 0 marks a lane with nothing to add. When the active lanes are not a prefix of the
// warp, every lane adds on its own.
__device__ __forceinline__ void ps_add_warp(const PSGrid& gr, int key, long long val)
{
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int nact = __popc(act);
    if (act != (nact == 32 ? 0xFFFFFFFFu : ((1u << nact) - 1u))) {
        if (key >= 0) gr.add(key, val);
        return;
    }
    const int prev = __shfl_up_sync(act, key, 1);
    const bool head = (lane == 0) || (prev != key);
    const unsigned heads = __ballot_sync(act, head);
    const unsigned after = heads & (0xFFFFFFFEu << lane);
    const int run_end = after ? (__ffs(after) - 2) : (nact - 1);
    long long s = val;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long o = __shfl_down_sync(act, s, off);
        if (lane + off <= run_end) s += o;
    }
    if (head && key >= 0) gr.add(key, s);
}

// Block-local restriction sample summed over bins of 2^b nodes (Haar restriction). A
// particle whose two CIC nodes fall in one bin adds its whole q 2^24 (q = w_q or m_q,
// |q| <= 2^23): kept as digits of q in u0 (q mod 2^16) and u1 (q >> 16). A particle
// split across a bin edge adds its two fixed-point parts as three digits each
// (v0, v1, v2, as in SmemGrid). The flush recombines
//   sum = (u0 + u1 2^16) 2^24 + v0 + v1 2^16 + v2 2^32
// exactly; the bounds of SmemGrid apply per bin (at most 65536 additions per block).
struct BinGrid {
    uint32_t* u0;
    int32_t* u1;
    uint32_t* v0;
    uint32_t* v1;
    int32_t* v2;
    unsigned long long* g;
    int nb;

    __device__ __forceinline__ uint32_t* bind(uint32_t* s, unsigned long long* global, int nbins)
    {
        u0 = s;
        u1 = reinterpret_cast<int32_t*>(s + nbins);
        v0 = s + 2 * nbins;
        v1 = s + 3 * nbins;
        v2 = reinterpret_cast<int32_t*>(s + 4 * nbins);
        g = global;
        nb = nbins;
        return s + 5 * nbins;
    }

    __device__ __forceinline__ void add_whole(int b, int32_t q) const
    {
        atomicAdd(&u0[b], (uint32_t)q & 0xFFFFu);
        atomicAdd(&u1[b], q >> 16);
    }

    __device__ __forceinline__ void add_part(int b, unsigned long long val) const
    {
        atomicAdd(&v0[b], (uint32_t)val & 0xFFFFu);
        atomicAdd(&v1[b], (uint32_t)(val >> 16) & 0xFFFFu);
        atomicAdd(&v2[b], (int32_t)((long long)val >> 32));
    }

    __device__ __forceinline__ void zero() const
    {
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            u0[i] = 0u;
            u1[i] = 0;
            v0[i] = 0u;
            v1[i] = 0u;
            v2[i] = 0;
        }
    }

    __device__ __forceinline__ void flush() const
    {
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const long long whole = (long long)u0[i] + ((long long)u1[i] << 16);
            const long long v = whole * (long long)kThetaOne + (long long)v0[i] + ((long long)v1[i] << 16) +
                                ((long long)v2[i] << 32);
            if (v) atomicAdd(&g[i], (unsigned long long)v);
        }
    }
};

// Per-lane sliding accumulator for a stream of particles whose cells change slowly
// (cell-sorted particles, or the smooth sweeps of a velocity-ordered cell): four
// consecutive nodes base..base+3 held in registers, flushed to the block grid only when
// a particle falls outside them.
struct LaneWindow {
    int base;
    unsigned long long s0, s1, s2, s3;

    __device__ __forceinline__ void reset(int b)
    {
        base = b;
        s0 = s1 = s2 = s3 = 0ull;
    }

    __device__ __forceinline__ void flush(const SmemGrid& grid) const
    {
        if (s0) grid.add(base & grid.mask, s0);
        if (s1) grid.add((base + 1) & grid.mask, s1);
        if (s2) grid.add((base + 2) & grid.mask, s2);
        if (s3) grid.add((base + 3) & grid.mask, s3);
    }

    // Deposits (left at node c, right at node c+1).
    __device__ __forceinline__ void add(int c, const FxSplit& q, const SmemGrid& grid)
    {
        int d = (c - base) & grid.mask;
        if (d > 2) {
            flush(grid);
            reset((c - 1) & grid.mask);
            d = 1;
        }
        // one pair of 64-bit adds under a predicate (no selects of 64-bit values)
        if (d == 1) {
            s1 += q.left;
            s2 += q.right;
        } else if (d == 0) {
            s0 += q.left;
            s1 += q.right;
        } else {
            s2 += q.left;
            s3 += q.right;
        }
    }
};

// Per-lane run of whole-particle bin contributions (BinGrid::add_whole) of the density and
// momentum samples over the lane's four neighbouring particles; a new bin sends the finished
// run to the grid. The run of a group is then summed across lanes (bin_add_warp).
struct BinAcc {
    int key;
    int32_t n, m;

    __device__ __forceinline__ void reset()
    {
        key = -1;
        n = m = 0;
    }
    __device__ __forceinline__ void add(int b, int32_t wq, int32_t mq, const BinGrid& gn, const BinGrid& gm)
    {
        if (b == key) {
            n += wq;
            m += mq;
        } else {
            if (key >= 0) {
                gn.add_whole(key, n);
                gm.add_whole(key, m);
            }
            key = b;
            n = wq;
            m = mq;
        }
    }
};

// Adds the active lanes' bin runs to the density and momentum BinGrids, summing runs of
// equal bins in consecutive lanes first (consecutive lanes hold neighbouring particles of a
// velocity-ordered cell, whose co-moving bins mostly agree): |sum| <= 32 * 4 * 2^23 = 2^30.
// One warp sum when every active lane holds the same bin, else a segmented sum per run.
// Lanes with key < 0 add nothing; if the active lanes are not a prefix of the warp, every
// lane adds on its own.
__device__ __forceinline__ void bin_add_warp(const BinGrid& gn, const BinGrid& gm, int key, int32_t n, int32_t m)
{
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int first = __ffs(act) - 1;
    const int k0 = __shfl_sync(act, key, first);
    if (__all_sync(act, key == k0)) {  // one bin for every active lane (the common case)
        const int32_t sn = __reduce_add_sync(act, n), sm = __reduce_add_sync(act, m);
        if (k0 >= 0 && lane == first) {
            gn.add_whole(k0, sn);
            gm.add_whole(k0, sm);
        }
        return;
    }
    const int nact = __popc(act);
    if (act != (nact == 32 ? 0xFFFFFFFFu : ((1u << nact) - 1u))) {
        if (key >= 0) {
            gn.add_whole(key, n);
            gm.add_whole(key, m);
        }
        return;
    }
    const int prev = __shfl_up_sync(act, key, 1);
    const bool head = (lane == 0) || (prev != key);
    const unsigned heads = __ballot_sync(act, head);
    const unsigned after = heads & (0xFFFFFFFEu << lane);
    const int run_end = after ? (__ffs(after) - 2) : (nact - 1);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t on = __shfl_down_sync(act, n, off), om = __shfl_down_sync(act, m, off);
        if (lane + off <= run_end) {
            n += on;
            m += om;
        }
    }
    if (head && key >= 0) {
        gn.add_whole(key, n);
        gm.add_whole(key, m);
    }
}

// Contiguous particle range [begin, end) of block b when n particles are split into
// chunks whose starts are multiples of 4 (so float4 loads stay aligned).
__device__ __forceinline__ void block_chunk(int64_t n, int64_t chunk, int64_t* begin, int64_t* end)
{
    int64_t b = (int64_t)blockIdx.x * chunk;
    *begin = b < n ? b : n;
    int64_t e = b + chunk;
    *end = e < n ? e : n;
}

// Contiguous range of 4-particle groups [*g0, *g1) of this warp inside the block's
// groups [gb0, gb1): warps take consecutive slices (multiples of 32 groups), so the
// particles a lane visits stay sorted and close in cell index.
__device__ __forceinline__ void warp_groups(int64_t gb0, int64_t gb1, int64_t* g0, int64_t* g1)
{
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    int64_t per = (gb1 - gb0 + nw - 1) / nw;
    per = (per + 31) & ~int64_t(31);
    int64_t a = gb0 + per * w, b = a + per;
    *g0 = a < gb1 ? a : gb1;
    *g1 = b < gb1 ? b : gb1;
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace pe
