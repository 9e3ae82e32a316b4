// Device helpers shared by the particle, field and coarse-variable kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

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

// Shared-memory reductions on a 32-bit shared-window address (one register per array
// instead of a 64-bit generic pointer; the digits of a node sit at fixed offsets from it).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int OFF>
__device__ __forceinline__ void red_u32(uint32_t a, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0+%2], %1;" ::"r"(a), "r"(v), "n"(OFF) : "memory");
}

template <int OFF>
__device__ __forceinline__ void red_s32(uint32_t a, int32_t v)
{
    asm volatile("red.shared.add.s32 [%0+%2], %1;" ::"r"(a), "r"(v), "n"(OFF) : "memory");
}

// The node's digits are interleaved, four words per node (d0, d1, d2, unused).
constexpr int kSmemGridWords = 4;

struct SmemGrid {
    uint32_t* p;  // generic pointer to node 0 (zero, flush)
    uint32_t s;   // shared address of node 0
    unsigned long long* g;
    int base, width, mask;

    // Carves `width` nodes from sm; returns the next free word.
    __device__ __forceinline__ uint32_t* bind(uint32_t* sm, unsigned long long* global, int b, int w, int m)
    {
        p = sm;
        s = smem_u32(sm);
        g = global;
        base = b;
        width = w;
        mask = m;
        return sm + kSmemGridWords * w;
    }

    // Adds one value given as its three digits (a = v mod 2^16, b = (v >> 16) mod 2^16,
    // c = v >> 32); digit sums of several values (each digit sum exact in 32 bits) add the
    // sum of the values.
    __device__ __forceinline__ void add_digits(int node, uint32_t a, uint32_t b, int32_t c) const
    {
        const int idx = (node - base) & mask;
        if (idx < width) {
            const uint32_t at = s + 16u * (uint32_t)idx;
            if (a) red_u32<0>(at, a);
            if (b) red_u32<4>(at, b);
            if (c) red_s32<8>(at, c);
        } else {
            const long long v = (long long)a + ((long long)b << 16) + ((long long)c << 32);
            if (v) atomicAdd(&g[node], (unsigned long long)v);
        }
    }

    __device__ __forceinline__ void add(int node, unsigned long long val) const
    {
        add_digits(node, (uint32_t)val & 0xFFFFu, (uint32_t)(val >> 16) & 0xFFFFu, (int32_t)((long long)val >> 32));
    }

    __device__ __forceinline__ void zero() const
    {
        for (int i = threadIdx.x; i < width; i += blockDim.x)
            reinterpret_cast<uint4*>(p)[i] = make_uint4(0u, 0u, 0u, 0u);
    }

    // Adds the non-zero node sums to the global grid; call after __syncthreads().
    __device__ __forceinline__ void flush() const
    {
        for (int i = threadIdx.x; i < width; i += blockDim.x) {
            const uint4 d = reinterpret_cast<const uint4*>(p)[i];
            const long long v = (long long)d.x + ((long long)d.y << 16) + ((long long)(int32_t)d.z << 32);
            if (v) atomicAdd(&g[(base + i) & mask], (unsigned long long)v);
        }
    }
};

// Charge-deposit window shared by the 32 lanes of a warp: four consecutive nodes base ..
// base+3, each lane holding its own partial sums of them in registers. The base is the same in
// every lane and moves only by warp-wide decisions, so the window's flushes are warp-uniform:
// each flushed node is summed across the warp (16/16/32-bit digit sums with redux.sync, each
// exact) and added to the block grid by one lane. Lanes that held a per-lane window of their own
// moved it at different particles, so the warp ran the flush code at almost every particle
// with a few lanes active, and those lanes hit the same shared-memory words.
// Every member function must be called by all 32 lanes of the warp, converged.
struct WarpWindow {
    int base;
    unsigned long long s0, s1, s2, s3;

    __device__ __forceinline__ void reset(int b)
    {
        base = b;
        s0 = s1 = s2 = s3 = 0ull;
    }

    // Adds the window's nodes 0 .. n-1 (n warp-uniform, <= 4) to the grid.
    __device__ __forceinline__ void flush_first(const SmemGrid& grid, int n) const
    {
        const int lane = threadIdx.x & 31;
        uint32_t A = 0u, B = 0u;
        int32_t C = 0;
        const unsigned long long s[4] = {s0, s1, s2, s3};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k < n) {
                const uint32_t a = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)s[k] & 0xFFFFu);
                const uint32_t b = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)(s[k] >> 16) & 0xFFFFu);
                const int32_t c = __reduce_add_sync(0xFFFFFFFFu, (int32_t)((long long)s[k] >> 32));
                if (lane == k) {
                    A = a;
                    B = b;
                    C = c;
                }
            }
        }
        if (lane < n) grid.add_digits((base + lane) & grid.mask, A, B, C);
    }

    // Moves the base by sh nodes (warp-uniform); the nodes that leave the window are flushed.
    __device__ __forceinline__ void move(const SmemGrid& grid, int sh)
    {
        if (sh >= 1 && sh <= 3) {
            flush_first(grid, sh);
            if (sh == 1) {
                s0 = s1;
                s1 = s2;
                s2 = s3;
            } else if (sh == 2) {
                s0 = s2;
                s1 = s3;
                s2 = 0ull;
            } else {
                s0 = s3;
                s1 = s2 = 0ull;
            }
            s3 = 0ull;
        } else {
            flush_first(grid, 4);
            s0 = s1 = s2 = s3 = 0ull;
        }
        base = (base + sh) & grid.mask;
    }

    // Deposits q (left part at window node d, right part at d + 1), d in {0, 1, 2}: one pair
    // of 64-bit adds under a predicate.
    __device__ __forceinline__ void add(int d, const FxSplit& q)
    {
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

    // key = (row << 16) | velocity cell
    __device__ __forceinline__ void add(int key, long long val) const { add_at(key >> 16, key & 0xFFFF, val); }

    // Adds val at (row xb, velocity cell j) without dividing the key.
    __device__ __forceinline__ void add_at(int xb, int j, long long val) const
    {
        const int d = (xb - base) & xmask;
        if (d < width) {
            const int idx = d * nv + j;
            const uint32_t a = (uint32_t)val & 0xFFFFu, b = (uint32_t)(val >> 16) & 0xFFFFu;
            const int32_t c = (int32_t)(val >> 32);
            if (a) atomicAdd(&d0[idx], a);
            if (b) atomicAdd(&d1[idx], b);
            if (c) atomicAdd(&d2[idx], c);
        } else {
            atomicAdd(&g[(size_t)xb * nv + j], (unsigned long long)val);
        }
    }

    // Hat rows: a run with key (xb << 16) | j, W = sum w_q and R = sum w_q f_q adds
    // W 2^24 - R to row xb and R to row xb + 1 (periodic).
    __device__ __forceinline__ void add_pair(int key, int32_t w, long long r) const
    {
        const int xb = key >> 16, j = key & 0xFFFF;
        add_at(xb, j, (long long)w * (1ll << 24) - r);
        add_at((xb + 1) & xmask, j, r);
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

// Per-lane run of equal phase-space keys over consecutive particles of a lane (a lane's four
// particles of a 16-byte group are neighbours in a velocity-ordered cell, so they usually share
// their phase-space cell), for particles whose two CIC nodes lie in one bin: W = sum w_q
// (|W| <= 4 2^23); the entry gets W 2^24. A new key sends the finished run to the grid.
struct PSAccW {
    int key;
    int32_t w;

    __device__ __forceinline__ void reset()
    {
        key = -1;
        w = 0;
    }
    __device__ __forceinline__ void add(int k, int32_t q, const PSGrid& gr)
    {
        if (k == key) {
            w += q;
        } else {
            if (key >= 0) gr.add(key, (long long)w * (long long)kThetaOne);
            key = k;
            w = q;
        }
    }
};

// Adds the lanes' runs (key, W) to a PSGrid, summing runs of equal keys in consecutive lanes
// first: a segmented suffix sum over the run in 32 bits (W over at most 128 particles stays
// below 2^30), added once by its first lane as W 2^24. key < 0 marks a lane with nothing to add.
// When the active lanes are not a prefix of the warp, every lane adds on its own.
__device__ __forceinline__ void ps_add_warp_w(const PSGrid& gr, int key, int32_t w)
{
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int nact = __popc(act);
    if (act != (nact == 32 ? 0xFFFFFFFFu : ((1u << nact) - 1u))) {
        if (key >= 0) gr.add(key, (long long)w * (long long)kThetaOne);
        return;
    }
    const int prev = __shfl_up_sync(act, key, 1);
    const bool head = (lane == 0) || (prev != key);
    const unsigned heads = __ballot_sync(act, head);
    const unsigned after = heads & (0xFFFFFFFEu << lane);
    const int run_end = after ? (__ffs(after) - 2) : (nact - 1);
    int32_t sw = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t o = __shfl_down_sync(act, sw, off);
        if (lane + off <= run_end) sw += o;
    }
    if (head && key >= 0) gr.add(key, (long long)sw * (long long)kThetaOne);
}

// Per-lane run of equal (coarse node, velocity cell) keys of the hat rows, over a lane's
// four particles of a group: W = sum w_q (32 bits: |W| <= 4 2^23) and R = sum w_q f_q.
struct PSAcc2 {
    int key;  // (xb << 16) | j; -1 while empty
    int32_t w;
    long long r;

    __device__ __forceinline__ void reset()
    {
        key = -1;
        w = 0;
        r = 0;
    }
    __device__ __forceinline__ void add(int k, int32_t wq, long long rq, const PSGrid& gr)
    {
        if (k == key) {
            w += wq;
            r += rq;
        } else {
            if (key >= 0) gr.add_pair(key, w, r);
            key = k;
            w = wq;
            r = rq;
        }
    }
};

// ps_add_warp_w for the hat rows: runs of equal keys in consecutive lanes summed (W over at most
// 128 particles stays below 2^30), added by the run's first lane as two rows.
__device__ __forceinline__ void ps_add_warp2(const PSGrid& gr, int key, int32_t w, long long r)
{
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int nact = __popc(act);
    if (act != (nact == 32 ? 0xFFFFFFFFu : ((1u << nact) - 1u))) {
        if (key >= 0) gr.add_pair(key, w, r);
        return;
    }
    const int prev = __shfl_up_sync(act, key, 1);
    const bool head = (lane == 0) || (prev != key);
    const unsigned heads = __ballot_sync(act, head);
    const unsigned after = heads & (0xFFFFFFFEu << lane);
    const int run_end = after ? (__ffs(after) - 2) : (nact - 1);
    int32_t sw = w;
    long long sr = r;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t ow = __shfl_down_sync(act, sw, off);
        const long long orr = __shfl_down_sync(act, sr, off);
        if (lane + off <= run_end) {
            sw += ow;
            sr += orr;
        }
    }
    if (head && key >= 0) gr.add_pair(key, sw, sr);
}

// Block-local restriction sample summed over bins of 2^b nodes (Haar restriction). A
// particle whose two CIC nodes fall in one bin adds its whole q 2^24 (q = w_q or m_q,
// |q| <= 2^23): kept as digits of q in u0 (q mod 2^16) and u1 (q >> 16). A particle
// split across a bin edge adds its two fixed-point parts as three digits each
// (v0, v1, v2, as in SmemGrid). The flush recombines
//   sum = (u0 + u1 2^16) 2^24 + v0 + v1 2^16 + v2 2^32
// exactly; the bounds of SmemGrid apply per bin (at most 65536 additions per block).
// The bin's counters are interleaved, eight words per bin (u0, u1, v0, v1, v2, unused).
constexpr int kBinGridWords = 8;

struct BinGrid {
    uint32_t* p;  // generic pointer to bin 0 (zero, flush)
    uint32_t s;   // shared address of bin 0
    unsigned long long* g;
    int nb;

    __device__ __forceinline__ uint32_t* bind(uint32_t* sm, unsigned long long* global, int nbins)
    {
        p = sm;
        s = smem_u32(sm);
        g = global;
        nb = nbins;
        return sm + kBinGridWords * nbins;
    }

    __device__ __forceinline__ void add_whole(int b, int32_t q) const
    {
        const uint32_t at = s + 32u * (uint32_t)b;
        red_u32<0>(at, (uint32_t)q & 0xFFFFu);
        red_s32<4>(at, q >> 16);
    }

    // Adds whole contributions given as digit sums: lo = sum (q mod 2^16), hi = sum (q >> 16).
    __device__ __forceinline__ void add_whole_digits(int b, uint32_t lo, int32_t hi) const
    {
        const uint32_t at = s + 32u * (uint32_t)b;
        if (lo) red_u32<0>(at, lo);
        if (hi) red_s32<4>(at, hi);
    }

    __device__ __forceinline__ void add_part(int b, unsigned long long val) const
    {
        const uint32_t at = s + 32u * (uint32_t)b;
        red_u32<8>(at, (uint32_t)val & 0xFFFFu);
        red_u32<12>(at, (uint32_t)(val >> 16) & 0xFFFFu);
        red_s32<16>(at, (int32_t)((long long)val >> 32));
    }

    // Moves t from bin b to bin b + 1 (periodic): the right CIC parts of particles whose two
    // nodes straddle the edge between the bins, counted whole in bin b.
    __device__ __forceinline__ void add_transfer(int b, long long t) const
    {
        if (t == 0) return;
        add_part(b, (unsigned long long)(-t));
        add_part((b + 1) & (nb - 1), (unsigned long long)t);
    }

    __device__ __forceinline__ void zero() const
    {
        for (int i = threadIdx.x; i < 2 * nb; i += blockDim.x)
            reinterpret_cast<uint4*>(p)[i] = make_uint4(0u, 0u, 0u, 0u);
    }

    __device__ __forceinline__ void flush() const
    {
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const uint4 a = reinterpret_cast<const uint4*>(p)[2 * i];
            const uint32_t v2 = p[8 * i + 4];
            const long long whole = (long long)a.x + ((long long)(int32_t)a.y << 16);
            const long long v = whole * (long long)kThetaOne + (long long)a.z + ((long long)a.w << 16) +
                                ((long long)(int32_t)v2 << 32);
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

// Sum over the lanes in `mask` of a 64-bit value, as three exact digit sums (each lane's
// value split into 16 + 16 + 32 bits); every lane in `mask` gets the total.
__device__ __forceinline__ long long warp_sum64(unsigned mask, long long v)
{
    const uint32_t a = __reduce_add_sync(mask, (uint32_t)v & 0xFFFFu);
    const uint32_t b = __reduce_add_sync(mask, (uint32_t)((unsigned long long)v >> 16) & 0xFFFFu);
    const int32_t c = __reduce_add_sync(mask, (int32_t)(v >> 32));
    return (long long)a + ((long long)b << 16) + ((long long)c << 32);
}

// Haar-binned restriction sample of one warp group (four particles per lane): a window of two
// bins K, K+1, with K the lowest bin the warp's particles sample (warp-uniform). Every particle
// adds its whole w_q (m_q) to the bin of its left node; a particle on the last node of bin K
// also adds its right part q theta_q to the transfers tn (tm), which move from bin K to K+1.
// The bin totals are then exactly those of the split CIC deposit summed over the bins. Samples
// outside the window (a spread over more than two bins) go straight to the grids. At the end of
// the group the window is summed across the warp and added once.
struct BinWindow {
    int K;
    int32_t n0, m0, n1, m1;
    long long tn, tm;

    __device__ __forceinline__ void begin(int k)
    {
        K = k;
        n0 = m0 = n1 = m1 = 0;
        tn = tm = 0;
    }

    __device__ __forceinline__ void add(int b, int32_t wq, int32_t mq, uint32_t tq, const BinGrid& gn,
                                        const BinGrid& gm)
    {
        const int d = (b - K) & (gn.nb - 1);
        if (d == 0) {
            n0 += wq;
            m0 += mq;
            tn += (long long)wq * (long long)tq;
            tm += (long long)mq * (long long)tq;
        } else if (d == 1 && tq == 0u) {
            n1 += wq;
            m1 += mq;
        } else {
            gn.add_whole(b, wq);
            gm.add_whole(b, mq);
            if (tq) {
                gn.add_transfer(b, (long long)wq * (long long)tq);
                gm.add_transfer(b, (long long)mq * (long long)tq);
            }
        }
    }

    // Sums the window across the warp and adds it (all 32 lanes, converged);
    // |sum of n| <= 32 * 4 * 2^23 = 2^30.
    __device__ __forceinline__ void end(const BinGrid& gn, const BinGrid& gm) const
    {
        const int lane = threadIdx.x & 31;
        const int32_t N0 = __reduce_add_sync(0xFFFFFFFFu, n0), M0 = __reduce_add_sync(0xFFFFFFFFu, m0);
        const int32_t N1 = __reduce_add_sync(0xFFFFFFFFu, n1), M1 = __reduce_add_sync(0xFFFFFFFFu, m1);
        // lanes 0..3 add bin K's and K+1's density and momentum, one each
        const int32_t v = lane == 0 ? N0 : (lane == 1 ? N1 : (lane == 2 ? M0 : M1));
        if (lane < 4 && v != 0) ((lane & 2) ? gm : gn).add_whole((K + (lane & 1)) & (gn.nb - 1), v);
        if (__any_sync(0xFFFFFFFFu, (tn | tm) != 0)) {
            const long long TN = warp_sum64(0xFFFFFFFFu, tn), TM = warp_sum64(0xFFFFFFFFu, tm);
            if (lane < 2) (lane ? gm : gn).add_transfer(K, lane ? TM : TN);
        }
    }
};

// BinWindow with a third moment (the second velocity moment of the pressure variable): the
// same window and transfers for e_q, summed and added by lanes 4, 5 and a third transfer.
struct BinWindow3 {
    BinWindow w;
    int32_t e0, e1;
    long long te;

    __device__ __forceinline__ void begin(int k)
    {
        w.begin(k);
        e0 = e1 = 0;
        te = 0;
    }

    __device__ __forceinline__ void add(int b, int32_t wq, int32_t mq, int32_t eq, uint32_t tq, const BinGrid& gn,
                                        const BinGrid& gm, const BinGrid& ge)
    {
        const int d = (b - w.K) & (gn.nb - 1);
        if (d == 0) {
            e0 += eq;
            te += (long long)eq * (long long)tq;
        } else if (d == 1 && tq == 0u) {
            e1 += eq;
        } else {
            ge.add_whole(b, eq);
            if (tq) ge.add_transfer(b, (long long)eq * (long long)tq);
        }
        w.add(b, wq, mq, tq, gn, gm);
    }

    __device__ __forceinline__ void end(const BinGrid& gn, const BinGrid& gm, const BinGrid& ge) const
    {
        w.end(gn, gm);
        const int lane = threadIdx.x & 31;
        const int32_t E0 = __reduce_add_sync(0xFFFFFFFFu, e0), E1 = __reduce_add_sync(0xFFFFFFFFu, e1);
        const int32_t v = lane == 0 ? E0 : E1;
        if (lane < 2 && v != 0) ge.add_whole((w.K + lane) & (gn.nb - 1), v);
        if (__any_sync(0xFFFFFFFFu, te != 0)) {
            const long long TE = warp_sum64(0xFFFFFFFFu, te);
            if (lane == 0) ge.add_transfer(w.K, TE);
        }
    }
};

// Warp-uniform base bin of a group: the lowest of the lanes' bins b (where ok), compared
// periodically around lane 0's bin; all 32 lanes, converged.
__device__ __forceinline__ int warp_low_bin(int b, bool ok, int nb)
{
    const int ref = __shfl_sync(0xFFFFFFFFu, b, 0);
    const int h = nb >> 1;
    const int rel = ok ? ((b - ref + h) & (nb - 1)) - h : INT_MAX;
    const int lo = __reduce_min_sync(0xFFFFFFFFu, rel);
    return lo == INT_MAX ? (ref & (nb - 1)) : ((ref + lo) & (nb - 1));
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
