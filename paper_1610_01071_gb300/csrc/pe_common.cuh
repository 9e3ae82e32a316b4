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

// Block-local copy of a nodal int64 grid in shared memory. Either the full periodic
// grid (width == ncell, base == 0) or a window [base, base + width) of it; nodes
// outside the window go straight to the global grid.
struct SmemGrid {
    unsigned long long* s;
    unsigned long long* g;
    int base, width, mask;

    __device__ __forceinline__ void add(int node, unsigned long long val) const
    {
        int idx = (node - base) & mask;
        if (idx < width)
            atomicAdd(&s[idx], val);
        else
            atomicAdd(&g[node], val);
    }

    __device__ __forceinline__ void zero() const
    {
        for (int i = threadIdx.x; i < width; i += blockDim.x) s[i] = 0ull;
    }

    // Adds the non-zero entries to the global grid; call after __syncthreads().
    __device__ __forceinline__ void flush() const
    {
        for (int i = threadIdx.x; i < width; i += blockDim.x) {
            unsigned long long val = s[i];
            if (val) atomicAdd(&g[(base + i) & mask], val);
        }
    }
};

// Per-lane sliding accumulator for a stream of particles whose cells change slowly
// (particles sorted by cell): four consecutive nodes base..base+3 held in registers,
// flushed to the block grid only when a particle falls outside them.
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
        s0 += (d == 0) ? q.left : 0ull;
        s1 += (d == 0) ? q.right : ((d == 1) ? q.left : 0ull);
        s2 += (d == 1) ? q.right : ((d == 2) ? q.left : 0ull);
        s3 += (d == 2) ? q.right : 0ull;
    }
};

// Contiguous particle range [begin, end) of block b when n particles are split into
// nblocks chunks whose starts are multiples of 4 (so float4 loads stay aligned).
__device__ __forceinline__ void block_chunk(int64_t n, int64_t chunk, int64_t* begin, int64_t* end)
{
    int64_t b = (int64_t)blockIdx.x * chunk;
    *begin = b < n ? b : n;
    int64_t e = b + chunk;
    *end = e < n ? e : n;
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
