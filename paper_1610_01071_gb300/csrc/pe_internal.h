// Host-side helpers shared by the translation units of libpepic (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pepic.h"

namespace pe {

inline bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
inline int ilog2(int64_t x)
{
    int l = 0;
    while ((int64_t(1) << l) < x) ++l;
    return l;
}

// Number of SMs of the current device (cached per device).
int sm_count();
// Maximum dynamic shared memory per block (opt-in) of the current device.
int max_smem_optin();

// Counts kernel launches (exported through pe_launch_count).
void note_launches(int n);

inline int launch_status(int kernels = 1)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return PE_ECUDA;
    note_launches(kernels);
    return PE_OK;
}

// Shared-memory grid widths used by the particle kernels (nodes of int64).
constexpr int kFullGridMax = 8192;  // ncell up to this uses a block-private copy of the whole grid
constexpr int kWindowNodes = 4096;  // otherwise a window of this many nodes

}  // namespace pe
