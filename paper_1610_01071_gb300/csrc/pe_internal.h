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

// Raises the kernel's dynamic shared-memory limit to at least smem bytes on the
// current device (cached, so repeated launches pay nothing).
int ensure_smem(const void* kernel, size_t smem);
// Resident blocks per SM for (kernel, block, smem) on the current device (cached).
int blocks_per_sm(const void* kernel, int block, size_t smem);

// Counts kernel launches (exported through pe_launch_count).
void note_launches(int n);

inline int launch_status(int kernels = 1)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return PE_ECUDA;
    note_launches(kernels);
    return PE_OK;
}

// Shared-memory grid widths used by the particle kernels (nodes).
constexpr int kFullGridMax = 8192;     // largest grid the context API accepts
constexpr int kRhoWindowNodes = 1024;  // charge deposit: window around the block's cells
constexpr int kWindowNodes = 4096;     // restriction samples: window (co-moving spread)

}  // namespace pe
