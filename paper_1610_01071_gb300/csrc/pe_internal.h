// Host-side helpers shared by the translation units of libpepic (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "pepic.h"

struct CUtensorMap_st;  // cuda.h's TMA tensor map

namespace pe {

// NVTX range over a context-level call (visible to a profiler's timeline; no cost without one).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

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

// Batched field solves (pe_field.cu): descriptor size, descriptor builder, cluster size
// used for a grid of ncell nodes, and the launch over R realisations of one cluster size.
size_t field_desc_size();
void make_field_desc(void* out, const int64_t* rho, int ncell, double dx, int s_w, int mode, int walls, double tol,
                     int maxit, double* phi, double* E, float* Ef, int32_t* diag, uint32_t* status,
                     double* phi_prev);
int newton_cluster_size(int ncell);
int newton_batch_cluster_size(int ncell);
int launch_newton_batch(const void* descs, int R, int G, int max_ncell, bool fp64, bool extrap, cudaStream_t s);
// Single field solve whose Newton start may extrapolate the solution history (context path).
int field_solve_history(const int64_t* rho_fx, int ncell, double dx, int s_w, int mode, int boundary, double tol,
                        int maxit, double* phi, double* E, float* Ef, int32_t* diag, uint32_t* status,
                        double* phi_prev, int extrap, cudaStream_t s);

// Grid of a particle pass (pe_particles.cu): one chunk of particles (a multiple of 4, at most
// max_chunk or 65536) per block, filling whole waves of resident blocks; returns the block count.
int particle_grid(const void* kernel, int block, size_t smem, int64_t n, int64_t* chunk, int64_t max_chunk = 0);

// pe_push_ex and pe_sample with their zeroing of the charge grid and of the sample row made
// optional (zero = false: the caller has zeroed both, e.g. all sample rows of a burst at once).
int push_pass(int32_t* cell, float* theta, float* v, float* w, int64_t n, const float* Ef, int32_t ncell,
              float dt_over_dx, float qm_dt, float kick, int32_t s_w, int32_t boundary, int64_t* rho_fx,
              const pe_sample_args* sample, uint32_t* status, void* stream, bool zero);
int sample_pass(const int32_t* cell, const float* theta, const float* v, const float* w, int64_t n, const float* Ef,
                int32_t ncell, float qm_dt, float kick, const pe_sample_args* sample, uint32_t* status, void* stream,
                bool zero);

// Batched particle passes (pe_particles.cu).
size_t push_desc_size();
size_t work_item_size();
void make_push_desc(void* out, int32_t* cell, float* theta, float* v, const float* w, int64_t n, const float* Ef,
                    int ncell, float dt_dx, float qm_dt, int s_w, int64_t* rho, const float* E0f, double dT, double dt,
                    float inv_dx, float qm, int comoving, int s_p, int bin_shift, int64_t* samp_base,
                    int64_t row_stride, int walls, uint32_t* status);
void make_work_item(void* out, int r, int64_t begin, int64_t end);
int launch_particles_batch(int mode, const void* descs, const void* items, int nitems, int p, float kick,
                           unsigned* counter, int max_ncell, int max_nb, int block, int priv, cudaStream_t s);

// Batched restriction + projection of Haar-binned samples (pe_coarse.cu).
size_t proj_desc_size();
void make_proj_desc(void* out, const int64_t* samp, int64_t row_stride, int ncell, int nc, int s_w, int s_p,
                    double* csamples, double* coarse, double* slope);
int launch_restrict_project_batch(const void* descs, int R, int K, double dt, double dT, cudaStream_t s);

// Batched lifting profiles (pe_coarse.cu): descriptor size and builder, and the launch over
// R realisations with the same wavelet.
size_t refine_desc_size();
void make_refine_desc(void* out, const double* coarse, int nc, int ncell, float* prof_n, float* prof_u);
int launch_refine_batch(const void* descs, int R, int wavelet, int max_ncell, cudaStream_t s);

// Kinetic electrons: folds the electrons' moments into the ions' (pe_diag.cu).
int combine_kinetic_moments(pe_moments* out, const pe_moments* electrons, double qm_e, cudaStream_t s);

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
constexpr int kWindowNodesE = 1024;    // the same with the second moment (three rows in shared memory)
// Bounded grids (vacuum regions, exp(phi) ~ 1e-6, cond(J) ~ 1e7) slow the FP32 Jacobian solve's
// contraction: about 7 Newton updates instead of 3 on the 8192-node slab from a warm start. Each
// FP32 update costs so much less than an FP64 one that the field solve is still faster (56 against
// 125 us on the slab), so the FP64 elimination stays compiled but unused (true selects it).
constexpr bool kWallsJacobianFP64 = false;
// TMA tensor map of a K-major BF16 GEMM operand: rows x K elements, row stride ld elements,
// box {64, box_rows}, 128-byte swizzle, zero fill (pe_tc.cu).
int tc_operand_map(::CUtensorMap_st* map, const void* base, int64_t rows, int64_t K, int64_t ld, int box_rows);
constexpr int kPSWindowBins = 64;      // phase-space samples: window of coarse x-bins

}  // namespace pe
