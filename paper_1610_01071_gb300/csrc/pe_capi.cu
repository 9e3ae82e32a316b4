// Context API: one realisation of the projective-integration cycle (Section 3.1):
// lift -> K fine PIC steps with a restriction sample after each -> least-squares
// slope -> forward-Euler leap of the coarse variables; plus the plain PIC path.
// Host orchestration only: every step runs in the kernels of the other files.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "pe_ctx.h"
#include "pe_internal.h"
#include "pepic.h"

namespace pe {

int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev < 0 || dev >= 64) return 1;
    if (!cache[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = v > 0 ? v : 1;
    }
    return cache[dev];
}

int max_smem_optin()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
    if (dev < 0 || dev >= 64) return 48 * 1024;
    if (!cache[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cache[dev] = v > 0 ? v : 48 * 1024;
    }
    return cache[dev];
}

namespace {
struct KernelInfo {
    const void* kernel;
    int device, block;
    size_t smem;
    int value;
};
std::mutex g_kmu;
std::vector<KernelInfo> g_smem_set, g_occ;
}  // namespace

int ensure_smem(const void* kernel, size_t smem)
{
    // below 48 KB less the kernel's static shared memory no attribute is needed; the static size
    // is not known here, so every non-zero request goes through the per-kernel record
    if (smem == 0) return PE_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PE_ECUDA;
    std::lock_guard<std::mutex> lk(g_kmu);
    for (auto& k : g_smem_set)
        if (k.kernel == kernel && k.device == dev && k.smem >= smem) return PE_OK;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return PE_ECUDA;
    for (auto& k : g_smem_set)
        if (k.kernel == kernel && k.device == dev) {
            k.smem = smem;
            return PE_OK;
        }
    g_smem_set.push_back({kernel, dev, 0, smem, 0});
    return PE_OK;
}

int blocks_per_sm(const void* kernel, int block, size_t smem)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(g_kmu);
    for (auto& k : g_occ)
        if (k.kernel == kernel && k.device == dev && k.block == block && k.smem == smem) return k.value;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    g_occ.push_back({kernel, dev, block, smem, per_sm});
    return per_sm;
}

static std::atomic<long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static int fx_shift(double cap)
{
    int e = 0;
    double m = frexp(cap, &e);
    return 22 - ((m == 0.5) ? e - 1 : e);
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace pe

using namespace pe;

extern "C" PE_API int pe_fixed_point_shifts(int64_t nparticles, int32_t ncell, double w_cap, double v_cap,
                                            int32_t* s_w, int32_t* s_p)
{
    if (nparticles < 1 || ncell < 1 || !s_w || !s_p) return PE_EINVAL;
    const double wc = w_cap > 0.0 ? w_cap : 8.0 * ncell / (double)nparticles;
    const double vc = v_cap > 0.0 ? v_cap : 32.0;
    *s_w = fx_shift(wc);
    *s_p = fx_shift(wc * vc);
    return PE_OK;
}

extern "C" PE_API int pe_second_moment_shift(int64_t nparticles, int32_t ncell, double w_cap, double v_cap, int32_t* s_e)
{
    if (nparticles < 1 || ncell < 1 || !s_e) return PE_EINVAL;
    const double wc = w_cap > 0.0 ? w_cap : 8.0 * ncell / (double)nparticles;
    const double vc = v_cap > 0.0 ? v_cap : 32.0;
    *s_e = fx_shift(wc * vc * vc);
    return PE_OK;
}


extern "C" PE_API const char* pe_strerror(int code)
{
    switch (code) {
    case PE_OK: return "ok";
    case PE_EINVAL: return "invalid argument";
    case PE_ECUDA: return "CUDA runtime error";
    case PE_ENOCONV: return "Newton iteration did not converge";
    case PE_EOVERFLOW: return "fixed-point range exceeded (weight or momentum too large)";
    case PE_ERANGE: return "particle cell index out of range";
    case PE_ESTATE: return "call out of order for the context state";
    case PE_ETIMEOUT: return "a bounded device-side wait timed out";
    default: return "unknown error";
    }
}

extern "C" PE_API const char* pe_version(void) { return "pepic 0.1 (sm_103a)"; }

extern "C" PE_API int pe_layout_for(const pe_config* cfg, pe_layout* out)
{
    if (!cfg || !out) return PE_EINVAL;
    const pe_config& c = *cfg;
    if (!is_pow2(c.ncell) || c.ncell < 8 || c.ncell > kFullGridMax) return PE_EINVAL;
    if (!is_pow2(c.n_coarse) || c.n_coarse > c.ncell) return PE_EINVAL;
    if (c.K < 1 || c.K > 4096) return PE_EINVAL;
    if (c.nparticles < c.ncell || c.nparticles % c.ncell != 0 || c.nparticles >= (int64_t(1) << 32)) return PE_EINVAL;
    if (!(c.L > 0.0) || !(c.dt > 0.0) || !(c.dT >= c.K * c.dt * (1.0 - 1e-12)) || !(c.v_th >= 0.0)) return PE_EINVAL;
    if (c.wavelet != PE_WAVELET_HAAR && c.wavelet != PE_WAVELET_D4 && c.wavelet != PE_WAVELET_COIF4) return PE_EINVAL;
    if (c.poisson != PE_POISSON_BOLTZMANN && c.poisson != PE_POISSON_LINEARIZED) return PE_EINVAL;
    if (c.newton_maxit < 1 || !(c.newton_tol > 0.0) || c.sort_every < 0) return PE_EINVAL;
    if (c.w_cap < 0.0 || c.v_cap < 0.0) return PE_EINVAL;
    if (c.coarse_kind != PE_COARSE_MOMENTS && c.coarse_kind != PE_COARSE_PHASE_SPACE &&
        c.coarse_kind != PE_COARSE_MOMENTS_PRESSURE)
        return PE_EINVAL;
    const bool ps = c.coarse_kind == PE_COARSE_PHASE_SPACE;
    // ion pressure: nodal samples of three moments, lifting at the local temperature (periodic
    // grids, Boltzmann electrons; four FP64 rows of the grid in shared memory at the lift)
    const bool pres = c.coarse_kind == PE_COARSE_MOMENTS_PRESSURE;
    if (pres && (c.boundary != PE_BOUNDARY_PERIODIC || c.electrons != PE_ELECTRONS_BOLTZMANN || c.ncell > 4096))
        return PE_EINVAL;
    if (c.n_v_coarse < 0 || (c.n_v_coarse > 0 && !ps)) return PE_EINVAL;
    const bool psw = ps && c.n_v_coarse > 0;  // the wavelet form
    if (ps && !psw && (c.wavelet != PE_WAVELET_HAAR || c.n_v < 2 || c.n_v > 256 || !(c.v_max > 0.0))) return PE_EINVAL;
    if (psw && (!is_pow2(c.n_v) || c.n_v > 1024 || !is_pow2(c.n_v_coarse) || c.n_v_coarse < 2 ||
                c.n_v_coarse > c.n_v || !(c.v_max > 0.0) || c.ps_filter != 0 || c.boundary != PE_BOUNDARY_PERIODIC ||
                c.electrons != PE_ELECTRONS_BOLTZMANN || c.n_coarse < 2))
        return PE_EINVAL;
    if (c.ps_filter < 0 || c.ps_filter > 3) return PE_EINVAL;
    if (c.boundary != PE_BOUNDARY_PERIODIC && c.boundary != PE_BOUNDARY_ABSORBING) return PE_EINVAL;
    const bool walls = c.boundary == PE_BOUNDARY_ABSORBING;
    if (c.electrons != PE_ELECTRONS_BOLTZMANN && c.electrons != PE_ELECTRONS_KINETIC) return PE_EINVAL;
    const bool kin = c.electrons == PE_ELECTRONS_KINETIC;
    // kinetic electrons: periodic grids, the exponential Boltzmann relation for the lifting,
    // a negative charge-to-mass ratio (0 selects the default)
    if (kin && (walls || c.poisson != PE_POISSON_BOLTZMANN || !(c.qm_e <= 0.0) || !(c.v_th_e >= 0.0) ||
                c.reset_every < 0))
        return PE_EINVAL;
    if (c.te_active != 0 && (c.te_active != 1 || !kin)) return PE_EINVAL;  // an electron temperature needs electrons
    const bool te = c.te_active == 1;
    memset(out, 0, sizeof(*out));
    const size_t N = (size_t)c.nparticles, nc = (size_t)c.ncell, ncoef = (size_t)c.n_coarse;
    const size_t nps = ps ? ncoef * (size_t)c.n_v : 0;                 // phase-space sample row
    const size_t npc = psw ? ncoef * (size_t)c.n_v_coarse : nps;         // phase-space coefficients
    const size_t row_fx = pres ? 3 * nc : (2 * nc > nps ? 2 * nc : nps);
    const size_t crow = pres ? 3 * ncoef : (2 * ncoef > npc ? 2 * ncoef : npc);
    const size_t bank = 4 * align256(4 * N);
    out->bytes[PE_BUF_PARTICLES_A] = bank;
    out->bytes[PE_BUF_PARTICLES_B] = bank;
    out->bytes[PE_BUF_RHO] = 8 * nc;
    out->bytes[PE_BUF_PHI] = 8 * 2 * nc;  // phi and the previous solution (Newton start)
    out->bytes[PE_BUF_E] = 8 * nc;
    out->bytes[PE_BUF_EF] = 4 * nc;
    out->bytes[PE_BUF_E0F] = 4 * nc;
    out->bytes[PE_BUF_SAMPLES_FX] = 8 * row_fx * (size_t)(c.K + 2);
    out->bytes[PE_BUF_COARSE_SAMPLES] = 8 * crow * (size_t)(c.K + 2);
    out->bytes[PE_BUF_COARSE] = 8 * crow;
    out->bytes[PE_BUF_SLOPE] = 8 * crow;
    out->bytes[PE_BUF_PROFILE] = 4 * (pres ? 3 : 2) * nc;
    out->bytes[PE_BUF_SORT] = 4 * (2 * nc + 64);
    out->bytes[PE_BUF_STATUS] = 64;
    out->bytes[PE_BUF_DIAG] = PE_MOMENTS_SCRATCH_BYTES + 256;
    out->bytes[PE_BUF_SURROGATE] = align256(8 * 2 * ncoef) + 256;
    out->bytes[PE_BUF_PHASE] = (ps ? align256(8 * ncoef) + align256(8 * ncoef * (size_t)(c.n_v + 1)) +
                                         align256(8 * 2 * ncoef * (size_t)(c.n_v + 1)) +
                                         align256(4 * ncoef * (size_t)(3 * c.n_v + 1)) + 256
                                   : 256) +
                                (psw ? align256(8 * ncoef * (size_t)c.n_v) + align256(4 * nc * (size_t)(3 * c.n_v + 1)) +
                                           align256(4 * nc)
                                     : 0) +
                                (walls ? align256(PE_PS_EQ_SCRATCH_BYTES(nc)) : 0);
    out->bytes[PE_BUF_ELECTRONS_A] = kin ? bank : 0;
    out->bytes[PE_BUF_ELECTRONS_B] = kin ? bank : 0;
    // electron deposit + ion moments [2][ncell]; te_active: K + 2 energy samples, the projected
    // energy and its slope
    out->bytes[PE_BUF_RHO_E] = kin ? 8 * 3 * nc + (te ? 8 * (size_t)(c.K + 4) : 0) : 0;
    size_t off = 0;
    for (int b = 0; b < PE_NBUF; ++b) {
        out->offset[b] = off;
        off += align256(out->bytes[b]);
    }
    out->total_bytes = off;
    return PE_OK;
}

extern "C" PE_API int pe_create(const pe_config* cfg, void* arena, size_t arena_bytes, void* stream, pe_ctx** out)
{
    if (!out) return PE_EINVAL;
    *out = nullptr;
    pe_layout lay;
    PE_TRY(pe_layout_for(cfg, &lay));
    if (!arena || ((uintptr_t)arena & 255u) || arena_bytes < lay.total_bytes) return PE_EINVAL;
    pe_ctx* x = (pe_ctx*)calloc(1, sizeof(pe_ctx));
    if (!x) return PE_EINVAL;
    x->cfg = *cfg;
    x->lay = lay;
    x->arena = (char*)arena;
    x->stream = (cudaStream_t)stream;
    x->dx = cfg->L / cfg->ncell;
    x->dT_cur = cfg->dT;
    x->K_cur = cfg->K;
    x->nc = cfg->n_coarse;
    x->ps = cfg->coarse_kind == PE_COARSE_PHASE_SPACE;
    x->psw = x->ps && cfg->n_v_coarse > 0;
    x->pres = cfg->coarse_kind == PE_COARSE_MOMENTS_PRESSURE;
    // Haar moments (with or without the pressure) and both phase-space forms restrict over 2^b
    // nodes in x (bins or hat rows)
    x->bin_shift = (cfg->wavelet == PE_WAVELET_HAAR || x->ps) ? ilog2(cfg->ncell / cfg->n_coarse) : 0;
    x->nb = cfg->ncell >> x->bin_shift;
    x->nv = x->ps ? cfg->n_v : 0;
    x->nvc = x->psw ? cfg->n_v_coarse : x->nv;
    x->vmin = x->ps ? -cfg->v_max : 0.0;
    x->dv = x->ps ? 2.0 * cfg->v_max / cfg->n_v : 1.0;
    x->ncoef = x->ps ? (int64_t)x->nc * x->nvc : (x->pres ? 3 : 2) * (int64_t)x->nc;
    const int64_t nps = x->ps ? (int64_t)x->nc * x->nv : 0;  // phase-space sample row
    x->row_fx = x->pres ? 3 * (int64_t)x->nb : (2 * (int64_t)x->nb > nps ? 2 * (int64_t)x->nb : nps);
    x->crow = x->pres ? x->ncoef : (2 * (int64_t)x->nc > (x->ps ? x->ncoef : 0) ? 2 * (int64_t)x->nc : x->ncoef);
    const double w_cap = cfg->w_cap > 0.0 ? cfg->w_cap : 8.0 * cfg->ncell / (double)cfg->nparticles;
    const double v_cap = cfg->v_cap > 0.0 ? cfg->v_cap : 32.0;
    x->s_w = fx_shift(w_cap);
    x->s_p = fx_shift(w_cap * v_cap);
    x->s_e = fx_shift(w_cap * v_cap * v_cap);
    const size_t N = (size_t)cfg->nparticles;
    for (int b = 0; b < 2; ++b) {
        char* base = x->arena + lay.offset[PE_BUF_PARTICLES_A + b];
        x->cell[b] = (int32_t*)base;
        x->theta[b] = (float*)(base + align256(4 * N));
        x->v[b] = (float*)(base + 2 * align256(4 * N));
        x->w[b] = (float*)(base + 3 * align256(4 * N));
    }
    x->rho = (int64_t*)(x->arena + lay.offset[PE_BUF_RHO]);
    x->kinetic = cfg->electrons == PE_ELECTRONS_KINETIC;
    x->qm_e = cfg->qm_e != 0.0 ? cfg->qm_e : -1800.0;
    x->v_th_e = cfg->v_th_e > 0.0 ? cfg->v_th_e : sqrt(-x->qm_e);
    if (x->kinetic) {
        for (int b = 0; b < 2; ++b) {
            char* base = x->arena + lay.offset[PE_BUF_ELECTRONS_A + b];
            x->ecell[b] = (int32_t*)base;
            x->etheta[b] = (float*)(base + align256(4 * N));
            x->ev[b] = (float*)(base + 2 * align256(4 * N));
            x->ew[b] = (float*)(base + 3 * align256(4 * N));
        }
        x->rho_e = (int64_t*)(x->arena + lay.offset[PE_BUF_RHO_E]);
        x->te_active = cfg->te_active;
        if (x->te_active) x->we = (double*)(x->rho_e + 3 * (size_t)cfg->ncell);
    }
    x->te = 1.0;
    x->phi = (double*)(x->arena + lay.offset[PE_BUF_PHI]);
    x->E = (double*)(x->arena + lay.offset[PE_BUF_E]);
    x->Ef = (float*)(x->arena + lay.offset[PE_BUF_EF]);
    x->E0f = (float*)(x->arena + lay.offset[PE_BUF_E0F]);
    x->samples = (int64_t*)(x->arena + lay.offset[PE_BUF_SAMPLES_FX]);
    x->csamples = (double*)(x->arena + lay.offset[PE_BUF_COARSE_SAMPLES]);
    x->coarse = (double*)(x->arena + lay.offset[PE_BUF_COARSE]);
    x->slope = (double*)(x->arena + lay.offset[PE_BUF_SLOPE]);
    x->prof = (float*)(x->arena + lay.offset[PE_BUF_PROFILE]);
    x->sort = (int32_t*)(x->arena + lay.offset[PE_BUF_SORT]);
    x->status = (uint32_t*)(x->arena + lay.offset[PE_BUF_STATUS]);
    x->diag = (int32_t*)(x->status + 4);
    {
        char* ph = x->arena + lay.offset[PE_BUF_PHASE];
        const size_t nc_ = (size_t)x->nc, nv1 = (size_t)x->nv + 1;
        x->ps_mass = (double*)ph;
        x->ps_cdf = (double*)(ph + align256(8 * nc_));
        x->ps_scratch = (double*)(ph + align256(8 * nc_) + align256(8 * nc_ * nv1));
        x->ps_table = (float*)(ph + align256(8 * nc_) + align256(8 * nc_ * nv1) + align256(8 * 2 * nc_ * nv1));
        x->ps_flags = (int32_t*)((char*)x->ps_table + align256(4 * nc_ * (3 * (size_t)x->nv + 1)));
        if (!x->ps) x->ps_flags = (int32_t*)ph;
        x->walls = cfg->boundary == PE_BOUNDARY_ABSORBING;
        // equal-weight loading scratch after the phase-space tables (bounded grids)
        const size_t ps_bytes = x->ps ? align256(8 * nc_) + align256(8 * nc_ * nv1) + align256(8 * 2 * nc_ * nv1) +
                                             align256(4 * nc_ * (3 * (size_t)x->nv + 1)) + 256
                                       : 256;
        x->eq_scratch = x->walls ? (void*)(ph + ps_bytes) : nullptr;
        if (x->psw) {  // after the phase-space tables (the wavelet form has no walls)
            char* q = ph + ps_bytes;
            x->ps_hist = (double*)q;
            q += align256(8 * nc_ * (size_t)x->nv);
            x->ps_node_table = (float*)q;
            q += align256(4 * (size_t)cfg->ncell * (3 * (size_t)x->nv + 1));
            x->ps_node_dens = (float*)q;
        }
    }
    if (cudaMemsetAsync(x->arena + lay.offset[PE_BUF_PHI], 0, lay.bytes[PE_BUF_PHI], x->stream) != cudaSuccess ||
        cudaMemsetAsync(x->status, 0, 64, x->stream) != cudaSuccess) {
        free(x);
        return PE_ECUDA;
    }
    *out = x;
    return PE_OK;
}

static void destroy_events(std::vector<cudaEvent_t>* v)
{
    if (!v) return;
    for (cudaEvent_t e : *v) cudaEventDestroy(e);
    delete v;
}

extern "C" PE_API void pe_destroy(pe_ctx* ctx)
{
    if (!ctx) return;
    for (int k = 0; k < PE_PROF_NKINDS; ++k) destroy_events(ctx->prof_ev[k]);
    free(ctx);
}

extern "C" PE_API int64_t pe_launch_count(void) { return g_launches.load(); }

// Records the event with index 2*slot (+1 for stop) of the pool, creating it on demand.
static int record(pe_ctx* x, std::vector<cudaEvent_t>*& pool, size_t slot, int stop)
{
    if (!pool) pool = new std::vector<cudaEvent_t>();
    const size_t i = 2 * slot + (size_t)stop;
    while (pool->size() <= i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return PE_ECUDA;
        pool->push_back(e);
    }
    return cudaEventRecord((*pool)[i], x->stream) == cudaSuccess ? PE_OK : PE_ECUDA;
}

// Wraps one launch in a start/stop event pair of the given kind (PE_PROF_*) when profiling is on.
template <class F>
static int timed(pe_ctx* x, int kind, F&& launch)
{
    if (!((x->profiling >> kind) & 1)) return launch();
    size_t& n = x->prof_n[kind];
    PE_TRY(record(x, x->prof_ev[kind], n, 0));
    PE_TRY(launch());
    PE_TRY(record(x, x->prof_ev[kind], n, 1));
    ++n;
    return PE_OK;
}

extern "C" PE_API int pe_profile(pe_ctx* ctx, int32_t enable)
{
    if (!ctx) return PE_EINVAL;
    ctx->profiling = enable ? (1 << PE_PROF_NKINDS) - 1 : 0;
    return PE_OK;
}

extern "C" PE_API int pe_profile_mask(pe_ctx* ctx, int32_t kinds)
{
    if (!ctx || kinds < 0 || kinds >= (1 << PE_PROF_NKINDS)) return PE_EINVAL;
    ctx->profiling = kinds;
    return PE_OK;
}

static double sum_pairs(std::vector<cudaEvent_t>* pool, size_t n)
{
    double tot = 0.0;
    for (size_t k = 0; k < n; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, (*pool)[2 * k], (*pool)[2 * k + 1]) == cudaSuccess) tot += ms;
    }
    return tot;
}

extern "C" PE_API int pe_profile_read_kinds(pe_ctx* ctx, double* ms, int64_t* launches)
{
    if (!ctx || !ms || !launches) return PE_EINVAL;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PE_ECUDA;
    for (int k = 0; k < PE_PROF_NKINDS; ++k) {
        ms[k] = ctx->prof_n[k] ? sum_pairs(ctx->prof_ev[k], ctx->prof_n[k]) : 0.0;
        launches[k] = (int64_t)ctx->prof_n[k];
        ctx->prof_n[k] = 0;
    }
    return PE_OK;
}

extern "C" PE_API int pe_profile_read(pe_ctx* ctx, double* push_ms, int64_t* push_launches, double* field_ms,
                                      int64_t* field_launches)
{
    double ms[PE_PROF_NKINDS];
    int64_t n[PE_PROF_NKINDS];
    PE_TRY(pe_profile_read_kinds(ctx, ms, n));
    double pm = 0.0;
    int64_t pn = 0;
    for (int k = 0; k < PE_PROF_NKINDS; ++k)
        if (k != PE_PROF_FIELD) {
            pm += ms[k];
            pn += n[k];
        }
    if (push_ms) *push_ms = pm;
    if (push_launches) *push_launches = pn;
    if (field_ms) *field_ms = ms[PE_PROF_FIELD];
    if (field_launches) *field_launches = n[PE_PROF_FIELD];
    return PE_OK;
}

// Field solve of the current charge. mode 0: a solve outside the time stepping (measurement,
// diagnostics): the solution history is left alone. mode 1: the solve that starts a burst or a
// plain-PIC step: records the history; its Newton start extrapolates the last two solutions
// when they belong to the same trajectory one fine step apart (phi_hist).
static int field_solve(pe_ctx* x, int step = 0)
{
    const pe_config& c = x->cfg;
    if (x->kinetic)  // Section 4.1's two-species bursts: Poisson for the net charge
        return timed(x, PE_PROF_FIELD, [&] {
            return pe_field_kinetic(x->rho, x->rho_e, c.ncell, x->dx, x->s_w, x->phi, x->E, x->Ef, x->stream);
        });
    const int extrap = step && x->phi_hist;
    double* prev = step ? x->phi + c.ncell : nullptr;
    PE_TRY(timed(x, PE_PROF_FIELD, [&] {
        return field_solve_history(x->rho, c.ncell, x->dx, x->s_w, c.poisson, c.boundary, c.newton_tol,
                                   c.newton_maxit, x->phi, x->E, x->Ef, x->diag, x->status, prev, extrap, x->stream);
    }));
    if (step) x->phi_hist = 1;
    return PE_OK;
}

static int deposit_current(pe_ctx* x)
{
    const int b = x->bank;
    PE_TRY(timed(x, PE_PROF_DEPOSIT, [&] {
        return pe_deposit(x->cell[b], x->theta[b], x->w[b], x->cfg.nparticles, x->cfg.ncell, x->s_w, x->rho,
                          x->status, x->stream);
    }));
    if (x->kinetic) {
        const int e = x->ebank;
        PE_TRY(pe_deposit(x->ecell[e], x->etheta[e], x->ew[e], x->cfg.nparticles, x->cfg.ncell, x->s_w, x->rho_e,
                          x->status, x->stream));
    }
    x->rho_valid = 1;
    return PE_OK;
}

// Electrons in Boltzmann equilibrium with the current ions (Eq. electronpassive: n_e = exp(phi),
// V_e = V_i, T_e = T_e0), as the lifting of Section 3.3 places them and as Section 4.1's reset
// runs reload them: the Poisson-Boltzmann potential of the ion density, then a quiet start on
// exp(phi) with the electrons' thermal speed, drifting with the ions' mean velocity. Leaves
// their deposit in rho_e.
static uint64_t electron_seed(uint64_t s) { return s ^ 0xD1B54A32D192ED03ULL; }

// Where the ions' mean velocity for V_e = V_i comes from: the lifting profile already in
// PE_BUF_PROFILE's u half (a load or a moment lift), the phase-space coarse state (a
// phase-space lift), or a moment sample of the ion particles (a plain-PIC reset).
enum ElectronDrift { kDriftProfile, kDriftPhaseSpace, kDriftParticles };

// The electrons' total kinetic energy sum w Vbar^2 dx / 2 (pe_compute_moments' kinetic term, Vbar
// at integer time in the current field) into we[row] (device): the global active variable of
// Section 4.2.
static int electron_energy_sample(pe_ctx* x, int row)
{
    const pe_config& c = x->cfg;
    double* scratch = (double*)(x->arena + x->lay.offset[PE_BUF_DIAG]);
    const int e = x->ebank;
    const float kick = x->e_v_at_integer ? 0.5f : 1.0f;
    return pe_kinetic_energy(x->ecell[e], x->etheta[e], x->ev[e], x->ew[e], c.nparticles, x->Ef, c.ncell, x->dx,
                             (float)(x->qm_e * c.dt), kick, scratch, x->we + row, x->status, x->stream);
}

// Electrons at temperature te (units of T_e0): the Poisson-Boltzmann potential with
// n_e = exp(phi / te) is solved for psi = phi / te, -te psi'' + e^psi = n_i, i.e. the same
// Newton at the grid step dx / sqrt(te); the quiet start loads exp(psi) with v_th_e sqrt(te).
static int load_boltzmann_electrons(pe_ctx* x, uint64_t seed, ElectronDrift drift, double te = 1.0)
{
    const pe_config& c = x->cfg;
    float* u = x->prof + c.ncell;
    int64_t* mom = nullptr;
    if (drift == kDriftParticles) {
        // the ions' nodal density and momentum at their stored velocities (kick 1/2: Vbar = v,
        // half a step before integer time in a plain-PIC reset)
        mom = x->rho_e + c.ncell;
        pe_sample_args a;
        memset(&a, 0, sizeof(a));
        a.E0f = x->Ef;  // tau = 0: the frame field is not used
        a.qm = (float)c.qm;
        a.inv_dx = (float)(1.0 / x->dx);
        a.s_w = x->s_w;
        a.s_p = x->s_p;
        a.sample_fx = mom;
        a.boundary = c.boundary;
        const int b = x->bank;
        PE_TRY(pe_sample(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, x->Ef, c.ncell,
                         (float)(c.qm * c.dt), 0.5f, &a, x->status, x->stream));
    } else if (drift == kDriftPhaseSpace) {
        PE_TRY(pe_ps_mean_velocity(x->ps_cdf, x->nc, x->nv, x->vmin, x->dv, x->bin_shift, c.ncell, u, x->stream));
    }
    PE_TRY(field_solve_history(x->rho, c.ncell, x->dx / sqrt(te), x->s_w, PE_POISSON_BOLTZMANN,
                               PE_BOUNDARY_PERIODIC, c.newton_tol, c.newton_maxit, x->phi, x->E, x->Ef, x->diag,
                               x->status, nullptr, 0, x->stream));
    PE_TRY(pe_boltzmann_profile(x->phi, mom, x->s_w, x->s_p, c.ncell, x->prof, mom ? u : nullptr, x->stream));
    const int e = x->ebank;
    PE_TRY(timed(x, PE_PROF_LOAD, [&] {
        return pe_quiet_start(x->ecell[e], x->etheta[e], x->ev[e], x->ew[e], c.nparticles, c.ncell, x->prof, u,
                              (float)(x->v_th_e * sqrt(te)), seed, x->s_w, x->rho_e, x->status, x->stream);
    }));
    x->e_v_at_integer = 1;
    return PE_OK;
}

// Electron push of a fine step (kinetic electrons), in the field Ef of the ions' push.
static int push_electrons(pe_ctx* x)
{
    const pe_config& c = x->cfg;
    const int e = x->ebank;
    const float kick = x->e_v_at_integer ? 0.5f : 1.0f;
    PE_TRY(timed(x, PE_PROF_PUSH, [&] {
        return pe_push_ex(x->ecell[e], x->etheta[e], x->ev[e], x->ew[e], c.nparticles, x->Ef, c.ncell,
                          (float)(c.dt / x->dx), (float)(x->qm_e * c.dt), kick, x->s_w, c.boundary, x->rho_e, nullptr,
                          x->status, x->stream);
    }));
    x->e_v_at_integer = 0;
    return PE_OK;
}

static int64_t* sample_row(pe_ctx* x, int p) { return x->samples + (size_t)p * (size_t)x->row_fx; }

static pe_sample_args sample_args(pe_ctx* x, double tau, int64_t* dst)
{
    pe_sample_args a;
    memset(&a, 0, sizeof(a));  // n_v = 0: moment sample
    a.bin_shift = x->bin_shift;
    a.E0f = x->E0f;
    a.tau = (float)tau;
    a.qm = (float)x->cfg.qm;
    a.inv_dx = (float)(1.0 / x->dx);
    a.s_w = x->s_w;
    a.s_p = x->s_p;
    a.sample_fx = dst;
    a.boundary = x->cfg.boundary;
    a.second_moment = x->pres;  // Section 3.2: the pressure's second moment beside n and nV
    a.s_e = x->s_e;
    if (x->ps) {  // Section 3.3 phase-space histogram instead of the moments
        a.n_v = x->nv;
        a.v_min = (float)x->vmin;
        a.inv_dv = (float)(1.0 / x->dv);
        a.x_tent = x->psw;  // wavelet form: coarse nodes of the repeated 1-2-1 rule
    }
    return a;
}

// Quiet start on the profiles in PE_BUF_PROFILE. Bounded grids load equal weights in
// proportion to the mass; wall_factor 2 when the profile's wall nodes hold deposits (a
// lifted restriction), 1 when they hold densities (an analytic initial profile).
static int quiet_start_from_profile(pe_ctx* x, uint64_t seed, float wall_factor)
{
    const pe_config& c = x->cfg;
    const int b = x->bank;
    PE_TRY(timed(x, PE_PROF_LOAD, [&] {
        if (x->walls)
            return pe_quiet_start_equal(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, c.ncell, x->prof,
                                        x->prof + c.ncell, wall_factor, (float)c.v_th, seed, x->s_w, x->eq_scratch,
                                        x->rho, x->status, x->stream);
        return pe_quiet_start(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, c.ncell, x->prof,
                              x->prof + c.ncell, (float)c.v_th, seed, x->s_w, x->rho, x->status, x->stream);
    }));
    x->rho_valid = 1;
    x->v_at_integer = 1;
    x->fresh = 1;
    x->phi_hist = 0;
    return PE_OK;
}

static uint64_t lift_seed(const pe_ctx* x) { return x->cfg.seed + 0x632BE59BD9B4E019ULL * (uint64_t)(x->macro_steps + 1); }

int pe_ctx_field_solve(pe_ctx* x) { return field_solve(x); }
uint64_t pe_ctx_lift_seed(const pe_ctx* x) { return lift_seed(x); }

extern "C" PE_API int pe_measure(pe_ctx* ctx, double* out, int32_t out_on_device)
{
    NvtxRange nvtx("pe_measure");
    if (!ctx || !out) return PE_EINVAL;
    pe_ctx* x = ctx;
    const pe_config& c = x->cfg;
    if (!x->rho_valid) PE_TRY(deposit_current(x));
    PE_TRY(field_solve(x));
    int64_t* dst = sample_row(x, c.K + 1);
    pe_sample_args a = sample_args(x, 0.0, dst);
    a.E0f = x->Ef;  // tau = 0: the frame field is not used
    a.n_v = 0;      // the measurement is always the density and momentum coefficients
    a.second_moment = 0;
    const int b = x->bank;
    const float kick = x->v_at_integer ? 0.5f : 1.0f;
    PE_TRY(pe_sample(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, x->Ef, c.ncell, (float)(c.qm * c.dt), kick,
                     &a, x->status, x->stream));
    double* cdst = x->csamples + (size_t)(c.K + 1) * (size_t)x->crow;
    PE_TRY(pe_coarsen(dst, 1, c.ncell, x->s_w, x->s_p, c.wavelet, x->nc, x->bin_shift, cdst, x->stream));
    const size_t bytes = sizeof(double) * 2 * x->nc;
    if (cudaMemcpyAsync(out, cdst, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        x->stream) != cudaSuccess)
        return PE_ECUDA;
    if (!out_on_device && cudaStreamSynchronize(x->stream) != cudaSuccess) return PE_ECUDA;
    return PE_OK;
}

// Density, momentum and second-moment coefficients of the current particles (the pressure
// variable's [3][n_coarse], tau = 0) into out (device).
static int measure_pressure(pe_ctx* x, double* out)
{
    const pe_config& c = x->cfg;
    if (!x->rho_valid) PE_TRY(deposit_current(x));
    PE_TRY(field_solve(x));
    int64_t* dst = sample_row(x, c.K + 1);
    pe_sample_args a = sample_args(x, 0.0, dst);
    a.E0f = x->Ef;
    const int b = x->bank;
    const float kick = x->v_at_integer ? 0.5f : 1.0f;
    PE_TRY(pe_sample(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, x->Ef, c.ncell, (float)(c.qm * c.dt), kick,
                     &a, x->status, x->stream));
    return pe_coarsen_pressure(dst, 1, c.ncell, x->s_w, x->s_p, x->s_e, c.wavelet, x->nc, x->bin_shift, out,
                               x->stream);
}

// Phase-space cell masses of the current particles (co-moving sample with tau = 0) into
// out[ncoef] (device).
static int measure_phase(pe_ctx* x, double* out)
{
    const pe_config& c = x->cfg;
    if (!x->rho_valid) PE_TRY(deposit_current(x));
    PE_TRY(field_solve(x));
    int64_t* dst = sample_row(x, c.K + 1);
    pe_sample_args a = sample_args(x, 0.0, dst);
    a.E0f = x->Ef;
    const int b = x->bank;
    const float kick = x->v_at_integer ? 0.5f : 1.0f;
    PE_TRY(pe_sample(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, x->Ef, c.ncell, (float)(c.qm * c.dt), kick,
                     &a, x->status, x->stream));
    if (x->psw) return pe_ps_coarsen_v(dst, x->nc, x->nv, x->s_w, x->bin_shift, c.wavelet, x->nvc, out, x->stream);
    return pe_ps_coarsen(dst, 1, x->ncoef, x->s_w, out, x->stream);
}

extern "C" PE_API int pe_initial_profile(int32_t profile, int32_t ncell, double L, double amplitude, float* prof_n,
                                         float* prof_u)
{
    if ((profile != PE_PROFILE_SINE && profile != PE_PROFILE_SLAB) || ncell < 1 || !(L > 0.0) || !prof_n || !prof_u)
        return PE_EINVAL;
    const double dx = L / ncell;
    for (int j = 0; j < ncell; ++j) {
        if (profile == PE_PROFILE_SLAB) {  // uniform slab on the central eighth, vacuum elsewhere
            prof_n[j] = (j >= 7 * ncell / 16 && j <= 9 * ncell / 16) ? 1.0f : 0.0f;
            prof_u[j] = 0.0f;
            continue;
        }
        const double xj = j * dx;
        const double pert = amplitude * cos(2.0 * M_PI * xj / L);
        prof_n[j] = (float)(1.0 + pert);
        prof_u[j] = (float)pert;
    }
    return PE_OK;
}

extern "C" PE_API int pe_load_initial(pe_ctx* ctx, int32_t profile, double amplitude)
{
    NvtxRange nvtx("pe_load_initial");
    if (!ctx || (profile != PE_PROFILE_SINE && profile != PE_PROFILE_SLAB)) return PE_EINVAL;
    pe_ctx* x = ctx;
    const pe_config& c = x->cfg;
    if (profile == PE_PROFILE_SLAB && !x->walls) return PE_EINVAL;
    std::vector<float> h(2 * (size_t)c.ncell);
    PE_TRY(pe_initial_profile(profile, c.ncell, c.L, amplitude, h.data(), h.data() + c.ncell));
    if (cudaMemcpyAsync(x->prof, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, x->stream) != cudaSuccess)
        return PE_ECUDA;
    if (cudaStreamSynchronize(x->stream) != cudaSuccess) return PE_ECUDA;  // host buffer goes out of scope
    if (cudaMemsetAsync(x->phi, 0, sizeof(double) * c.ncell, x->stream) != cudaSuccess) return PE_ECUDA;
    x->bank = 0;
    x->macro_steps = 0;
    x->fine_steps = 0;
    x->time = 0.0;
    x->coarse_state = 0;
    PE_TRY(quiet_start_from_profile(x, c.seed, 1.0f));
    if (x->kinetic) {
        x->ebank = 0;
        x->te = 1.0;
        PE_TRY(load_boltzmann_electrons(x, electron_seed(c.seed), kDriftProfile));
        if (x->te_active) {  // the reference energy of T_e = T_e0
            PE_TRY(electron_energy_sample(x, c.K + 2));
            double w = 0.0;
            if (cudaMemcpyAsync(&w, x->we + (c.K + 2), sizeof(w), cudaMemcpyDeviceToHost, x->stream) != cudaSuccess ||
                cudaStreamSynchronize(x->stream) != cudaSuccess)
                return PE_ECUDA;
            x->we_ref = w;
            x->we_last = w;
        }
    }
    if (x->ps) return measure_phase(x, x->coarse);
    if (x->pres) return measure_pressure(x, x->coarse);
    return pe_measure(x, x->coarse, 1);
}

// Fine steps p_begin .. p_end-1 of a burst, each a fused push + co-moving sample of row p
// followed by a field solve; then, with final_sample, the sample-only row p_end. A burst
// that starts (p_begin == 0) first solves the field of the current particles and keeps it
// as the frame field E_n (Appendix B). A later range continues the same burst.
int pe_ctx_burst_range(pe_ctx* x, int p_begin, int p_end, int final_sample)
{
    const pe_config& c = x->cfg;
    if (p_begin < 0 || p_end < p_begin || p_end > x->K_cur) return PE_EINVAL;
    const int b = x->bank;
    if (p_begin == 0) {
        if (!x->rho_valid) PE_TRY(deposit_current(x));
        x->phi_hist = 0;  // a burst starts a new stretch of trajectory (after a lift or a load)
        PE_TRY(field_solve(x, 1));
        if (cudaMemcpyAsync(x->E0f, x->Ef, sizeof(float) * c.ncell, cudaMemcpyDeviceToDevice, x->stream) != cudaSuccess)
            return PE_ECUDA;
    }
    float kick = x->v_at_integer ? 0.5f : 1.0f;
    const float dt_dx = (float)(c.dt / x->dx), qm_dt = (float)(c.qm * c.dt);
    // the sample rows of the range accumulate from zero: cleared at once here, not per pass
    const int last_row = final_sample ? p_end : p_end - 1;
    if (last_row >= p_begin &&
        cudaMemsetAsync(sample_row(x, p_begin), 0, sizeof(int64_t) * (size_t)x->row_fx * (size_t)(last_row - p_begin + 1),
                        x->stream) != cudaSuccess)
        return PE_ECUDA;
    for (int p = p_begin; p < p_end; ++p) {
        if (x->te_active) PE_TRY(electron_energy_sample(x, p));
        const double tau = c.comoving ? x->dT_cur - p * c.dt : 0.0;
        pe_sample_args a = sample_args(x, tau, sample_row(x, p));
        if (cudaMemsetAsync(x->rho, 0, sizeof(int64_t) * (size_t)c.ncell, x->stream) != cudaSuccess) return PE_ECUDA;
        PE_TRY(timed(x, x->ps ? PE_PROF_PUSH_SAMPLE_PS : PE_PROF_PUSH_SAMPLE, [&] {
            return push_pass(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, x->Ef, c.ncell, dt_dx, qm_dt,
                             kick, x->s_w, c.boundary, x->rho, &a, x->status, x->stream, false);
        }));
        if (x->kinetic) PE_TRY(push_electrons(x));
        PE_TRY(field_solve(x, 1));
        kick = 1.0f;
        x->v_at_integer = 0;
        x->rho_valid = 1;
        x->fine_steps += 1;
    }
    if (final_sample) {
        if (x->te_active) PE_TRY(electron_energy_sample(x, p_end));
        const double tau = c.comoving ? x->dT_cur - p_end * c.dt : 0.0;
        pe_sample_args a = sample_args(x, tau, sample_row(x, p_end));
        PE_TRY(timed(x, PE_PROF_SAMPLE, [&] {
            return sample_pass(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, x->Ef, c.ncell, qm_dt, kick, &a,
                               x->status, x->stream, false);
        }));
    }
    x->fresh = 0;
    return PE_OK;
}

extern "C" PE_API int pe_burst(pe_ctx* ctx)
{
    NvtxRange nvtx("pe_burst");
    if (!ctx) return PE_EINVAL;
    return pe_ctx_burst_range(ctx, 0, ctx->K_cur, 1);
}

extern "C" PE_API int pe_restrict(pe_ctx* ctx)
{
    NvtxRange nvtx("pe_restrict");
    if (!ctx) return PE_EINVAL;
    const pe_config& c = ctx->cfg;
    if (ctx->psw)  // rows of consecutive samples are contiguous: [K+1][n_coarse][n_vf] -> [K+1][n_coarse][n_vc]
        return pe_ps_coarsen_v(ctx->samples, (int64_t)(ctx->K_cur + 1) * ctx->nc, ctx->nv, ctx->s_w, ctx->bin_shift,
                               c.wavelet, ctx->nvc, ctx->csamples, ctx->stream);
    if (ctx->ps) return pe_ps_coarsen(ctx->samples, ctx->K_cur + 1, ctx->ncoef, ctx->s_w, ctx->csamples, ctx->stream);
    if (ctx->pres)  // Section 3.2: n, nV and the second moment, each to its scaling coefficients
        return pe_coarsen_pressure(ctx->samples, ctx->K_cur + 1, c.ncell, ctx->s_w, ctx->s_p, ctx->s_e, c.wavelet,
                                   ctx->nc, ctx->bin_shift, ctx->csamples, ctx->stream);
    return pe_coarsen(ctx->samples, ctx->K_cur + 1, c.ncell, ctx->s_w, ctx->s_p, c.wavelet, ctx->nc, ctx->bin_shift,
                      ctx->csamples, ctx->stream);
}

extern "C" PE_API int pe_project(pe_ctx* ctx)
{
    NvtxRange nvtx("pe_project");
    if (!ctx) return PE_EINVAL;
    const pe_config& c = ctx->cfg;
    if (ctx->ps && c.ps_filter) {
        double* work = ctx->csamples + (size_t)(c.K + 1) * (size_t)ctx->crow;  // measurement row as scratch
        const int filt = c.ps_filter | ((ctx->walls && (c.ps_filter & 2)) ? 4 : 0);  // reflecting x at walls
        PE_TRY(pe_ps_project(ctx->csamples, ctx->K_cur, ctx->nc, ctx->nv, c.dt, ctx->dT_cur, filt, work, ctx->coarse,
                             ctx->slope,
                             ctx->stream));
    } else {
        PE_TRY(pe_ls_project(ctx->csamples, ctx->K_cur, (int32_t)ctx->ncoef, c.dt, ctx->dT_cur, ctx->coarse, ctx->slope,
                             ctx->stream));
    }
    if (ctx->te_active)  // the electrons' energy: the same least-squares leap, into we[K+2] (slope we[K+3])
        PE_TRY(pe_ls_project(ctx->we, ctx->K_cur, 1, c.dt, ctx->dT_cur, ctx->we + (c.K + 2), ctx->we + (c.K + 3),
                             ctx->stream));
    ctx->macro_steps += 1;
    ctx->coarse_state = 1;
    ctx->time += ctx->dT_cur;
    ctx->fresh = 0;
    return PE_OK;
}

extern "C" PE_API int pe_lift(pe_ctx* ctx)
{
    NvtxRange nvtx("pe_lift");
    if (!ctx) return PE_EINVAL;
    pe_ctx* x = ctx;
    const pe_config& c = x->cfg;
    if (x->psw) {
        // Section 3.3 lifting: synthesis in v, Appendix C's reconstruction per coarse node,
        // Eq. (interpolation) to the fine nodes, quiet start on the fine-node tables
        PE_TRY(pe_ps_refine_v(x->coarse, x->nc, x->nvc, c.wavelet, x->nv, x->ps_hist, x->stream));
        PE_TRY(pe_ps_lift_tables(x->ps_hist, x->nc, x->nv, x->ps_mass, x->ps_cdf, x->ps_table, x->ps_scratch,
                                 x->ps_flags, x->stream));
        PE_TRY(pe_ps_node_tables(x->ps_mass, x->ps_cdf, x->nc, c.ncell, x->nv, x->ps_node_table, x->ps_node_dens,
                                 x->stream));
        const int b = x->bank;
        PE_TRY(timed(x, PE_PROF_LOAD, [&] {
            return pe_ps_quiet_start_nodes(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, c.ncell,
                                           x->ps_node_table, x->ps_node_dens, x->nv, x->vmin, x->dv, lift_seed(x),
                                           x->s_w, x->rho, x->status, x->stream);
        }));
        x->rho_valid = 1;
        x->v_at_integer = 1;
        x->fresh = 1;
        x->phi_hist = 0;
    } else if (x->ps) {
        // Appendix C: per-bin CDF reconstruction, then quiet start on the tables
        PE_TRY(pe_ps_lift_tables(x->coarse, x->nc, x->nv, x->ps_mass, x->ps_cdf, x->ps_table, x->ps_scratch, x->ps_flags,
                                 x->stream));
        const int b = x->bank;
        PE_TRY(timed(x, PE_PROF_LOAD, [&] {
            if (x->walls)
                return pe_ps_quiet_start_equal(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, c.ncell,
                                               x->bin_shift, x->ps_mass, x->ps_table, x->nv, x->vmin, x->dv,
                                               lift_seed(x), x->s_w, x->eq_scratch, x->rho, x->status, x->stream);
            return pe_ps_quiet_start(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, c.ncell, x->bin_shift,
                                     x->ps_mass, x->ps_table, x->nv, x->vmin, x->dv, lift_seed(x), x->s_w, x->rho,
                                     x->status, x->stream);
        }));
        x->rho_valid = 1;
        x->v_at_integer = 1;
        x->fresh = 1;
        x->phi_hist = 0;
    } else if (x->pres) {
        // Section 3.2 lifting with the pressure active: n, u and T = P / n on the nodes, then
        // Maxwellians of the local temperature (periodic grids)
        PE_TRY(pe_refine_pressure(x->coarse, x->nc, c.wavelet, c.ncell, x->prof, x->prof + c.ncell,
                                  x->prof + 2 * (size_t)c.ncell, x->stream));
        const int b = x->bank;
        PE_TRY(timed(x, PE_PROF_LOAD, [&] {
            return pe_quiet_start_thermal(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, c.ncell, x->prof,
                                          x->prof + c.ncell, x->prof + 2 * (size_t)c.ncell, lift_seed(x), x->s_w,
                                          x->rho, x->status, x->stream);
        }));
        x->rho_valid = 1;
        x->v_at_integer = 1;
        x->fresh = 1;
        x->phi_hist = 0;
    } else {
        PE_TRY(pe_refine(x->coarse, x->nc, c.wavelet, c.ncell, x->prof, x->prof + c.ncell, x->stream));
        PE_TRY(quiet_start_from_profile(x, lift_seed(x), 2.0f));  // refined restriction: wall nodes hold deposits
    }
    if (x->kinetic) {
        if (x->te_active) {  // T_e / T_e0 = projected energy / energy at the initial load
            double w = 0.0;
            if (cudaMemcpyAsync(&w, x->we + (c.K + 2), sizeof(w), cudaMemcpyDeviceToHost, x->stream) != cudaSuccess ||
                cudaStreamSynchronize(x->stream) != cudaSuccess)
                return PE_ECUDA;
            x->we_last = w;
            const double t = (x->we_ref > 0.0) ? w / x->we_ref : 1.0;
            x->te = (t > 1e-3 && t < 1e3) ? t : (t >= 1e3 ? 1e3 : 1e-3);  // NaN and negatives clamp low
        }
        PE_TRY(load_boltzmann_electrons(x, electron_seed(lift_seed(x)), x->ps ? kDriftPhaseSpace : kDriftProfile,
                                        x->te));
    }
    return PE_OK;
}

extern "C" PE_API int pe_step(pe_ctx* ctx)
{
    NvtxRange nvtx("pe_step");
    if (!ctx) return PE_EINVAL;
    if (!ctx->fresh) PE_TRY(pe_lift(ctx));
    PE_TRY(pe_burst(ctx));
    PE_TRY(pe_restrict(ctx));
    return pe_project(ctx);
}

extern "C" PE_API int pe_set_macro_step(pe_ctx* ctx, double dT)
{
    if (!ctx || !(dT >= ctx->K_cur * ctx->cfg.dt * (1.0 - 1e-12)) || !(dT < 1e300)) return PE_EINVAL;
    ctx->dT_cur = dT;
    return PE_OK;
}

// Leap length L >= 0 with ||q|| L (L + K dt) = tol ||c_K||; infinite when the trajectory has
// no curvature.
static double leap_for_tol(double qn, double cn, double Kdt, double tol)
{
    if (!(qn > 0.0)) return INFINITY;
    const double r = tol * cn / qn;
    return 0.5 * (-Kdt + sqrt(Kdt * Kdt + 4.0 * r));
}

// Smallest burst length K' in [K_min, K_max] whose least-squares slope noise, scaled from the
// measured sn at K by var ~ 1 / (K (K+1) (K+2)), moves a leap of length L by at most
// tol_noise relative to cn; K_max when none does.
static int burst_length_for_noise(double sn, int K, double L, double cn, double tol_noise, int K_min, int K_max)
{
    if (!(L > 0.0) || !(sn > 0.0) || !(cn > 0.0)) return K_min;
    const double base = (double)K * (K + 1) * (K + 2);
    for (int Kp = K_min; Kp <= K_max; ++Kp)
        if (L * sn * sqrt(base / ((double)Kp * (Kp + 1) * (Kp + 2))) <= tol_noise * cn) return Kp;
    return K_max;
}

extern "C" PE_API int pe_step_adaptive(pe_ctx* ctx, const pe_adapt_cfg* a, pe_adapt_stats* out)
{
    NvtxRange nvtx("pe_step_adaptive");
    if (!ctx || !a || !(a->tol > 0.0) || a->M_min < 1 || a->M_max < a->M_min || !(a->safety > 0.0) ||
        !(a->safety <= 1.0) || !(a->grow >= 1.0))
        return PE_EINVAL;
    pe_ctx* x = ctx;
    const pe_config& c = x->cfg;
    const bool adapt_K = a->K_max > 0;
    if (adapt_K && (a->K_min < 3 || a->K_max < a->K_min || a->K_max > c.K || !(a->noise_frac >= 0.0) ||
                    !(a->noise_frac <= 1.0)))
        return PE_EINVAL;
    if (x->K_cur < 2) return PE_EINVAL;
    if (adapt_K) x->K_cur = std::min(a->K_max, std::max(a->K_min, x->K_cur));
    const double noise_frac = a->noise_frac > 0.0 ? a->noise_frac : 0.5;
    const int K = x->K_cur;
    const double Kdt = K * c.dt;
    auto bursts = [&](double dT) { return std::max(1, (int)floor(dT / Kdt + 1e-9)); };
    int M = std::min(a->M_max, std::max(a->M_min, bursts(x->dT_cur)));
    // the moments scratch (64 KB) is free here: partial sums, then the four results
    double* part = (double*)(x->arena + x->lay.offset[PE_BUF_DIAG]);
    double* qc = part + 4 * 1024;
    const int64_t f0 = x->fine_steps;
    int rejected = 0;
    double err = 0.0, L_tol = 0.0, h[4] = {0.0, 0.0, 0.0, 0.0};
    for (;;) {
        x->dT_cur = M * Kdt;
        if (!x->fresh) PE_TRY(pe_lift(x));
        PE_TRY(pe_burst(x));
        PE_TRY(pe_restrict(x));
        PE_TRY(pe_leap_curvature(x->csamples, K, (int32_t)x->ncoef, c.dt, part, qc, x->stream));
        if (cudaMemcpyAsync(h, qc, sizeof(h), cudaMemcpyDeviceToHost, x->stream) != cudaSuccess) return PE_ECUDA;
        if (cudaStreamSynchronize(x->stream) != cudaSuccess) return PE_ECUDA;
        const double L = x->dT_cur - Kdt;
        err = h[1] > 0.0 ? h[0] * L * (L + Kdt) / h[1] : 0.0;
        L_tol = leap_for_tol(h[0], h[1], Kdt, a->tol);
        if (err > a->tol && M > a->M_min) {  // rejected: rerun from the same coarse state
            const int Mt = bursts(Kdt + a->safety * L_tol);
            M = std::max(a->M_min, std::min(M - 1, Mt));
            rejected += 1;
            continue;  // the burst consumed the lifted particles: pe_lift runs again
        }
        break;
    }
    const double taken = x->dT_cur;
    const double L_taken = taken - Kdt;
    PE_TRY(pe_project(x));
    int K_next = K;
    if (adapt_K) K_next = burst_length_for_noise(h[3], K, L_taken, h[1], noise_frac * a->tol, a->K_min, a->K_max);
    // the next macro step in whole bursts of the next burst length: the leap allowed by the
    // curvature (L_tol, measured with bursts of K), capped by growth of the current Delta t
    const double Kdt_n = K_next * c.dt;
    const double Mn = isinf(L_tol) ? (double)a->M_max : floor((Kdt_n + a->safety * L_tol) / Kdt_n + 1e-9);
    const double cap = std::min((double)a->M_max, floor(a->grow * taken / Kdt_n + 1e-9));
    const int M_next = (int)std::max((double)a->M_min, std::min(cap, Mn));
    x->K_cur = K_next;
    x->dT_cur = M_next * Kdt_n;
    if (out) {
        out->dT = taken;
        out->err = err;
        out->dT_next = x->dT_cur;
        out->rejected = rejected;
        out->fine_steps = (int32_t)(x->fine_steps - f0);
        out->noise = h[1] > 0.0 ? L_taken * h[3] / h[1] : 0.0;
        out->K = K;
        out->K_next = K_next;
    }
    return PE_OK;
}

extern "C" PE_API int pe_pic_steps(pe_ctx* ctx, int32_t nsteps)
{
    NvtxRange nvtx("pe_pic_steps");
    if (!ctx || nsteps < 0) return PE_EINVAL;
    pe_ctx* x = ctx;
    const pe_config& c = x->cfg;
    const float dt_dx = (float)(c.dt / x->dx), qm_dt = (float)(c.qm * c.dt);
    if (nsteps > 0) x->coarse_state = 0;  // the particles move on alone
    for (int s = 0; s < nsteps; ++s) {
        if (c.sort_every > 0 && (x->fine_steps % c.sort_every) == 0 && !x->fresh) {
            const int b = x->bank, o = 1 - b;
            PE_TRY(pe_sort(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, c.ncell, x->cell[o], x->theta[o],
                           x->v[o], x->w[o], x->sort, x->status, x->stream));
            x->bank = o;
            if (x->kinetic) {
                const int e = x->ebank, eo = 1 - e;
                PE_TRY(pe_sort(x->ecell[e], x->etheta[e], x->ev[e], x->ew[e], c.nparticles, c.ncell, x->ecell[eo],
                               x->etheta[eo], x->ev[eo], x->ew[eo], x->sort, x->status, x->stream));
                x->ebank = eo;
            }
        }
        if (!x->rho_valid) PE_TRY(deposit_current(x));
        if (x->kinetic && c.reset_every > 0 && (x->fine_steps % c.reset_every) == 0 && !x->fresh)
            PE_TRY(load_boltzmann_electrons(x, electron_seed(c.seed + 0x9E3779B97F4A7C15ULL * (uint64_t)x->fine_steps),
                                            kDriftParticles));
        PE_TRY(field_solve(x, 1));
        const int b = x->bank;
        const float kick = x->v_at_integer ? 0.5f : 1.0f;
        PE_TRY(timed(x, PE_PROF_PUSH, [&] {
            return pe_push_ex(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, x->Ef, c.ncell, dt_dx, qm_dt,
                              kick, x->s_w, c.boundary, x->rho, nullptr, x->status, x->stream);
        }));
        if (x->kinetic) PE_TRY(push_electrons(x));
        x->v_at_integer = 0;
        x->rho_valid = 1;
        x->fresh = 0;
        x->fine_steps += 1;
        x->time += c.dt;
    }
    return PE_OK;
}

extern "C" PE_API int pe_get_slope(pe_ctx* ctx, double* out, int32_t out_on_device)
{
    if (!ctx || !out) return PE_EINVAL;
    const size_t bytes = sizeof(double) * (size_t)ctx->ncoef;
    if (cudaMemcpyAsync(out, ctx->slope, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        ctx->stream) != cudaSuccess)
        return PE_ECUDA;
    if (!out_on_device && cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PE_ECUDA;
    return PE_OK;
}

extern "C" PE_API int pe_get_coarse(pe_ctx* ctx, double* out, int32_t out_on_device)
{
    if (!ctx || !out) return PE_EINVAL;
    const size_t bytes = sizeof(double) * (size_t)ctx->ncoef;
    if (cudaMemcpyAsync(out, ctx->coarse, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        ctx->stream) != cudaSuccess)
        return PE_ECUDA;
    if (!out_on_device && cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PE_ECUDA;
    return PE_OK;
}

extern "C" PE_API int pe_set_coarse(pe_ctx* ctx, const double* in, int32_t in_on_device)
{
    if (!ctx || !in) return PE_EINVAL;
    const size_t bytes = sizeof(double) * (size_t)ctx->ncoef;
    if (cudaMemcpyAsync(ctx->coarse, in, bytes, in_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess)
        return PE_ECUDA;
    if (!in_on_device && cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PE_ECUDA;
    ctx->fresh = 0;  // the next step lifts from this state
    ctx->coarse_state = 1;
    return PE_OK;
}

// Checkpoint image: header, coarse[ncoef], slope[ncoef], phi[2 ncell] (phi and its history).
struct CheckpointHeader {
    uint32_t magic, version;
    int32_t ncell, phi_hist;
    int64_t ncoef, macro_steps, fine_steps;
    double time, dT_cur;
    pe_config cfg;  // a restore needs the same configuration, byte for byte
    int32_t K_cur, pad;  // burst length of the next bursts
    double te, we_ref, we_proj;  // electrons' temperature state (te_active)
};
constexpr uint32_t kCheckpointMagic = 0x50455043u;  // "PEPC"

extern "C" PE_API int pe_checkpoint_bytes(const pe_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return PE_EINVAL;
    *bytes = sizeof(CheckpointHeader) + sizeof(double) * (2 * (size_t)ctx->ncoef + 2 * (size_t)ctx->cfg.ncell);
    return PE_OK;
}

extern "C" PE_API int pe_checkpoint_save(pe_ctx* ctx, void* host_buf, size_t bytes)
{
    NvtxRange nvtx("pe_checkpoint_save");
    size_t need = 0;
    PE_TRY(pe_checkpoint_bytes(ctx, &need));
    if (!host_buf || bytes < need) return PE_EINVAL;
    pe_ctx* x = ctx;
    if (!x->coarse_state || x->macro_steps < 1) return PE_ESTATE;  // the particles are the state
    CheckpointHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kCheckpointMagic;
    h.version = 2u;
    h.ncell = x->cfg.ncell;
    h.phi_hist = x->phi_hist;
    h.ncoef = x->ncoef;
    h.macro_steps = x->macro_steps;
    h.fine_steps = x->fine_steps;
    h.time = x->time;
    h.dT_cur = x->dT_cur;
    h.cfg = x->cfg;
    h.K_cur = x->K_cur;
    h.te = x->te;
    h.we_ref = x->we_ref;
    if (x->te_active) {
        if (cudaMemcpyAsync(&h.we_proj, x->we + (x->cfg.K + 2), sizeof(double), cudaMemcpyDeviceToHost, x->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(x->stream) != cudaSuccess)
            return PE_ECUDA;
    }
    char* p = (char*)host_buf;
    memcpy(p, &h, sizeof(h));
    double* d = (double*)(p + sizeof(h));
    const size_t nco = (size_t)x->ncoef, nphi = 2 * (size_t)x->cfg.ncell;
    if (cudaMemcpyAsync(d, x->coarse, sizeof(double) * nco, cudaMemcpyDeviceToHost, x->stream) != cudaSuccess ||
        cudaMemcpyAsync(d + nco, x->slope, sizeof(double) * nco, cudaMemcpyDeviceToHost, x->stream) != cudaSuccess ||
        cudaMemcpyAsync(d + 2 * nco, x->phi, sizeof(double) * nphi, cudaMemcpyDeviceToHost, x->stream) != cudaSuccess)
        return PE_ECUDA;
    return cudaStreamSynchronize(x->stream) == cudaSuccess ? PE_OK : PE_ECUDA;
}

extern "C" PE_API int pe_checkpoint_restore(pe_ctx* ctx, const void* host_buf, size_t bytes)
{
    NvtxRange nvtx("pe_checkpoint_restore");
    size_t need = 0;
    PE_TRY(pe_checkpoint_bytes(ctx, &need));
    if (!host_buf || bytes < need) return PE_EINVAL;
    pe_ctx* x = ctx;
    CheckpointHeader h;
    memcpy(&h, host_buf, sizeof(h));
    if (h.magic != kCheckpointMagic || h.version != 2u || h.ncell != x->cfg.ncell || h.ncoef != x->ncoef ||
        h.macro_steps < 1 || h.K_cur < 1 || h.K_cur > x->cfg.K || !(h.dT_cur >= h.K_cur * x->cfg.dt * (1.0 - 1e-12)) ||
        !(h.dT_cur < 1e300) || memcmp(&h.cfg, &x->cfg, sizeof(pe_config)) != 0)
        return PE_EINVAL;
    // the clock and the Newton history drive the lifting seed, the sort and reset cadence and
    // the first solve: a header that passes the checks above but carries an impossible clock
    // (a negative step count, a non-finite or negative time, a history flag other than 0/1)
    // is refused rather than loaded
    if (h.fine_steps < 0 || !(h.time >= 0.0 && h.time < 1e300) || (h.phi_hist != 0 && h.phi_hist != 1))
        return PE_EINVAL;
    const double* d = (const double*)((const char*)host_buf + sizeof(h));
    const size_t nco = (size_t)x->ncoef, nphi = 2 * (size_t)x->cfg.ncell;
    if (cudaMemcpyAsync(x->coarse, d, sizeof(double) * nco, cudaMemcpyHostToDevice, x->stream) != cudaSuccess ||
        cudaMemcpyAsync(x->slope, d + nco, sizeof(double) * nco, cudaMemcpyHostToDevice, x->stream) != cudaSuccess ||
        cudaMemcpyAsync(x->phi, d + 2 * nco, sizeof(double) * nphi, cudaMemcpyHostToDevice, x->stream) != cudaSuccess)
        return PE_ECUDA;
    if (cudaStreamSynchronize(x->stream) != cudaSuccess) return PE_ECUDA;
    x->macro_steps = h.macro_steps;
    x->fine_steps = h.fine_steps;
    x->time = h.time;
    x->dT_cur = h.dT_cur;
    x->K_cur = h.K_cur;
    x->te = h.te;
    x->we_ref = h.we_ref;
    if (x->te_active) {
        x->we_last = h.we_proj;
        if (cudaMemcpyAsync(x->we + (x->cfg.K + 2), &h.we_proj, sizeof(double), cudaMemcpyHostToDevice, x->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(x->stream) != cudaSuccess)
            return PE_ECUDA;
    }
    x->phi_hist = h.phi_hist;
    x->fresh = 0;  // the next step lifts from the restored coarse state
    x->coarse_state = 1;
    x->rho_valid = 0;
    return PE_OK;
}

extern "C" PE_API int pe_sync_status(pe_ctx* ctx)
{
    if (!ctx) return PE_EINVAL;
    uint32_t st = 0;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PE_ECUDA;
    if (cudaMemcpy(&st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return PE_ECUDA;
    if (cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t), ctx->stream) != cudaSuccess) return PE_ECUDA;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PE_ECUDA;
    if (st & PE_FLAG_TIMEOUT) return PE_ETIMEOUT;
    if (st & PE_FLAG_RANGE) return PE_ERANGE;
    if (st & PE_FLAG_OVERFLOW) return PE_EOVERFLOW;
    if (st & PE_FLAG_NOCONV) return PE_ENOCONV;
    return PE_OK;
}

extern "C" PE_API int pe_state_moments(pe_ctx* ctx, pe_moments* out, int32_t out_on_device)
{
    NvtxRange nvtx("pe_state_moments");
    if (!ctx || !out) return PE_EINVAL;
    pe_ctx* x = ctx;
    const pe_config& c = x->cfg;
    if (!x->rho_valid) PE_TRY(deposit_current(x));
    PE_TRY(field_solve(x));
    char* scratch = x->arena + x->lay.offset[PE_BUF_DIAG];
    pe_moments* res = (pe_moments*)(scratch + PE_MOMENTS_SCRATCH_BYTES);
    const int b = x->bank;
    const float kick = x->v_at_integer ? 0.5f : 1.0f;
    // kinetic electrons: no Boltzmann free energy (phi not passed); the electron particles'
    // moments are folded in below
    PE_TRY(pe_compute_moments(x->cell[b], x->theta[b], x->v[b], x->w[b], c.nparticles, x->Ef,
                              x->kinetic ? nullptr : x->phi, x->E, c.ncell, x->dx, c.dt, (float)(c.qm * c.dt), kick,
                              x->s_w, c.poisson, scratch, res, x->status, x->stream));
    if (x->kinetic) {
        pe_moments* eres = (pe_moments*)(scratch + PE_MOMENTS_SCRATCH_BYTES + 128);
        const int e = x->ebank;
        const float ekick = x->e_v_at_integer ? 0.5f : 1.0f;
        PE_TRY(pe_compute_moments(x->ecell[e], x->etheta[e], x->ev[e], x->ew[e], c.nparticles, x->Ef, nullptr, nullptr,
                                  c.ncell, x->dx, c.dt, (float)(x->qm_e * c.dt), ekick, x->s_w, c.poisson, scratch,
                                  eres, x->status, x->stream));
        PE_TRY(combine_kinetic_moments(res, eres, x->qm_e, x->stream));
    }
    if (cudaMemcpyAsync(out, res, sizeof(pe_moments), out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        x->stream) != cudaSuccess)
        return PE_ECUDA;
    if (!out_on_device && cudaStreamSynchronize(x->stream) != cudaSuccess) return PE_ECUDA;
    return PE_OK;
}

extern "C" PE_API int pe_diagnostics(pe_ctx* ctx, pe_diag* out)
{
    if (!ctx || !out) return PE_EINVAL;
    memset(out, 0, sizeof(*out));
    out->macro_steps = ctx->macro_steps;
    out->fine_steps = ctx->fine_steps;
    out->time = ctx->time;
    out->particle_bank = ctx->bank;
    out->v_at_integer = ctx->v_at_integer;
    out->s_w = ctx->s_w;
    out->s_p = ctx->s_p;
    out->electron_bank = ctx->ebank;
    out->e_v_at_integer = ctx->e_v_at_integer;
    out->T_e = ctx->te;
    out->W_e = ctx->we_last;
    int32_t d[2] = {0, 0};
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PE_ECUDA;
    if (cudaMemcpy(d, ctx->diag, sizeof(d), cudaMemcpyDeviceToHost) != cudaSuccess) return PE_ECUDA;
    if (cudaMemcpy(&out->status, ctx->status, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return PE_ECUDA;
    out->newton_iters = d[0];
    return PE_OK;
}
