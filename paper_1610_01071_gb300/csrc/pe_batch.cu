// Batched ensemble of realisations: many independent contexts (different grids and
// particle counts, the same burst length) advanced together. Each fine step of all
// realisations is one persistent particle launch over a shared work list plus one
// launch of field-solve clusters (one cluster per realisation); the whole burst,
// restriction and projection are captured once as a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "pe_ctx.h"
#include "pe_internal.h"
#include "pepic.h"

using namespace pe;

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t push, field, proj, items, counter, rho, e0, samp, total;
    int64_t rho_total, samp_row, max_items;
};

// The smallest chunk the tuner may choose bounds the work-list length.
constexpr int64_t kMinChunk = 4096;
const int64_t kChunkCandidates[] = {8192, 16384, 32768, 65536};

int layout_for(pe_ctx* const* ctxs, int n, Layout* L)
{
    if (!ctxs || n < 1) return PE_EINVAL;
    const int K = ctxs[0]->cfg.K;
    int64_t rho = 0, row = 0, items = 0;
    for (int r = 0; r < n; ++r) {
        const pe_ctx* x = ctxs[r];
        if (!x || x->cfg.K != K || x->cfg.wavelet != PE_WAVELET_HAAR || x->cfg.ncell < 64 || x->ps || x->kinetic)
            return PE_EINVAL;
        rho += x->cfg.ncell;
        row += 2 * (int64_t)x->nb;
        items += (x->cfg.nparticles + kMinChunk - 1) / kMinChunk;
    }
    L->rho_total = rho;
    L->samp_row = row;
    L->max_items = items;
    size_t off = 0;
    L->push = off;
    off += a256(push_desc_size() * n);
    L->field = off;
    off += a256(field_desc_size() * n);
    L->proj = off;
    off += a256(proj_desc_size() * n);
    L->items = off;
    off += a256(work_item_size() * (size_t)items);
    L->counter = off;
    off += 256;
    L->rho = off;
    off += a256(8 * (size_t)rho);
    L->e0 = off;
    off += a256(4 * (size_t)rho);
    L->samp = off;
    off += a256(8 * (size_t)row * (size_t)(K + 2));  // rows 0..K, row K+1 is tuning scratch
    L->total = off;
    return PE_OK;
}

}  // namespace

struct pe_batch {
    std::vector<pe_ctx*> ctx;
    Layout L;
    char* scratch;
    cudaStream_t stream;
    int K;
    int64_t chunk;
    int nitems;
    int max_ncell, max_nb;
    // Field-solve groups, one launch each: (multi-block clusters of size G | single blocks) x
    // (FP32 | FP64 Jacobian solve: bounded grids). Every realisation is solved exactly as its
    // context alone would solve it.
    std::vector<int> field_ids[4];
    int field_maxn[4];
    int G;  // cluster size of the multi-block groups
    std::vector<int64_t> rho_off, e0_off, samp_off;
    std::vector<int> banks;  // particle bank of each context when the descriptors were built
    cudaGraphExec_t graph;
    long long graph_kernels;
    int steps_done;
    cudaEvent_t ev_in, ev_out;  // ordering against the contexts' streams
};

static char* at(pe_batch* b, size_t off) { return b->scratch + off; }

// Work list: particles of every realisation in chunks of at most b->chunk (multiples of 4).
static int build_items(pe_batch* b)
{
    std::vector<char> host(work_item_size() * (size_t)b->L.max_items);
    int n = 0;
    for (int r = 0; r < (int)b->ctx.size(); ++r) {
        const int64_t N = b->ctx[r]->cfg.nparticles;
        for (int64_t s = 0; s < N; s += b->chunk) {
            if (n >= b->L.max_items) return PE_EINVAL;
            make_work_item(host.data() + work_item_size() * n, r, s, s + b->chunk < N ? s + b->chunk : N);
            ++n;
        }
    }
    b->nitems = n;
    if (cudaMemcpy(at(b, b->L.items), host.data(), work_item_size() * n, cudaMemcpyHostToDevice) != cudaSuccess)
        return PE_ECUDA;
    return PE_OK;
}

static int build_descs(pe_batch* b)
{
    const int R = (int)b->ctx.size();
    std::vector<char> push(push_desc_size() * R), proj(proj_desc_size() * R);
    std::vector<char> fd(field_desc_size() * R);
    std::vector<int> slot(R, 0);  // position of each realisation's field descriptor
    {
        int o = 0;
        for (int g = 0; g < 4; ++g)
            for (int r : b->field_ids[g]) slot[r] = o++;
    }
    int64_t* rho_all = reinterpret_cast<int64_t*>(at(b, b->L.rho));
    float* e0_all = reinterpret_cast<float*>(at(b, b->L.e0));
    int64_t* samp_all = reinterpret_cast<int64_t*>(at(b, b->L.samp));
    b->banks.assign(R, 0);
    for (int r = 0; r < R; ++r) {
        pe_ctx* x = b->ctx[r];
        const pe_config& c = x->cfg;
        const int k = x->bank;
        b->banks[r] = k;
        make_push_desc(push.data() + push_desc_size() * r, x->cell[k], x->theta[k], x->v[k], x->w[k], c.nparticles,
                       x->Ef, c.ncell, (float)(c.dt / x->dx), (float)(c.qm * c.dt), x->s_w, rho_all + b->rho_off[r],
                       e0_all + b->e0_off[r], c.dT, c.dt, (float)(1.0 / x->dx), (float)c.qm, c.comoving,
                       x->s_p, x->bin_shift, samp_all + b->samp_off[r], b->L.samp_row, x->walls, x->status);
        make_proj_desc(proj.data() + proj_desc_size() * r, samp_all + b->samp_off[r], b->L.samp_row, c.ncell, x->nc,
                       x->s_w, x->s_p, x->csamples, x->coarse, x->slope);
        char* dst = fd.data() + field_desc_size() * slot[r];
        make_field_desc(dst, rho_all + b->rho_off[r], c.ncell, x->dx, x->s_w, c.poisson, x->walls, c.newton_tol,
                        c.newton_maxit, x->phi, x->E, x->Ef, x->diag, x->status, x->phi + c.ncell);
    }
    if (cudaMemcpy(at(b, b->L.push), push.data(), push.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(at(b, b->L.proj), proj.data(), proj.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(at(b, b->L.field), fd.data(), fd.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return PE_ECUDA;
    return PE_OK;
}

// extrap: the Newton starts extrapolate the last two solutions (the solves after a push), as
// the context path's burst does.
static int field_all(pe_batch* b, bool extrap)
{
    const char* base = at(b, b->L.field);
    size_t o = 0;
    for (int g = 0; g < 4; ++g) {
        const int n = (int)b->field_ids[g].size();
        if (n)
            PE_TRY(launch_newton_batch(base + field_desc_size() * o, n, g < 2 ? b->G : 1, b->field_maxn[g], g & 1,
                                       extrap, b->stream));
        o += (size_t)n;
    }
    return PE_OK;
}

// Burst of every realisation (after lifting) + restriction + projection: the graph body.
static int burst_restrict_project(pe_batch* b)
{
    cudaStream_t s = b->stream;
    const int R = (int)b->ctx.size();
    int64_t* rho_all = reinterpret_cast<int64_t*>(at(b, b->L.rho));
    int64_t* samp_all = reinterpret_cast<int64_t*>(at(b, b->L.samp));
    float* e0_all = reinterpret_cast<float*>(at(b, b->L.e0));
    unsigned* counter = reinterpret_cast<unsigned*>(at(b, b->L.counter));
    PE_TRY(field_all(b, false));  // field at burst start (charge deposited by the lifting)
    for (int r = 0; r < R; ++r)
        if (cudaMemcpyAsync(e0_all + b->e0_off[r], b->ctx[r]->Ef, 4 * (size_t)b->ctx[r]->cfg.ncell,
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return PE_ECUDA;
    const size_t row_bytes = 8 * (size_t)b->L.samp_row;
    for (int p = 0; p <= b->K; ++p) {
        if (cudaMemsetAsync(samp_all + (size_t)p * b->L.samp_row, 0, row_bytes, s) != cudaSuccess) return PE_ECUDA;
        if (p == b->K) {
            PE_TRY(launch_particles_batch(1, at(b, b->L.push), at(b, b->L.items), b->nitems, p, 1.0f, counter,
                                          b->max_ncell, b->max_nb, s));
            break;
        }
        if (cudaMemsetAsync(rho_all, 0, 8 * (size_t)b->L.rho_total, s) != cudaSuccess) return PE_ECUDA;
        PE_TRY(launch_particles_batch(0, at(b, b->L.push), at(b, b->L.items), b->nitems, p, p == 0 ? 0.5f : 1.0f,
                                      counter, b->max_ncell, b->max_nb, s));
        PE_TRY(field_all(b, true));
    }
    const pe_config& c0 = b->ctx[0]->cfg;
    return launch_restrict_project_batch(at(b, b->L.proj), R, b->K, c0.dt, c0.dT, s);
}

extern "C" PE_API int pe_batch_scratch_bytes(pe_ctx* const* ctxs, int32_t n, size_t* bytes)
{
    if (!bytes) return PE_EINVAL;
    Layout L;
    PE_TRY(layout_for(ctxs, n, &L));
    *bytes = L.total;
    return PE_OK;
}

extern "C" PE_API int pe_batch_create(pe_ctx* const* ctxs, int32_t n, void* scratch, size_t scratch_bytes,
                                      void* stream, pe_batch** out)
{
    if (!out) return PE_EINVAL;
    *out = nullptr;
    Layout L;
    PE_TRY(layout_for(ctxs, n, &L));
    if (!scratch || ((uintptr_t)scratch & 255u) || scratch_bytes < L.total) return PE_EINVAL;
    for (int r = 0; r < n; ++r)
        if (ctxs[r]->cfg.dt != ctxs[0]->cfg.dt || ctxs[r]->cfg.dT != ctxs[0]->cfg.dT) return PE_EINVAL;
    pe_batch* b = new pe_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->L = L;
    b->scratch = static_cast<char*>(scratch);
    b->stream = (cudaStream_t)stream;
    b->K = ctxs[0]->cfg.K;
    b->chunk = 65536;
    b->graph = nullptr;
    b->graph_kernels = 0;
    b->steps_done = 0;
    if (cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        delete b;
        return PE_ECUDA;
    }
    b->G = 1;
    for (int r = 0; r < n; ++r) b->G = newton_cluster_size(ctxs[r]->cfg.ncell) > b->G ? newton_cluster_size(ctxs[r]->cfg.ncell) : b->G;
    b->max_ncell = 0;
    for (int g = 0; g < 4; ++g) b->field_maxn[g] = 0;
    b->max_nb = 0;
    int64_t ro = 0, so = 0;
    for (int r = 0; r < n; ++r) {
        const pe_ctx* x = ctxs[r];
        b->rho_off.push_back(ro);
        b->e0_off.push_back(ro);
        b->samp_off.push_back(so);
        ro += x->cfg.ncell;
        so += 2 * (int64_t)x->nb;
        if (x->nb > b->max_nb) b->max_nb = x->nb;
        if (x->cfg.ncell > b->max_ncell) b->max_ncell = x->cfg.ncell;
        const bool cl = b->G > 1 && newton_cluster_size(x->cfg.ncell) == b->G;
        const int g = (cl ? 0 : 2) + (x->walls ? 1 : 0);
        b->field_ids[g].push_back(r);
        if (x->cfg.ncell > b->field_maxn[g]) b->field_maxn[g] = x->cfg.ncell;
    }
    int rc = build_descs(b);
    if (rc == PE_OK) rc = build_items(b);
    if (rc == PE_OK && cudaMemset(at(b, L.e0), 0, 4 * (size_t)L.rho_total) != cudaSuccess) rc = PE_ECUDA;
    if (rc != PE_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return PE_OK;
}

extern "C" PE_API void pe_batch_destroy(pe_batch* b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaEventDestroy(b->ev_in);
    cudaEventDestroy(b->ev_out);
    delete b;
}

static void drop_graph(pe_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

extern "C" PE_API int pe_batch_tune(pe_batch* b, int64_t* chosen_chunk)
{
    if (!b) return PE_EINVAL;
    unsigned* counter = reinterpret_cast<unsigned*>(at(b, b->L.counter));
    const int maxn = b->max_ncell;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PE_ECUDA;
    float best = 1e30f;
    int64_t best_chunk = b->chunk;
    for (int64_t cand : kChunkCandidates) {
        b->chunk = cand;
        PE_TRY(build_items(b));
        // the read-only sample pass, written to the scratch row K+1, times the particle stream
        PE_TRY(launch_particles_batch(1, at(b, b->L.push), at(b, b->L.items), b->nitems, b->K + 1, 1.0f, counter,
                                      maxn, b->max_nb, b->stream));
        cudaEventRecord(e0, b->stream);
        for (int rep = 0; rep < 3; ++rep)
            PE_TRY(launch_particles_batch(1, at(b, b->L.push), at(b, b->L.items), b->nitems, b->K + 1, 1.0f, counter,
                                          maxn, b->max_nb, b->stream));
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return PE_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_chunk = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chunk = best_chunk;
    PE_TRY(build_items(b));
    drop_graph(b);
    if (chosen_chunk) *chosen_chunk = best_chunk;
    return PE_OK;
}

extern "C" PE_API int pe_batch_step(pe_batch* b)
{
    NvtxRange nvtx("pe_batch_step");
    if (!b) return PE_EINVAL;
    const int R = (int)b->ctx.size();
    const bool fresh = b->ctx[0]->fresh != 0;
    for (int r = 0; r < R; ++r) {
        pe_ctx* x = b->ctx[r];
        if ((x->fresh != 0) != fresh) return PE_ESTATE;  // all realisations must be in the same state
        if (x->bank != b->banks[r]) return PE_ESTATE;      // particles moved banks (plain PIC sort)
        if (x->dT_cur != x->cfg.dT) return PE_ESTATE;     // the ensemble steps by the configured Delta t
    }
    // The batch stream waits for work already queued on the contexts' streams.
    for (int r = 0; r < R; ++r) {
        if (b->ctx[r]->stream == b->stream) continue;
        if (cudaEventRecord(b->ev_in, b->ctx[r]->stream) != cudaSuccess ||
            cudaStreamWaitEvent(b->stream, b->ev_in, 0) != cudaSuccess)
            return PE_ECUDA;
    }
    // Lifting (or, after pe_load_initial, the charge of the loaded particles) into rho_all
    int64_t* rho_all = reinterpret_cast<int64_t*>(at(b, b->L.rho));
    for (int r = 0; r < R; ++r) {
        pe_ctx* x = b->ctx[r];
        const pe_config& c = x->cfg;
        const int k = x->bank;
        if (!fresh) {
            PE_TRY(pe_refine(x->coarse, x->nc, c.wavelet, c.ncell, x->prof, x->prof + c.ncell, b->stream));
            if (x->walls)  // bounded grid: equal weights, wall deposits doubled to densities
                PE_TRY(pe_quiet_start_equal(x->cell[k], x->theta[k], x->v[k], x->w[k], c.nparticles, c.ncell,
                                            x->prof, x->prof + c.ncell, 2.0f, (float)c.v_th, pe_ctx_lift_seed(x),
                                            x->s_w, x->eq_scratch, rho_all + b->rho_off[r], x->status, b->stream));
            else
                PE_TRY(pe_quiet_start(x->cell[k], x->theta[k], x->v[k], x->w[k], c.nparticles, c.ncell, x->prof,
                                      x->prof + c.ncell, (float)c.v_th, pe_ctx_lift_seed(x), x->s_w,
                                      rho_all + b->rho_off[r], x->status, b->stream));
        } else {
            PE_TRY(pe_deposit(x->cell[k], x->theta[k], x->w[k], c.nparticles, c.ncell, x->s_w,
                              rho_all + b->rho_off[r], x->status, b->stream));
        }
    }
    // Burst + restriction + projection: eager on the first call, then a captured graph
    // (always eager on the legacy default stream, which cannot be captured).
    const bool capturable = b->stream != nullptr && b->stream != cudaStreamLegacy && b->stream != cudaStreamPerThread;
    if (b->steps_done == 0 || !b->graph) {
        if (b->steps_done == 0 || !capturable) {
            PE_TRY(burst_restrict_project(b));
        } else {
            cudaGraph_t g;
            const long long k0 = pe_launch_count();
            if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PE_ECUDA;
            const int rc = burst_restrict_project(b);
            if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess || rc != PE_OK) return rc != PE_OK ? rc : PE_ECUDA;
            b->graph_kernels = pe_launch_count() - k0;
            const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return PE_ECUDA;
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return PE_ECUDA;
        }
    } else {
        if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return PE_ECUDA;
        note_launches((int)b->graph_kernels);
    }
    // The contexts' streams wait for the batch before any later call on them.
    if (cudaEventRecord(b->ev_out, b->stream) != cudaSuccess) return PE_ECUDA;
    for (int r = 0; r < R; ++r)
        if (b->ctx[r]->stream != b->stream && cudaStreamWaitEvent(b->ctx[r]->stream, b->ev_out, 0) != cudaSuccess)
            return PE_ECUDA;
    for (int r = 0; r < R; ++r) {
        pe_ctx* x = b->ctx[r];
        x->macro_steps += 1;
        x->coarse_state = 1;
        x->fine_steps += b->K;
        x->time += x->cfg.dT;
        x->v_at_integer = 0;
        x->rho_valid = 0;  // the charge lives in the batch's grid, not the context's
        x->fresh = 0;
    }
    b->steps_done += 1;
    return PE_OK;
}
