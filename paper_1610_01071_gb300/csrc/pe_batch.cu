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

#include <map>
#include <mutex>
#include <vector>

#include "pe_ctx.h"
#include "pe_internal.h"
#include "pepic.h"

using namespace pe;

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t push, field, proj, refine, coarse_ptrs, items, counter, rho, e0, samp, total;
    int64_t rho_total, samp_row, max_items;
};

// The smallest chunk the tuner may choose bounds the work-list length.
constexpr int64_t kMinChunk = 4096;
const int64_t kChunkCandidates[] = {16384, 32768, 65536};
const int kBlockCandidates[] = {128, 256, 512};

// Tuned launch shapes, cached by the ensemble's composition: the (ncell, N) of every realisation
// in order, and the device.
struct Tuned {
    int64_t chunk;
    int block, priv;
};
std::mutex g_tune_mu;
std::map<std::vector<int64_t>, Tuned> g_tuned;

int layout_for(pe_ctx* const* ctxs, int n, Layout* L)
{
    if (!ctxs || n < 1) return PE_EINVAL;
    const int K = ctxs[0]->cfg.K;
    int64_t rho = 0, row = 0, items = 0;
    for (int r = 0; r < n; ++r) {
        const pe_ctx* x = ctxs[r];
        if (!x || x->cfg.K != K || x->cfg.wavelet != PE_WAVELET_HAAR || x->cfg.ncell < 64 || x->ps || x->pres || x->kinetic)
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
    L->refine = off;
    off += a256(refine_desc_size() * n);
    L->coarse_ptrs = off;
    off += a256(sizeof(double*) * n);
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
    int block, priv;  // particle launch shape: threads per block, shared-memory deposit window
    int nitems;
    int max_ncell, max_nb;
    // Field-solve groups, one launch each: (cluster size G) x (FP32 | FP64 Jacobian solve; FP64
    // only for bounded grids with kWallsJacobianFP64). The batch sizes clusters for throughput
    // (newton_batch_cluster_size), so its solves can differ from a lone context's in the last
    // bits (the same equations, another partition of the linear solve); both converge to the
    // Newton tolerance.
    struct FieldGroup {
        int G;
        bool fp64;
        int maxn;
        std::vector<int> ids;
    };
    std::vector<FieldGroup> fgroups;
    std::vector<int64_t> rho_off, e0_off, samp_off;
    std::vector<int> banks;  // particle bank of each context when the descriptors were built
    cudaGraphExec_t graph;
    long long graph_kernels;
    int steps_done;
    cudaEvent_t ev_in, ev_out;  // ordering against the contexts' streams
    // field-solve groups run concurrently: forked onto side streams and joined (in the captured
    // graph these become parallel branches)
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork;
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

// frozen: push descriptors with dt/dx = 0 (the tuner's probe: with kick 0 a fused pass then
// rewrites every particle unchanged while doing all of a real pass's work).
static int build_descs(pe_batch* b, bool frozen = false)
{
    const int R = (int)b->ctx.size();
    std::vector<char> push(push_desc_size() * R), proj(proj_desc_size() * R);
    std::vector<char> fd(field_desc_size() * R);
    std::vector<int> slot(R, 0);  // position of each realisation's field descriptor
    {
        int o = 0;
        for (const auto& fg : b->fgroups)
            for (int r : fg.ids) slot[r] = o++;
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
                       x->Ef, c.ncell, frozen ? 0.0f : (float)(c.dt / x->dx), (float)(c.qm * c.dt), x->s_w,
                       rho_all + b->rho_off[r],
                       e0_all + b->e0_off[r], c.dT, c.dt, (float)(1.0 / x->dx), (float)c.qm, c.comoving,
                       x->s_p, x->bin_shift, samp_all + b->samp_off[r], b->L.samp_row, x->walls, x->status);
        make_proj_desc(proj.data() + proj_desc_size() * r, samp_all + b->samp_off[r], b->L.samp_row, c.ncell, x->nc,
                       x->s_w, x->s_p, x->csamples, x->coarse, x->slope);
        char* dst = fd.data() + field_desc_size() * slot[r];
        make_field_desc(dst, rho_all + b->rho_off[r], c.ncell, x->dx, x->s_w, c.poisson, x->walls, c.newton_tol,
                        c.newton_maxit, x->phi, x->E, x->Ef, x->diag, x->status, x->phi + c.ncell);
    }
    std::vector<char> ref(refine_desc_size() * R);
    std::vector<const double*> cptr(R);
    for (int r = 0; r < R; ++r) {
        pe_ctx* x = b->ctx[r];
        make_refine_desc(ref.data() + refine_desc_size() * r, x->coarse, x->nc, x->cfg.ncell, x->prof,
                         x->prof + x->cfg.ncell);
        cptr[r] = x->coarse;
    }
    if (cudaMemcpy(at(b, b->L.refine), ref.data(), ref.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(at(b, b->L.coarse_ptrs), cptr.data(), sizeof(double*) * R, cudaMemcpyHostToDevice) != cudaSuccess)
        return PE_ECUDA;
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
    const bool fork = b->fgroups.size() > 1;
    if (fork && cudaEventRecord(b->ev_fork, b->stream) != cudaSuccess) return PE_ECUDA;
    size_t o = 0;
    for (size_t k = 0; k < b->fgroups.size(); ++k) {
        const auto& fg = b->fgroups[k];
        const int n = (int)fg.ids.size();
        cudaStream_t s = fork ? b->side[k] : b->stream;
        if (fork && cudaStreamWaitEvent(s, b->ev_fork, 0) != cudaSuccess) return PE_ECUDA;
        PE_TRY(launch_newton_batch(base + field_desc_size() * o, n, fg.G, fg.maxn, fg.fp64, extrap, s));
        if (fork && cudaEventRecord(b->ev_join[k], s) != cudaSuccess) return PE_ECUDA;
        o += (size_t)n;
    }
    if (fork)
        for (size_t k = 0; k < b->fgroups.size(); ++k)
            if (cudaStreamWaitEvent(b->stream, b->ev_join[k], 0) != cudaSuccess) return PE_ECUDA;
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
                                          b->max_ncell, b->max_nb, b->block, b->priv, s));
            break;
        }
        if (cudaMemsetAsync(rho_all, 0, 8 * (size_t)b->L.rho_total, s) != cudaSuccess) return PE_ECUDA;
        PE_TRY(launch_particles_batch(0, at(b, b->L.push), at(b, b->L.items), b->nitems, p, p == 0 ? 0.5f : 1.0f,
                                      counter, b->max_ncell, b->max_nb, b->block, b->priv, s));
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
    b->block = 256;
    b->priv = 1;
    b->graph = nullptr;
    b->graph_kernels = 0;
    b->steps_done = 0;
    if (cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        delete b;
        return PE_ECUDA;
    }
    b->max_ncell = 0;
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
        const int G = newton_batch_cluster_size(x->cfg.ncell);
        if (G < 1) {
            cudaEventDestroy(b->ev_in);
            cudaEventDestroy(b->ev_out);
            delete b;
            return PE_EINVAL;
        }
        const bool fp64 = x->walls != 0 && kWallsJacobianFP64;
        bool placed = false;
        for (auto& fg : b->fgroups)
            if (fg.G == G && fg.fp64 == fp64) {
                fg.ids.push_back(r);
                if (x->cfg.ncell > fg.maxn) fg.maxn = x->cfg.ncell;
                placed = true;
            }
        if (!placed) b->fgroups.push_back({G, fp64, x->cfg.ncell, {r}});
    }
    int rc = PE_OK;
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) rc = PE_ECUDA;
    for (size_t k = 0; rc == PE_OK && k < b->fgroups.size(); ++k) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            rc = PE_ECUDA;
            break;
        }
        b->side.push_back(st);
        b->ev_join.push_back(ev);
    }
    if (rc == PE_OK) rc = build_descs(b);
    if (rc == PE_OK) rc = build_items(b);
    if (rc == PE_OK && cudaMemset(at(b, L.e0), 0, 4 * (size_t)L.rho_total) != cudaSuccess) rc = PE_ECUDA;
    if (rc != PE_OK) {
        pe_batch_destroy(b);
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
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    for (cudaStream_t st : b->side) cudaStreamDestroy(st);
    delete b;
}

static void drop_graph(pe_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

static std::vector<int64_t> composition(const pe_batch* b)
{
    std::vector<int64_t> key;
    int dev = 0;
    cudaGetDevice(&dev);
    key.push_back(dev);
    for (const pe_ctx* x : b->ctx) {
        key.push_back(x->cfg.ncell);
        key.push_back(x->cfg.nparticles);
    }
    return key;
}

// Times one launch shape: the read-only sample pass (row K + 1, scratch) and the deposit pass
// (into the ensemble's charge grid, rewritten before every push) over every realisation's
// particles, the two halves of the fused push; best of two.
// Time of one fused pass of the burst (push + deposit + binned sample, mode 0) in the current
// shape, on frozen descriptors with kick 0: the particles are rewritten unchanged, the deposit
// and sample land in the batch's charge grid and sample row 0, which every burst clears before
// use. Best of two after a warm-up.
static int time_shape(pe_batch* b, cudaEvent_t e0, cudaEvent_t e1, float* ms_out)
{
    unsigned* counter = reinterpret_cast<unsigned*>(at(b, b->L.counter));
    int64_t* rho_all = reinterpret_cast<int64_t*>(at(b, b->L.rho));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {  // the first repetition warms up
        cudaEventRecord(e0, b->stream);
        if (cudaMemsetAsync(rho_all, 0, 8 * (size_t)b->L.rho_total, b->stream) != cudaSuccess) return PE_ECUDA;
        PE_TRY(launch_particles_batch(0, at(b, b->L.push), at(b, b->L.items), b->nitems, 0, 0.0f, counter,
                                      b->max_ncell, b->max_nb, b->block, b->priv, b->stream));
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return PE_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    *ms_out = best;
    return PE_OK;
}

extern "C" PE_API int pe_batch_tune(pe_batch* b, int64_t* chosen_chunk)
{
    if (!b) return PE_EINVAL;
    const std::vector<int64_t> key = composition(b);
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            b->chunk = it->second.chunk;
            b->block = it->second.block;
            b->priv = it->second.priv;
            cached = true;
        }
    }
    if (!cached) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PE_ECUDA;
        float best = 1e30f;
        Tuned pick{b->chunk, b->block, b->priv};
        int rc = build_descs(b, true);
        for (int64_t cand : kChunkCandidates) {
            if (rc != PE_OK) break;
            b->chunk = cand;
            rc = build_items(b);
            for (int blk : kBlockCandidates)
                for (int pv = 1; pv >= 0 && rc == PE_OK; --pv) {
                    b->block = blk;
                    b->priv = pv;
                    float ms = 0.f;
                    rc = time_shape(b, e0, e1, &ms);
                    if (rc == PE_OK && ms < best) {
                        best = ms;
                        pick = Tuned{cand, blk, pv};
                    }
                }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const int rc_descs = build_descs(b);  // the real steps' descriptors again, also after an error
        if (rc != PE_OK) return rc;
        if (rc_descs != PE_OK) return rc_descs;
        b->chunk = pick.chunk;
        b->block = pick.block;
        b->priv = pick.priv;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = pick;
    }
    PE_TRY(build_items(b));
    drop_graph(b);
    if (chosen_chunk) *chosen_chunk = b->chunk;
    return PE_OK;
}

extern "C" PE_API int pe_batch_tuned(const pe_batch* b, int64_t* chunk, int32_t* block, int32_t* privatised)
{
    if (!b || !chunk || !block || !privatised) return PE_EINVAL;
    *chunk = b->chunk;
    *block = b->block;
    *privatised = b->priv;
    return PE_OK;
}

// Mean of the coarse states of a group of realisations: thread k sums component k over the
// members in the given order (fixed, so repeated calls return the same bits).
constexpr int kGroupMax = 128;
struct GroupMembers {
    int n;
    int idx[kGroupMax];
};

__global__ void k_group_mean(const double* const* coarse, GroupMembers m, int ncoef, double* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncoef) return;
    double s = 0.0;
    for (int i = 0; i < m.n; ++i) s += coarse[m.idx[i]][k];
    out[k] = s / (double)m.n;
}

extern "C" PE_API int pe_batch_group_mean(pe_batch* b, const int32_t* members, int32_t nmembers, double* out)
{
    if (!b || !members || !out || nmembers < 1 || nmembers > kGroupMax) return PE_EINVAL;
    GroupMembers m{};
    m.n = nmembers;
    int64_t ncoef = -1;
    for (int i = 0; i < nmembers; ++i) {
        const int r = members[i];
        if (r < 0 || r >= (int)b->ctx.size()) return PE_EINVAL;
        const int64_t nc = 2 * (int64_t)b->ctx[r]->nc;
        if (ncoef >= 0 && nc != ncoef) return PE_EINVAL;  // one coarse layout per group
        ncoef = nc;
        m.idx[i] = r;
    }
    k_group_mean<<<(int)((ncoef + 255) / 256), 256, 0, b->stream>>>(
        reinterpret_cast<const double* const*>(at(b, b->L.coarse_ptrs)), m, (int)ncoef, out);
    return launch_status();
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
        if (x->dT_cur != x->cfg.dT || x->K_cur != x->cfg.K) return PE_ESTATE;  // the configured step and burst
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
    if (!fresh)  // every realisation's lifting profile in one launch
        PE_TRY(launch_refine_batch(at(b, b->L.refine), R, PE_WAVELET_HAAR, b->max_ncell, b->stream));
    // The realisations' loadings are independent: spread over the side streams so that small
    // ones overlap (each is a few short launches), then joined.
    const int nside = (int)std::min<size_t>(b->side.size(), (size_t)R);
    const bool fork = nside > 1;
    if (fork) {
        if (cudaEventRecord(b->ev_fork, b->stream) != cudaSuccess) return PE_ECUDA;
        for (int k = 0; k < nside; ++k)
            if (cudaStreamWaitEvent(b->side[k], b->ev_fork, 0) != cudaSuccess) return PE_ECUDA;
    }
    for (int r = 0; r < R; ++r) {
        pe_ctx* x = b->ctx[r];
        const pe_config& c = x->cfg;
        const int k = x->bank;
        cudaStream_t ls = fork ? b->side[r % nside] : b->stream;
        if (!fresh) {
            if (x->walls)  // bounded grid: equal weights, wall deposits doubled to densities
                PE_TRY(pe_quiet_start_equal(x->cell[k], x->theta[k], x->v[k], x->w[k], c.nparticles, c.ncell,
                                            x->prof, x->prof + c.ncell, 2.0f, (float)c.v_th, pe_ctx_lift_seed(x),
                                            x->s_w, x->eq_scratch, rho_all + b->rho_off[r], x->status, ls));
            else
                PE_TRY(pe_quiet_start(x->cell[k], x->theta[k], x->v[k], x->w[k], c.nparticles, c.ncell, x->prof,
                                      x->prof + c.ncell, (float)c.v_th, pe_ctx_lift_seed(x), x->s_w,
                                      rho_all + b->rho_off[r], x->status, ls));
        } else {
            PE_TRY(pe_deposit(x->cell[k], x->theta[k], x->w[k], c.nparticles, c.ncell, x->s_w,
                              rho_all + b->rho_off[r], x->status, ls));
        }
    }
    if (fork) {
        for (int k = 0; k < nside; ++k) {
            if (cudaEventRecord(b->ev_join[k], b->side[k]) != cudaSuccess ||
                cudaStreamWaitEvent(b->stream, b->ev_join[k], 0) != cudaSuccess)
                return PE_ECUDA;
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
