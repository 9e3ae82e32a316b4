// Particle kernels: charge deposit, leapfrog gather+push fused with the deposit and
// the co-moving restriction sample, quiet-start loading, and the counting sort.
//
// Layout: structure of arrays (cell int32, theta f32, v f32, w f32), read and written
// as 16-byte vectors of four consecutive particles; each block owns one contiguous
// chunk of the (cell-sorted) particle array, so its deposits land in a narrow range
// of nodes: per-lane register windows absorb most of them, the rest go to a
// block-private int64 grid in shared memory that is flushed once with global atomics.
// All sums are integers, so the result is exact and independent of order.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <climits>
#include <type_traits>

#include "pe_common.cuh"
#include "pe_eq.cuh"
#include "pe_internal.h"

namespace pe {

struct PushParams {
    int32_t* cell;
    float* theta;
    float* v;
    const float* w;
    int64_t n;
    int64_t chunk;
    const float* Ef;
    int ncell, mask;
    float dt_dx, qm_dt, kick, wscale;
    unsigned long long* rho;  // charge of the pushed particles (PUSH) or current ones (DEPOSIT)
    int rho_width;
    const float* E0f;  // restriction sample (SAMPLE)
    float tau_dx, qm_tau, pscale;
    unsigned long long* samp_n;
    unsigned long long* samp_m;
    int samp_width;
    int bin_shift;  // > 0: samples summed over bins of 2^bin_shift nodes (BINNED modes)
    uint32_t* status;
    // batched launches: per-step fields derived on the device from these
    double dT, dt;                     // tau = comoving ? (float)(dT - p dt) : 0, as on the host
    float inv_dx, qm;
    int comoving;
    unsigned long long* samp_base;     // sample row p starts at samp_base + p * row_stride
    int64_t row_stride;
    int64_t max_chunk;                 // largest particle chunk per block (<= 65536; 0 = 65536)
    // phase-space sample (PS modes): samp_n is the histogram [(ncell >> bin_shift)][nv]
    int nv, ps_width;
    float vmin, inv_dv;
    float tent_scale;  // hat rows (the TENT modes): 2^(24 - bin_shift)
    // second velocity moment (the E modes): samp_e[ncell], fixed point at escale = 2^s_e
    unsigned long long* samp_e;
    float escale;
    // bounded grid (walls at nodes 0 and ncell-1, Section 4.2): a particle whose drift ends
    // outside [0, (ncell-1) dx) is absorbed (weight 0 written to w_out, parked on the wall node
    // with v = 0); particles of weight 0 are not moved; co-moving targets outside are dropped
    int walls;
    float* w_out;
};

enum Mode {
    kDeposit = 0,
    kPush = 1,
    kPushSample = 2,
    kSample = 3,
    kPushSampleBinned = 4,
    kSampleBinned = 5,
    kPushSamplePS = 6,  // push + phase-space sample
    kSamplePS = 7,
    kPushSamplePSW = 8,  // push + phase-space sample with hat rows (the wavelet form)
    kSamplePSW = 9,
    kPushSampleE = 10,  // push + nodal sample of density, momentum and second moment
    kSampleE = 11,
    kPushSampleBinnedE = 12,  // push + Haar-binned sample of the three moments
    kSampleBinnedE = 13
};

template <int MODE>
struct ModeTraits {
    static constexpr bool rho = (MODE == kDeposit || MODE == kPush || MODE == kPushSample || MODE == kPushSampleBinned ||
                                 MODE == kPushSamplePS || MODE == kPushSamplePSW || MODE == kPushSampleE ||
                                 MODE == kPushSampleBinnedE);
    static constexpr bool push = (MODE == kPush || MODE == kPushSample || MODE == kPushSampleBinned ||
                                  MODE == kPushSamplePS || MODE == kPushSamplePSW || MODE == kPushSampleE ||
                                  MODE == kPushSampleBinnedE);
    static constexpr bool sample = (MODE == kPushSample || MODE == kSample || MODE == kPushSampleBinned ||
                                    MODE == kSampleBinned || MODE == kPushSamplePS || MODE == kSamplePS ||
                                    MODE == kPushSamplePSW || MODE == kSamplePSW || MODE == kPushSampleE ||
                                    MODE == kSampleE || MODE == kPushSampleBinnedE || MODE == kSampleBinnedE);
    // third moment (the second velocity moment), nodal or binned
    static constexpr bool energy = (MODE == kPushSampleE || MODE == kSampleE || MODE == kPushSampleBinnedE ||
                                    MODE == kSampleBinnedE);
    static constexpr bool binned = (MODE == kPushSampleBinned || MODE == kSampleBinned || MODE == kPushSampleBinnedE ||
                                    MODE == kSampleBinnedE);
    static constexpr bool tent = (MODE == kPushSamplePSW || MODE == kSamplePSW);
    static constexpr bool ps = (MODE == kPushSamplePS || MODE == kSamplePS || tent);
    // particle streams staged through shared memory (cp.async, one group ahead): the phase-space
    // passes (three blocks an SM) and the deposit gain from it; the other passes, at four blocks
    // an SM with their loads already in flight, run faster on direct loads and a larger L1
    static constexpr bool stage = ps || MODE == kDeposit;
};

// Fixed-point value rn(x 2^s); records in *ovf whether it left the range |q| <= 2^23.
__device__ __forceinline__ int32_t fx_weight(float x, float scale, bool* ovf)
{
    const int32_t q = __float2int_rn(x * scale);
    *ovf |= (q > (1 << 23)) | (q < -(1 << 23));
    return q;
}

constexpr int kThreads = 256;

// Block-local table of the nodal fields the gathers read, for the nodes [base, base + width)
// (mod ncell) around the block's first cell: entry i holds, for node c = base + i,
// {E_c, E_{c+1} - E_c, E0_c, E0_{c+1} - E0_c} (E0 only when the pass samples). A CIC gather is
// then one shared-memory load and one fma per field; the differences are the same FP32
// subtractions the gather would do, so results are unchanged. Nodes outside the window (a
// particle far from its block's cells) read the global fields.
constexpr int kFieldTabNodes = 256;

struct FieldTab {
    uint32_t s;  // shared address of entry 0
    int base, width;
};

__device__ __forceinline__ float4 lds_f4(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ float2 lds_f2(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ int4 lds_i4(uint32_t a)
{
    int4 v;
    asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

// 16-byte asynchronous copy global -> shared (cached in L2 only) and its group controls: each
// lane copies its own next group of particles and waits only for its own copies.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Staging of the particle streams: per warp two slots (the group being processed and the next
// one, in flight), each holding the four arrays' 16-byte vectors of the 32 lanes.
constexpr int kStageSlotBytes = 4 * 32 * 16;
constexpr int kStageWarpBytes = 2 * kStageSlotBytes;

// True when cell c + k (k = fl, an integer-valued float) lies between the walls,
// [0, ncell - 1); NaN counts as outside.
__device__ __forceinline__ bool inside_walls(const PushParams& P, int c, float fl)
{
    return fl >= -(float)c && fl < (float)(P.ncell - 1 - c);
}

// One particle: gather, co-moving restriction sample, kick and drift (as the mode asks). Returns
// true when the particle's charge is to be deposited at (c_out, th_out) with fixed-point weight
// wq_out (the caller deposits a whole group at once, see deposit_group).
// Binned restriction sample of one particle, left for the caller's warp-uniform bin window:
// the bin of its left node, its fixed-point weight and momentum, and theta_q when its right
// node lies in the next bin (0 otherwise); ok = false when it samples nothing.
struct BinSample {
    int b;
    int32_t mq;
    int32_t eq;  // second moment (the energy modes)
    uint32_t tq;
    bool ok;
};

template <int MODE, bool WALLS>
__device__ __forceinline__ bool process(const PushParams& P, const FieldTab& ft, bool act, int c, float th,
                                        float vv, float ww, BinSample& bs, const SmemGrid& gsn, const SmemGrid& gsm,
                                        const SmemGrid& gse, const PSGrid& gps, PSAccW& acc, PSAcc2& acc2, bool* ovf, int& c_out, float& th_out,
                                        float& v_out, float& w_out, int32_t& wq_out)
{
    using Tr = ModeTraits<MODE>;
    c_out = c;
    th_out = th;
    v_out = vv;
    w_out = ww;
    wq_out = 0;
    bs.b = 0;
    bs.mq = 0;
    if (Tr::energy) bs.eq = 0;
    bs.tq = 0u;
    bs.ok = false;
    if (!act) return false;  // a lane past the end of its warp's slice
    if ((unsigned)c >= (unsigned)P.ncell) {
        raise_flag(P.status, PE_FLAG_RANGE);
        return false;
    }
    if (WALLS) {
        if (ww == 0.0f) return false;  // absorbed: frozen, carries nothing
        if (c >= P.ncell - 1) {        // a live particle must lie between the walls
            raise_flag(P.status, PE_FLAG_RANGE);
            return false;
        }
    }
    const int32_t wq = fx_weight(ww, P.wscale, ovf);
    wq_out = wq;
    if (MODE == kDeposit) return true;
    // CIC gather of E (and of the frame field E0 when sampling) at the particle
    float Ec, dE, E0c = 0.f, dE0 = 0.f;
    const int fi = (c - ft.base) & P.mask;
    if (fi < ft.width) {
        if (Tr::sample) {
            const float4 f = lds_f4(ft.s + 16u * (uint32_t)fi);
            Ec = f.x;
            dE = f.y;
            E0c = f.z;
            dE0 = f.w;
        } else {
            const float2 f = lds_f2(ft.s + 8u * (uint32_t)fi);
            Ec = f.x;
            dE = f.y;
        }
    } else {
        const int c1 = (c + 1) & P.mask;
        Ec = __ldg(P.Ef + c);
        dE = __ldg(P.Ef + c1) - Ec;
        if (Tr::sample) {
            E0c = __ldg(P.E0f + c);
            dE0 = __ldg(P.E0f + c1) - E0c;
        }
    }
    const float Ep = fmaf(th, dE, Ec);
    if (Tr::sample) {
        // Appendix B: carry the particle along the approximate characteristic to t_{n+1}
        const float vbar = fmaf((P.kick - 0.5f) * P.qm_dt, Ep, vv);  // integer-time velocity
        const float E0p = fmaf(th, dE0, E0c);
        const float xs = fmaf(P.tau_dx, vbar, th);
        float fl = floorf(xs);
        float ths = xs - fl;
        if (ths >= 1.0f) {
            ths = 0.0f;
            fl += 1.0f;
        }
        const int k = (int)fl;
        const int cs = (c + k) & P.mask, cs1 = (cs + 1) & P.mask;
        const float vt = fmaf(P.qm_tau, E0p, vbar);
        // bounded grid: a target beyond a wall has left the domain by t_{n+1}
        const bool counted = !WALLS || inside_walls(P, c, fl);
        if (Tr::ps && counted) {
            // Section 3.3 restriction: CIC in x (summed over the coarse bin), nearest cell in v
            const float jf = floorf((vt - P.vmin) * P.inv_dv);
            const int j = jf < 0.0f ? 0 : (jf >= (float)P.nv ? P.nv - 1 : (int)jf);
            const int b0 = cs >> P.bin_shift, b1 = cs1 >> P.bin_shift;
            if (Tr::tent) {
                // hat of half-width 2^b around the coarse nodes (Eq. restriction applied b times
                // to the CIC histogram): the fraction f of the way from node b0 to the next one
                const float f = ((float)(cs & ((1 << P.bin_shift) - 1)) + ths) * P.tent_scale;
                acc2.add((b0 << 16) | j, wq, (long long)wq * (long long)__float2uint_rn(f), gps);
            } else if (b0 == b1) {
                acc.add((b0 << 16) | j, wq, gps);
            } else {  // split across a bin edge (rare): both parts go straight to the grid
                const FxSplit qn = fx_split(wq, ths);
                gps.add_at(b0, j, (long long)qn.left);
                gps.add_at(b1, j, (long long)qn.right);
            }
        }
        if (!Tr::ps && counted) {
            const int32_t mq = fx_weight(ww * vt, P.pscale, ovf);
            if (Tr::binned) {
                // whole particle in the bin of its left node; the right part of a particle on a
                // bin's last node moves to the next bin (theta_q as in fx_split)
                const int bm = (1 << P.bin_shift) - 1;
                bs.b = cs >> P.bin_shift;
                bs.mq = mq;
                if (Tr::energy) bs.eq = fx_weight(__fmul_rn(__fmul_rn(ww, vt), vt), P.escale, ovf);
                bs.tq = ((cs & bm) == bm) ? __float2uint_rn(ths * kThetaOneF) : 0u;
                bs.ok = true;
            } else {
                const FxSplit qn = fx_split(wq, ths);
                const FxSplit qp = fx_split(mq, ths);
                gsn.add(cs, qn.left);
                gsn.add(cs1, qn.right);
                gsm.add(cs, qp.left);
                gsm.add(cs1, qp.right);
                if (Tr::energy) {  // Section 3.2: the second moment w V~^2 with the same split
                    const int32_t eq = fx_weight(__fmul_rn(__fmul_rn(ww, vt), vt), P.escale, ovf);
                    const FxSplit qe = fx_split(eq, ths);
                    gse.add(cs, qe.left);
                    gse.add(cs1, qe.right);
                }
            }
        }
    }
    if (Tr::push) {
        // Section 2.2 leapfrog: kick with the gathered field, then drift
        const float vn = fmaf(P.kick * P.qm_dt, Ep, vv);
        const float s = fmaf(vn, P.dt_dx, th);
        float fl = floorf(s);
        float thn = s - fl;
        if (thn >= 1.0f) {
            thn = 0.0f;
            fl += 1.0f;
        }
        if (WALLS && !inside_walls(P, c, fl)) {  // absorbed at the wall it crossed
            c_out = (fl < 0.0f) ? 0 : P.ncell - 1;
            th_out = 0.0f;
            v_out = 0.0f;
            w_out = 0.0f;
            return false;
        }
        c_out = (c + (int)fl) & P.mask;
        th_out = thn;
        v_out = vn;
        return true;
    }
    return false;
}

// Charge deposit of one particle straight to the block grid (outside the warp window).
__device__ __forceinline__ void deposit_direct(const SmemGrid& g, int c, float th, int32_t wq, int mask)
{
    const FxSplit q = fx_split(wq, th);
    g.add(c, q.left);
    g.add((c + 1) & mask, q.right);
}

// Deposits a group (four particles per lane, dep_k set where particle k deposits at cell c_k,
// offset th_k, weight q_k) through the warp window: when the warp's cells leave the window's
// three cells, the window moves (warp-uniformly) to the lowest cell; cells still beyond it
// (a spread of more than three cells) go straight to the grid. Called by all 32 lanes.
__device__ __forceinline__ void deposit_group(WarpWindow& win, const SmemGrid& g, int ncell, int mask, const int4& c,
                                              const float4& th, int32_t q0, int32_t q1, int32_t q2, int32_t q3,
                                              bool e0, bool e1, bool e2, bool e3)
{
    const int H = ncell >> 1;  // cells as signed offsets from the base (periodic)
    int r0 = ((c.x - win.base + H) & mask) - H, r1 = ((c.y - win.base + H) & mask) - H;
    int r2 = ((c.z - win.base + H) & mask) - H, r3 = ((c.w - win.base + H) & mask) - H;
    int lo = INT_MAX, hi = INT_MIN;
    if (e0) lo = min(lo, r0), hi = max(hi, r0);
    if (e1) lo = min(lo, r1), hi = max(hi, r1);
    if (e2) lo = min(lo, r2), hi = max(hi, r2);
    if (e3) lo = min(lo, r3), hi = max(hi, r3);
    lo = __reduce_min_sync(0xFFFFFFFFu, lo);
    hi = __reduce_max_sync(0xFFFFFFFFu, hi);
    if (lo == INT_MAX) return;  // nothing to deposit in this group
    if (lo < 0 || hi > 2) {
        win.move(g, lo);
        r0 -= lo;
        r1 -= lo;
        r2 -= lo;
        r3 -= lo;
    }
    if (e0) {
        if ((unsigned)r0 <= 2u) win.add(r0, fx_split(q0, th.x));
        else deposit_direct(g, c.x, th.x, q0, mask);
    }
    if (e1) {
        if ((unsigned)r1 <= 2u) win.add(r1, fx_split(q1, th.y));
        else deposit_direct(g, c.y, th.y, q1, mask);
    }
    if (e2) {
        if ((unsigned)r2 <= 2u) win.add(r2, fx_split(q2, th.z));
        else deposit_direct(g, c.z, th.z, q2, mask);
    }
    if (e3) {
        if ((unsigned)r3 <= 2u) win.add(r3, fx_split(q3, th.w));
        else deposit_direct(g, c.w, th.w, q3, mask);
    }
}

// One block owns a contiguous chunk of <= 65536 particles; each warp a contiguous slice
// of it, read with 16-byte loads (4 particles per lane).
template <int MODE, bool WALLS>
__device__ __forceinline__ void particle_chunk(const PushParams& P, int64_t begin, int64_t end, uint32_t* smem)
{
    using Tr = ModeTraits<MODE>;
    constexpr bool kRho = Tr::rho;
    constexpr bool kSamp = Tr::sample && !Tr::binned;
    constexpr bool kBin = Tr::binned;
    constexpr bool kWrite = Tr::push;
    constexpr bool kNeedV = (MODE != kDeposit);

    const int c_first = (begin < end) ? (P.cell[begin] & P.mask) : 0;

    SmemGrid grho{}, gsn{}, gsm{}, gse{};
    BinGrid bsn{}, bsm{}, bse{};
    PSGrid gps{};
    constexpr bool kPS = Tr::ps;
    uint32_t* s = smem;
    FieldTab ft{0u, 0, 0};
    if (kNeedV) {  // field table first (16-byte aligned); filled before the block barrier below
        ft.width = P.ncell < kFieldTabNodes ? P.ncell : kFieldTabNodes;
        ft.base = P.ncell <= kFieldTabNodes ? 0 : ((c_first - kFieldTabNodes / 4) & P.mask);
        ft.s = smem_u32(s);
        for (int i = threadIdx.x; i < ft.width; i += blockDim.x) {
            const int n0 = (ft.base + i) & P.mask, n1 = (n0 + 1) & P.mask;
            const float e0 = __ldg(P.Ef + n0), e1 = __ldg(P.Ef + n1);
            if (Tr::sample) {
                const float f0 = __ldg(P.E0f + n0), f1 = __ldg(P.E0f + n1);
                reinterpret_cast<float4*>(s)[i] = make_float4(e0, e1 - e0, f0, f1 - f0);
            } else {
                reinterpret_cast<float2*>(s)[i] = make_float2(e0, e1 - e0);
            }
        }
        s += (Tr::sample ? 4 : 2) * kFieldTabNodes;
    }
    if (kRho) s = grho.bind(s, P.rho, P.rho_width < P.ncell ? ((c_first - 64) & P.mask) : 0, P.rho_width, P.mask);
    if (kSamp) {
        const int sb = P.samp_width < P.ncell ? ((c_first - P.samp_width / 2) & P.mask) : 0;
        s = gsn.bind(s, P.samp_n, sb, P.samp_width, P.mask);
        s = gsm.bind(s, P.samp_m, sb, P.samp_width, P.mask);
        if (Tr::energy) s = gse.bind(s, P.samp_e, sb, P.samp_width, P.mask);
    }
    if (kBin) {
        const int nb = P.ncell >> P.bin_shift;
        s = bsn.bind(s, P.samp_n, nb);
        if (Tr::energy) s = bse.bind(s, P.samp_e, nb);
        s = bsm.bind(s, P.samp_m, nb);
    }
    if (kPS) {
        const int nxc = P.ncell >> P.bin_shift;
        s = gps.bind(s, P.samp_n, ((c_first >> P.bin_shift) - P.ps_width / 2) & (nxc - 1), P.ps_width, nxc, P.nv);
        gps.zero();
    }
    // this warp's staging slots, after the grids (16-byte aligned)
    const uint32_t stage = ((smem_u32(s) + 15u) & ~15u) + (uint32_t)(threadIdx.x >> 5) * (uint32_t)kStageWarpBytes +
                           16u * (uint32_t)(threadIdx.x & 31);
    if (kRho) grho.zero();
    if (kSamp) {
        gsn.zero();
        gsm.zero();
        if (Tr::energy) gse.zero();
    }
    if (kBin) {
        if (Tr::energy) bse.zero();
        bsn.zero();
        bsm.zero();
    }
    __syncthreads();

    const int64_t gb0 = begin >> 2, gb1 = end >> 2;  // begin is a multiple of 4
    int64_t g0, g1;
    warp_groups(gb0, gb1, &g0, &g1);
    const int lane = threadIdx.x & 31;
    WarpWindow win;
    win.reset(((g0 < g1 ? P.cell[g0 << 2] : c_first) - 1) & P.mask);  // the same address in every lane
    typename std::conditional<Tr::energy, BinWindow3, BinWindow>::type bw;
    bw.begin(0);
    BinSample bs;
    // adds this lane's binned sample of one particle (weight q) through the warp's bin window
    auto bin_add = [&](int32_t q) {
        if constexpr (Tr::energy)
            bw.add(bs.b, q, bs.mq, bs.eq, bs.tq, bsn, bsm, bse);
        else
            bw.add(bs.b, q, bs.mq, bs.tq, bsn, bsm);
    };
    PSAccW acc;
    PSAcc2 acc2;  // hat rows
    acc.reset();
    acc2.reset();
    bool ovf = false;

    int4* cell4 = reinterpret_cast<int4*>(P.cell);
    float4* th4 = reinterpret_cast<float4*>(P.theta);
    float4* v4 = reinterpret_cast<float4*>(P.v);
    const float4* w4 = reinterpret_cast<const float4*>(P.w);
    // one 16-byte group (four particles) per lane per iteration: a single inlined copy of the
    // particle step keeps the kernel small enough for the instruction cache. The loop bound is
    // the same for the whole warp (the deposit and sample windows are warp-uniform); lanes past
    // the end of the slice process nothing. Each lane's next group is copied to shared memory
    // (cp.async) while the current one is processed, so the streams' latency overlaps the work;
    // a slot is refilled one iteration after it was read (its values long in registers).
    auto fetch = [&](int64_t g, uint32_t slot) {
        cp_async16(slot, cell4 + g);
        cp_async16(slot + 512u, th4 + g);
        if (kNeedV) cp_async16(slot + 1024u, v4 + g);
        cp_async16(slot + 1536u, w4 + g);
    };
    if (Tr::stage) {
        if (g0 + lane < g1) fetch(g0 + lane, stage);
        cp_async_commit();
    }
    uint32_t it = 0;
    for (int64_t gs = g0; gs < g1; gs += 32, ++it) {
        const int64_t g = gs + lane;
        const bool act = g < g1;
        int4 ca = make_int4(0, 0, 0, 0);
        float4 ta = make_float4(0.f, 0.f, 0.f, 0.f), va = ta, wa = ta;
        if (Tr::stage) {
            const uint32_t cur = stage + (it & 1u) * (uint32_t)kStageSlotBytes;
            cp_async_wait_all();
            if (act) {
                ca = lds_i4(cur);
                ta = lds_f4(cur + 512u);
                if (kNeedV) va = lds_f4(cur + 1024u);
                wa = lds_f4(cur + 1536u);
            }
            if (g + 32 < g1) fetch(g + 32, stage + ((it + 1u) & 1u) * (uint32_t)kStageSlotBytes);
            cp_async_commit();
        } else if (act) {
            ca = cell4[g];
            ta = th4[g];
            if (kNeedV) va = v4[g];
            wa = __ldg(w4 + g);
        }
        int4 co;
        float4 to, vo, wo;
        int32_t q0, q1, q2, q3;
        const bool e0 = process<MODE, WALLS>(P, ft, act, ca.x, ta.x, va.x, wa.x, bs, gsn, gsm, gse, gps, acc, acc2, &ovf, co.x,
                                             to.x, vo.x, wo.x, q0);
        if (kBin) {  // the group's bin window starts at the lowest bin of the lanes' first particles
            bw.begin(warp_low_bin(bs.b, bs.ok, P.ncell >> P.bin_shift));
            if (bs.ok) bin_add(q0);
        }
        const bool e1 = process<MODE, WALLS>(P, ft, act, ca.y, ta.y, va.y, wa.y, bs, gsn, gsm, gse, gps, acc, acc2, &ovf, co.y,
                                             to.y, vo.y, wo.y, q1);
        if (kBin && bs.ok) bin_add(q1);
        const bool e2 = process<MODE, WALLS>(P, ft, act, ca.z, ta.z, va.z, wa.z, bs, gsn, gsm, gse, gps, acc, acc2, &ovf, co.z,
                                             to.z, vo.z, wo.z, q2);
        if (kBin && bs.ok) bin_add(q2);
        const bool e3 = process<MODE, WALLS>(P, ft, act, ca.w, ta.w, va.w, wa.w, bs, gsn, gsm, gse, gps, acc, acc2, &ovf, co.w,
                                             to.w, vo.w, wo.w, q3);
        if (kBin && bs.ok) bin_add(q3);
        if (kWrite && act) {
            cell4[g] = co;
            th4[g] = to;
            v4[g] = vo;
            if (WALLS && (wo.x != wa.x || wo.y != wa.y || wo.z != wa.z || wo.w != wa.w))
                reinterpret_cast<float4*>(P.w_out)[g] = wo;  // an absorption in this group
        }
        if (kPS) {  // one warp-aggregated add per group of four particles per lane
            if (Tr::tent) {
                ps_add_warp2(gps, acc2.key, acc2.w, acc2.r);
                acc2.reset();
            } else {
                ps_add_warp_w(gps, acc.key, acc.w);
                acc.reset();
            }
        }
        if constexpr (kBin && Tr::energy)
            bw.end(bsn, bsm, bse);
        else if constexpr (kBin)
            bw.end(bsn, bsm);
        if (kRho) deposit_group(win, grho, P.ncell, P.mask, co, to, q0, q1, q2, q3, e0, e1, e2, e3);
    }
    if (kRho) win.flush_first(grho, 4);
    for (int64_t i = (gb1 << 2) + threadIdx.x; i < end; i += blockDim.x) {  // ragged tail (< 4 particles)
        int co;
        float to, vo, wo;
        int32_t q;
        const float vi = kNeedV ? P.v[i] : 0.f;
        const float wi = P.w[i];
        const bool e = process<MODE, WALLS>(P, ft, true, P.cell[i], P.theta[i], vi, wi, bs, gsn, gsm, gse, gps, acc, acc2, &ovf, co,
                                            to, vo, wo, q);
        if (kWrite) {
            P.cell[i] = co;
            P.theta[i] = to;
            P.v[i] = vo;
            if (WALLS && wo != wi) P.w_out[i] = wo;
        }
        if (kPS) {
            if (Tr::tent) {
                ps_add_warp2(gps, acc2.key, acc2.w, acc2.r);
                acc2.reset();
            } else {
                ps_add_warp_w(gps, acc.key, acc.w);
                acc.reset();
            }
        }
        if (kBin && bs.ok) {  // straight to the grids
            bsn.add_whole(bs.b, q);
            bsm.add_whole(bs.b, bs.mq);
            if (Tr::energy) bse.add_whole(bs.b, bs.eq);
            if (bs.tq) {
                bsn.add_transfer(bs.b, (long long)q * (long long)bs.tq);
                bsm.add_transfer(bs.b, (long long)bs.mq * (long long)bs.tq);
                if (Tr::energy) bse.add_transfer(bs.b, (long long)bs.eq * (long long)bs.tq);
            }
        }
        if (kRho && e) deposit_direct(grho, co, to, q, P.mask);
    }
    if (ovf) raise_flag(P.status, PE_FLAG_OVERFLOW);
    __syncthreads();
    if (kRho) grho.flush();
    if (kSamp) {
        gsn.flush();
        gsm.flush();
        if (Tr::energy) gse.flush();
    }
    if (kBin) {
        if (Tr::energy) bse.flush();
        bsn.flush();
        bsm.flush();
    }
    if (kPS) gps.flush();
}

// WALLS: bounded grid (a separate instantiation, so that periodic launches carry no wall code)
// Resident blocks per SM the register budget is set for (the phase-space passes hold a larger
// shared-memory window and more registers).
template <int MODE>
constexpr int min_blocks()
{
    return (ModeTraits<MODE>::ps || (ModeTraits<MODE>::energy && !ModeTraits<MODE>::binned)) ? 3 : 4;
}

template <int MODE, bool WALLS>
__global__ void __launch_bounds__(kThreads, min_blocks<MODE>()) k_particles(PushParams P)
{
    extern __shared__ uint32_t smem[];
    int64_t begin, end;
    block_chunk(P.n, P.chunk, &begin, &end);
    particle_chunk<MODE, WALLS>(P, begin, end, smem);
}

// Work item of a batched launch: particles [begin, end) of realisation r.
struct WorkItem {
    int64_t begin, end;
    int r, pad;
};

// Persistent batched launch over the work items of many realisations: each block takes
// the next item from a global counter until none are left. Step p and the kick are the
// same for every realisation; tau and the sample row follow from each descriptor.
// Blocks of 128, 256 or 512 threads (the tuner's choice), at the register budget of 1024 threads
// per SM; priv = 0 sends every deposit straight to the global grid (no shared-memory window).
template <int MODE>
__global__ void __launch_bounds__(512, 2) k_particles_batch(const PushParams* descs, const WorkItem* items,
                                                           int nitems, int p, float kick, unsigned* counter, int priv)
{
    extern __shared__ uint32_t smem[];
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = next;
        __syncthreads();
        if (it >= nitems) break;
        const WorkItem wi = items[it];
        PushParams P = descs[wi.r];
        P.kick = kick;
        if (!priv) P.rho_width = 0;
        const float tau = P.comoving ? (float)(P.dT - p * P.dt) : 0.f;
        P.tau_dx = tau * P.inv_dx;
        P.qm_tau = P.qm * tau;
        if (ModeTraits<MODE>::sample) {
            P.samp_n = P.samp_base + (int64_t)p * P.row_stride;
            P.samp_m = P.samp_n + (P.ncell >> P.bin_shift);
        }
        if (P.walls)  // per realisation: uniform in the block
            particle_chunk<MODE, true>(P, wi.begin, wi.end, smem);
        else
            particle_chunk<MODE, false>(P, wi.begin, wi.end, smem);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ quiet start

struct LoadParams {
    int64_t first;  // global storage slot of local particle 0 (a slice of the point set)
    int log2ppc;    // >= 0 when ppc is a power of two: cells store their particles by velocity quantile
    int32_t* cell;
    float* theta;
    float* v;
    float* w;
    int64_t n;
    int64_t chunk;
    uint32_t ppc;
    int ncell, mask;
    float inv_ppc, two_ppc, inv_two_ppc;
    const float* prof_n;
    const float* prof_u;
    const float* prof_t;  // THERMAL loads: nodal temperature (velocity variance), linear in X
    float v_th, wscale;
    uint32_t half, shift;
    unsigned long long* rho;
    int rho_width;
    uint32_t* status;
};

template <bool THERMAL>
__device__ __forceinline__ void load_one(const LoadParams& P, uint32_t i, int& c, float& th, float& vv, float& ww)
{
    // Storage slot i holds Hammersley point h. With ppc = 2^m the cell's slots are filled
    // in ascending order of the velocity quantile: slot k of a cell takes the point whose
    // in-cell index is the m-bit reversal of k (the same point set, permuted in the cell).
    if (P.log2ppc > 0) {
        const uint32_t k = i & (P.ppc - 1u);
        i = (i & ~(P.ppc - 1u)) | (__brev(k) >> (32 - P.log2ppc));
    }
    uint32_t j;
    if (P.log2ppc >= 0) {  // ppc = 2^m: shifts, and theta scaled by the exact 1 / (2 ppc)
        j = i & (P.ppc - 1u);
        c = (int)(i >> P.log2ppc);
        th = (float)(2u * j + 1u) * P.inv_two_ppc;
    } else {
        j = i % P.ppc;
        c = (int)(i / P.ppc);
        th = __fdiv_rn((float)(2u * j + 1u), P.two_ppc);
    }
    const int c1 = (c + 1) & P.mask;
    const float n0 = __ldg(P.prof_n + c), n1 = __ldg(P.prof_n + c1);
    const float u0 = __ldg(P.prof_u + c), u1 = __ldg(P.prof_u + c1);
    const float nX = fmaf(th, n1 - n0, n0);
    const float uX = fmaf(th, u1 - u0, u0);
    ww = nX * P.inv_ppc;
    // Hammersley second coordinate (radical inverse in base 2) with a Cranley-Patterson shift
    const uint32_t Bi = __brev(i) + P.half + P.shift;
    const bool upper = (Bi & 0x80000000u) != 0u;
    const uint32_t bs = upper ? ~Bi : Bi;  // distance to the nearer end of (0, 1), in 2^-32 units
    const float b = fmaf(__uint2float_rn(bs), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float z = normcdfinvf(b);
    float vt = P.v_th;
    if (THERMAL) {  // Section 3.2: a Maxwellian of the local temperature T(X)
        const float t0 = __ldg(P.prof_t + c), t1 = __ldg(P.prof_t + c1);
        vt = sqrtf(fmaf(th, t1 - t0, t0));
    }
    vv = fmaf(vt, upper ? -z : z, uX);
}

template <bool THERMAL>
__global__ void __launch_bounds__(256) k_quiet_start(LoadParams P)
{
    extern __shared__ uint32_t smem[];
    int64_t begin, end;
    block_chunk(P.n, P.chunk, &begin, &end);  // local slots; global slot = P.first + local
    const bool dep = P.rho != nullptr;
    const int c_first = (begin < end) ? (int)((uint64_t)(P.first + begin) / P.ppc) : 0;
    SmemGrid grho{};
    if (dep) {
        grho.bind(smem, P.rho, P.rho_width < P.ncell ? ((c_first - 64) & P.mask) : 0, P.rho_width, P.mask);
        grho.zero();
    }
    __syncthreads();

    const int64_t gb0 = begin >> 2, gb1 = end >> 2;
    int64_t g0, g1;
    warp_groups(gb0, gb1, &g0, &g1);
    LaneWindow lw;
    lw.reset(((int)((uint64_t)(P.first + (g0 << 2)) / P.ppc) - 1) & P.mask);
    bool ovf = false;
    int4* cell4 = reinterpret_cast<int4*>(P.cell);
    float4* th4 = reinterpret_cast<float4*>(P.theta);
    float4* v4 = reinterpret_cast<float4*>(P.v);
    float4* w4 = reinterpret_cast<float4*>(P.w);
    for (int64_t g = g0 + (threadIdx.x & 31); g < g1; g += 32) {
        int4 c;
        float4 t, vv, ww;
        const uint32_t i0 = (uint32_t)(P.first + (g << 2));
        load_one<THERMAL>(P, i0, c.x, t.x, vv.x, ww.x);
        load_one<THERMAL>(P, i0 + 1, c.y, t.y, vv.y, ww.y);
        load_one<THERMAL>(P, i0 + 2, c.z, t.z, vv.z, ww.z);
        load_one<THERMAL>(P, i0 + 3, c.w, t.w, vv.w, ww.w);
        cell4[g] = c;
        th4[g] = t;
        v4[g] = vv;
        w4[g] = ww;
        if (dep) {
            lw.add(c.x, fx_split(fx_weight(ww.x, P.wscale, &ovf), t.x), grho);
            lw.add(c.y, fx_split(fx_weight(ww.y, P.wscale, &ovf), t.y), grho);
            lw.add(c.z, fx_split(fx_weight(ww.z, P.wscale, &ovf), t.z), grho);
            lw.add(c.w, fx_split(fx_weight(ww.w, P.wscale, &ovf), t.w), grho);
        }
    }
    for (int64_t i = (gb1 << 2) + threadIdx.x; i < end; i += blockDim.x) {
        int c;
        float t, vv, ww;
        load_one<THERMAL>(P, (uint32_t)(P.first + i), c, t, vv, ww);
        P.cell[i] = c;
        P.theta[i] = t;
        P.v[i] = vv;
        P.w[i] = ww;
        if (dep) lw.add(c, fx_split(fx_weight(ww, P.wscale, &ovf), t), grho);
    }
    if (dep) lw.flush(grho);
    if (ovf) raise_flag(P.status, PE_FLAG_OVERFLOW);
    __syncthreads();
    if (dep) grho.flush();
}

// ------------------------------------------------------------------ equal-weight loading
// (cumulative-mass table, positions and storage order: pe_eq.cuh)

struct EqParams {
    int32_t* cell;
    float* theta;
    float* v;
    float* w;
    int64_t n;
    int64_t chunk;
    int ncell, mask;
    float wall_factor;
    const float* prof_n;
    const float* prof_u;
    EqTable tab;
    float v_th, wscale;
    uint32_t half, shift;
    unsigned long long* rho;
    int rho_width;
    uint32_t* status;
};

__device__ __forceinline__ void eq_one(const EqParams& P, uint32_t i, int& c, float& th, float& vv, float& ww,
                                         EqCellCache& cache)
{
    const float t = eq_position(P.tab, P.prof_n, P.wall_factor, P.ncell, i, c, cache);
    th = t;
    const float u0 = __ldg(P.prof_u + c), u1 = __ldg(P.prof_u + c + 1);
    const float uX = fmaf(t, u1 - u0, u0);
    ww = (float)__ldg(P.tab.MoN);
    const uint32_t Bi = __brev(i) + P.half + P.shift;
    const bool upper = (Bi & 0x80000000u) != 0u;
    const uint32_t bs = upper ? ~Bi : Bi;
    const float b = fmaf(__uint2float_rn(bs), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float z = normcdfinvf(b);
    vv = fmaf(P.v_th, upper ? -z : z, uX);
}

__global__ void __launch_bounds__(256) k_quiet_start_equal(EqParams P)
{
    extern __shared__ uint32_t smem[];
    int64_t begin, end;
    block_chunk(P.n, P.chunk, &begin, &end);
    const bool dep = P.rho != nullptr;
    const int c_first = (begin < end) ? eq_cell_of(P.tab, P.ncell, eq_point_of_slot((uint32_t)begin, P.n)) : 0;
    SmemGrid grho{};
    if (dep) {
        grho.bind(smem, P.rho, P.rho_width < P.ncell ? ((c_first - 64) & P.mask) : 0, P.rho_width, P.mask);
        grho.zero();
    }
    __syncthreads();

    const int64_t gb0 = begin >> 2, gb1 = end >> 2;
    int64_t g0, g1;
    warp_groups(gb0, gb1, &g0, &g1);
    LaneWindow lw;
    lw.reset((c_first - 1) & P.mask);
    EqCellCache cache;
    cache.reset();
    bool ovf = false;
    int4* cell4 = reinterpret_cast<int4*>(P.cell);
    float4* th4 = reinterpret_cast<float4*>(P.theta);
    float4* v4 = reinterpret_cast<float4*>(P.v);
    float4* w4 = reinterpret_cast<float4*>(P.w);
    for (int64_t g = g0 + (threadIdx.x & 31); g < g1; g += 32) {
        int4 c;
        float4 t, vv, ww;
        const uint32_t s0 = (uint32_t)(g << 2);
        const uint32_t p0 = eq_point_of_slot(s0, P.n), p1 = eq_point_of_slot(s0 + 1, P.n),
                       p2 = eq_point_of_slot(s0 + 2, P.n), p3 = eq_point_of_slot(s0 + 3, P.n);
        // the four points lie within one block; search from the smallest
        const uint32_t pmin = min(min(p0, p1), min(p2, p3));
        const int cb = eq_cell_of(P.tab, P.ncell, pmin);
        c.x = c.y = c.z = c.w = cb;
        eq_one(P, p0, c.x, t.x, vv.x, ww.x, cache);
        eq_one(P, p1, c.y, t.y, vv.y, ww.y, cache);
        eq_one(P, p2, c.z, t.z, vv.z, ww.z, cache);
        eq_one(P, p3, c.w, t.w, vv.w, ww.w, cache);
        cell4[g] = c;
        th4[g] = t;
        v4[g] = vv;
        w4[g] = ww;
        if (dep) {
            lw.add(c.x, fx_split(fx_weight(ww.x, P.wscale, &ovf), t.x), grho);
            lw.add(c.y, fx_split(fx_weight(ww.y, P.wscale, &ovf), t.y), grho);
            lw.add(c.z, fx_split(fx_weight(ww.z, P.wscale, &ovf), t.z), grho);
            lw.add(c.w, fx_split(fx_weight(ww.w, P.wscale, &ovf), t.w), grho);
        }
    }
    for (int64_t i = (gb1 << 2) + threadIdx.x; i < end; i += blockDim.x) {
        const uint32_t pi = eq_point_of_slot((uint32_t)i, P.n);
        int c = eq_cell_of(P.tab, P.ncell, pi);
        float t, vv, ww;
        eq_one(P, pi, c, t, vv, ww, cache);
        P.cell[i] = c;
        P.theta[i] = t;
        P.v[i] = vv;
        P.w[i] = ww;
        if (dep) lw.add(c, fx_split(fx_weight(ww, P.wscale, &ovf), t), grho);
    }
    if (dep) lw.flush(grho);
    if (ovf) raise_flag(P.status, PE_FLAG_OVERFLOW);
    __syncthreads();
    if (dep) grho.flush();
}

// ------------------------------------------------------------------ counting sort

__device__ __forceinline__ void warp_count(unsigned* hist, int c)
{
    const unsigned peers = __match_any_sync(__activemask(), c);
    const int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader) atomicAdd(&hist[c], (unsigned)__popc(peers));
}

__global__ void __launch_bounds__(512) k_sort_count(const int32_t* cell, int64_t n, int64_t chunk, int ncell,
                                                    unsigned* counts, uint32_t* status)
{
    extern __shared__ unsigned hist[];
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    int64_t begin, end;
    block_chunk(n, chunk, &begin, &end);
    for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
        int c = cell[i];
        if ((unsigned)c >= (unsigned)ncell) {
            raise_flag(status, PE_FLAG_RANGE);
            c = 0;  // keep the particle (it is copied, and flagged)
        }
        warp_count(hist, c);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ncell; i += blockDim.x)
        if (hist[i]) atomicAdd(&counts[i], hist[i]);
}

// Exclusive scan of counts[ncell] into cursor[ncell]; one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_sort_scan(const unsigned* counts, unsigned* cursor, int ncell)
{
    __shared__ unsigned part[1024];
    const int per = (ncell + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per;
    unsigned s = 0;
    for (int i = lo; i < lo + per && i < ncell; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // Hillis-Steele inclusive scan
        unsigned t = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    unsigned run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int i = lo; i < lo + per && i < ncell; ++i) {
        cursor[i] = run;
        run += counts[i];
    }
}

__global__ void __launch_bounds__(512) k_sort_scatter(const int32_t* cell, const float* theta, const float* v,
                                                      const float* w, int64_t n, int64_t chunk, int ncell,
                                                      unsigned* cursor, int32_t* oc, float* ot, float* ov,
                                                      float* ow)
{
    extern __shared__ unsigned sh[];
    unsigned* hist = sh;          // count of this block's particles per cell
    unsigned* base = sh + ncell;  // first output slot of this block per cell
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    int64_t begin, end;
    block_chunk(n, chunk, &begin, &end);
    for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
        int c = cell[i];
        if ((unsigned)c >= (unsigned)ncell) c = 0;
        warp_count(hist, c);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
        unsigned h = hist[i];
        base[i] = h ? atomicAdd(&cursor[i], h) : 0u;
        hist[i] = 0u;
    }
    __syncthreads();
    for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
        int c = cell[i];
        if ((unsigned)c >= (unsigned)ncell) c = 0;
        const unsigned peers = __match_any_sync(__activemask(), c);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        unsigned first = 0;
        if (lane == leader) first = atomicAdd(&hist[c], (unsigned)__popc(peers));
        first = __shfl_sync(peers, first, leader);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        const int64_t dst = (int64_t)base[c] + first + rank;
        oc[dst] = cell[i];
        ot[dst] = theta[i];
        ov[dst] = v[i];
        ow[dst] = w[i];
    }
}

// Counter storage of pe_sort_noalloc: counts[ncell] and cursor[ncell] for grids of up to
// PE_SORT_STATIC_MAX_CELLS cells (plus 64 spare words), resident on every device that
// loads the library. Host code must not pass this symbol itself to a kernel: it is a
// host-side stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned g_sort_static[2 * PE_SORT_STATIC_MAX_CELLS + 64];

// ------------------------------------------------------------------ host side

// Grid of a particle pass: one chunk of particles per block, as many blocks as are resident
// at once (one wave). When the chunk cap (which keeps the shared-memory digit counters exact)
// forces more blocks than that, the chunk is shrunk so that the blocks fill whole waves: a
// last wave holding a few full-size blocks would leave most SMs idle while it runs.
int particle_grid(const void* kernel, int block, size_t smem, int64_t n, int64_t* chunk, int64_t max_chunk)
{
    const int64_t slots = (int64_t)sm_count() * blocks_per_sm(kernel, block, smem);
    const int64_t cap = (max_chunk > 0 && max_chunk < kMaxChunk) ? (max_chunk & ~int64_t(3)) : kMaxChunk;
    const int64_t waves = (n + slots * cap - 1) / (slots * cap);
    const int64_t blocks = slots * (waves < 1 ? 1 : waves);
    int64_t c = (n + blocks - 1) / blocks;
    c = (c + 3) & ~int64_t(3);
    if (c < 4) c = 4;
    if (c > cap) c = cap;
    *chunk = c;
    int64_t g = (n + c - 1) / c;
    return (int)(g < 1 ? 1 : g);
}

// Rows of the block-private phase-space window: up to kPSWindowBins, halved while the window
// (three 32-bit digit counters per cell) would exceed 24 KB, so that three blocks and their
// staging slots fit on an SM (targets outside the window go to the global histogram).
static int ps_window_rows(int nxc, int nv)
{
    int w = nxc <= kPSWindowBins ? nxc : kPSWindowBins;
    while (w > 1 && (size_t)3 * sizeof(uint32_t) * (size_t)w * (size_t)nv > 24 * 1024) w >>= 1;
    return w;
}

// Shared memory of a particle pass: the grids (smem bytes), rounded up to 16 bytes, then the
// staging slots of the block's warps (passes that stage their streams).
static size_t with_stage(size_t smem, int block, bool staged)
{
    return staged ? ((smem + 15) & ~size_t(15)) + (size_t)(block / 32) * kStageWarpBytes : smem;
}

template <int MODE>
static int launch_particles(PushParams& P, cudaStream_t s, bool zero = true)
{
    const int block = kThreads;
    const bool rho = ModeTraits<MODE>::rho;
    const bool samp = ModeTraits<MODE>::sample;
    const bool bin = ModeTraits<MODE>::binned;
    // charge window: 64 nodes before the chunk's first cell, then the chunk's cells at a uniform
    // density (chunks of <= 65536 particles) twice over; no wider than needed, so that the shared
    // memory left to L1 stays large (the streaming loads' in-flight capacity)
    if (rho) {
        const int64_t span = (int64_t)65536 * P.ncell / (P.n > 0 ? P.n : 1) + 1;
        int w = 128;
        while (w < 128 + 2 * span && w < kRhoWindowNodes) w <<= 1;
        P.rho_width = P.ncell <= w ? P.ncell : w;
    } else {
        P.rho_width = 0;
    }
    P.samp_width = (samp && !bin) ? (P.ncell <= kWindowNodes ? P.ncell : kWindowNodes) : 0;
    // three nodal moments: a narrower window (co-moving targets beyond it go to the global rows),
    // so that three blocks fit on an SM
    if (ModeTraits<MODE>::energy && !bin) P.samp_width = P.ncell <= kWindowNodesE ? P.ncell : kWindowNodesE;
    const int nb = bin ? (P.ncell >> P.bin_shift) : 0;
    const bool ps = ModeTraits<MODE>::ps;
    const int nxc = P.ncell >> P.bin_shift;
    P.ps_width = ps ? ps_window_rows(nxc, P.nv) : 0;
    if (ps) P.samp_width = 0;
    const size_t tab = MODE == kDeposit ? 0 : (samp ? sizeof(float4) : sizeof(float2)) * (size_t)kFieldTabNodes;
    const int nmom = ModeTraits<MODE>::energy ? 3 : 2;
    size_t smem = tab + kSmemGridWords * sizeof(uint32_t) * (size_t)(P.rho_width + nmom * P.samp_width) +
                  kBinGridWords * sizeof(uint32_t) * (size_t)nmom * nb +
                  3 * sizeof(uint32_t) * (size_t)P.ps_width * (size_t)P.nv;
    smem = with_stage(smem, block, ModeTraits<MODE>::stage);
    if (smem > (size_t)max_smem_optin()) return PE_EINVAL;
    const void* k = P.walls ? (const void*)k_particles<MODE, true> : (const void*)k_particles<MODE, false>;
    if (ensure_smem(k, smem) != PE_OK) return PE_ECUDA;
    int grid = particle_grid(k, block, smem, P.n, &P.chunk, P.max_chunk);
    // the pass accumulates into a zeroed charge grid and sample row (zeroed by the caller when !zero)
    if (zero && rho && cudaMemsetAsync(P.rho, 0, sizeof(int64_t) * (size_t)P.ncell, s) != cudaSuccess)
        return PE_ECUDA;
    const size_t samp_words = ps ? (size_t)nxc * (size_t)P.nv : (size_t)nmom * (size_t)(P.ncell >> P.bin_shift);
    if (zero && samp && cudaMemsetAsync(P.samp_n, 0, sizeof(int64_t) * samp_words, s) != cudaSuccess)
        return PE_ECUDA;
    if (P.n == 0) return PE_OK;
    if (P.walls)
        k_particles<MODE, true><<<grid, block, smem, s>>>(P);
    else
        k_particles<MODE, false><<<grid, block, smem, s>>>(P);
    return launch_status();
}

static bool particles_ok(const void* a, const void* b, const void* c, const void* d, int64_t n)
{
    if (n < 0 || n > (int64_t(1) << 32)) return false;
    if (n == 0) return true;
    return a && b && c && d && aligned16(a) && aligned16(b) && aligned16(c) && aligned16(d);
}

static bool sample_ok(const pe_sample_args* s, int ncell)
{
    if (!s || !s->E0f || !s->sample_fx || !aligned16(s->sample_fx)) return false;
    if (s->boundary != PE_BOUNDARY_PERIODIC && s->boundary != PE_BOUNDARY_ABSORBING) return false;
    if (s->bin_shift < 0 || (1 << s->bin_shift) > ncell) return false;
    if (s->n_v < 0 || s->n_v > 1024) return false;
    if (s->second_moment != 0 && (s->second_moment != 1 || s->n_v != 0 || s->boundary != PE_BOUNDARY_PERIODIC ||
                                  s->s_e < -64 || s->s_e > 64))
        return false;
    if (s->x_tent != 0 && (s->x_tent != 1 || s->n_v <= 0 || s->boundary != PE_BOUNDARY_PERIODIC)) return false;
    if (s->n_v > 0 && (ncell >> s->bin_shift) > 32767) return false;  // phase-space keys pack (row << 16) | cell
    if (s->n_v > 0) {
        const int nxc = ncell >> s->bin_shift;
        const size_t w = (size_t)ps_window_rows(nxc, s->n_v);
        return s->inv_dv > 0.0f && 3 * sizeof(uint32_t) * w * (size_t)s->n_v <= 160 * 1024;
    }
    if (s->bin_shift == 0) return true;
    const size_t nmom = s->second_moment ? 3 : 2;
    return (kBinGridWords * nmom * (size_t)(ncell >> s->bin_shift)) * sizeof(uint32_t) <= 96 * 1024;  // bins fit in shared memory
}

// ------------------------------------------------------------------ batched launches

size_t push_desc_size() { return sizeof(PushParams); }
size_t work_item_size() { return sizeof(WorkItem); }

void make_push_desc(void* out, int32_t* cell, float* theta, float* v, const float* w, int64_t n, const float* Ef,
                    int ncell, float dt_dx, float qm_dt, int s_w, int64_t* rho, const float* E0f, double dT, double dt,
                    float inv_dx, float qm, int comoving, int s_p, int bin_shift, int64_t* samp_base,
                    int64_t row_stride, int walls, uint32_t* status)
{
    PushParams P{};
    P.cell = cell;
    P.theta = theta;
    P.v = v;
    P.w = w;
    P.walls = walls ? 1 : 0;
    P.w_out = const_cast<float*>(w);  // written only for absorbed ions of a bounded grid
    P.n = n;
    P.Ef = Ef;
    P.ncell = ncell;
    P.mask = ncell - 1;
    P.dt_dx = dt_dx;
    P.qm_dt = qm_dt;
    P.wscale = ldexpf(1.0f, s_w);
    P.rho = reinterpret_cast<unsigned long long*>(rho);
    P.rho_width = ncell <= kRhoWindowNodes ? ncell : kRhoWindowNodes;
    P.E0f = E0f;
    P.pscale = ldexpf(1.0f, s_p);
    P.samp_width = 0;
    P.bin_shift = bin_shift;
    P.status = status;
    P.dT = dT;
    P.dt = dt;
    P.inv_dx = inv_dx;
    P.qm = qm;
    P.comoving = comoving;
    P.samp_base = reinterpret_cast<unsigned long long*>(samp_base);
    P.row_stride = row_stride;
    memcpy(out, &P, sizeof(P));
}

void make_work_item(void* out, int r, int64_t begin, int64_t end)
{
    WorkItem wi{begin, end, r, 0};
    memcpy(out, &wi, sizeof(wi));
}

// Shared memory of a batched launch: the field table, the deposit window (priv), the bins.
static size_t batch_smem(int mode, int max_ncell, int max_nb, int priv, int block)
{
    const int rw = (mode != 1 && priv) ? (max_ncell <= kRhoWindowNodes ? max_ncell : kRhoWindowNodes) : 0;
    return with_stage((mode == 2 ? 0 : sizeof(float4) * (size_t)kFieldTabNodes) +
                          kSmemGridWords * sizeof(uint32_t) * (size_t)rw +
                          (mode == 2 ? 0 : kBinGridWords * sizeof(uint32_t) * 2 * (size_t)max_nb),
                      block, mode == 2);
}

template <int MODE>
static int launch_batch_mode(const void* descs, const void* items, int nitems, int p, float kick, unsigned* counter,
                             size_t smem, int block, int priv, cudaStream_t s)
{
    const void* k = (const void*)k_particles_batch<MODE>;
    if (ensure_smem(k, smem) != PE_OK) return PE_ECUDA;
    const int grid = sm_count() * blocks_per_sm(k, block, smem);
    k_particles_batch<MODE><<<grid, block, smem, s>>>(static_cast<const PushParams*>(descs),
                                                      static_cast<const WorkItem*>(items), nitems, p, kick, counter,
                                                      priv);
    return launch_status();
}

// mode 0: fused push + binned sample of step p; mode 1: binned sample only; mode 2: charge
// deposit only (the tuner's probe of the deposit path). block: 128, 256 or 512 threads.
int launch_particles_batch(int mode, const void* descs, const void* items, int nitems, int p, float kick,
                           unsigned* counter, int max_ncell, int max_nb, int block, int priv, cudaStream_t s)
{
    if (block != 128 && block != 256 && block != 512) return PE_EINVAL;
    const size_t smem = batch_smem(mode, max_ncell, max_nb, priv, block);
    if (smem > (size_t)max_smem_optin()) return PE_EINVAL;
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned), s) != cudaSuccess) return PE_ECUDA;
    if (mode == 0) return launch_batch_mode<kPushSampleBinned>(descs, items, nitems, p, kick, counter, smem, block, priv, s);
    if (mode == 1) return launch_batch_mode<kSampleBinned>(descs, items, nitems, p, kick, counter, smem, block, priv, s);
    return launch_batch_mode<kDeposit>(descs, items, nitems, p, kick, counter, smem, block, priv, s);
}

}  // namespace pe

using namespace pe;

extern "C" PE_API int pe_deposit(const int32_t* cell, const float* theta, const float* w, int64_t n, int32_t ncell,
                                 int32_t s_w, int64_t* rho_fx, uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !rho_fx || !particles_ok(cell, theta, w, w, n)) return PE_EINVAL;
    PushParams P{};
    P.cell = const_cast<int32_t*>(cell);
    P.theta = const_cast<float*>(theta);
    P.w = w;
    P.n = n;
    P.ncell = ncell;
    P.mask = ncell - 1;
    P.wscale = ldexpf(1.0f, s_w);
    P.rho = reinterpret_cast<unsigned long long*>(rho_fx);
    P.status = status;
    return launch_particles<kDeposit>(P, (cudaStream_t)stream);
}

namespace pe {

int push_pass(int32_t* cell, float* theta, float* v, float* w, int64_t n, const float* Ef, int32_t ncell,
              float dt_over_dx, float qm_dt, float kick, int32_t s_w, int32_t boundary, int64_t* rho_fx,
              const pe_sample_args* sample, uint32_t* status, void* stream, bool zero)
{
    if (!is_pow2(ncell) || ncell < 8 || !rho_fx || !Ef || !particles_ok(cell, theta, v, w, n)) return PE_EINVAL;
    if (boundary != PE_BOUNDARY_PERIODIC && boundary != PE_BOUNDARY_ABSORBING) return PE_EINVAL;
    if (sample && (!sample_ok(sample, ncell) || sample->s_w != s_w || sample->boundary != boundary)) return PE_EINVAL;
    PushParams P{};
    P.cell = cell;
    P.theta = theta;
    P.v = v;
    P.w = w;
    P.n = n;
    P.Ef = Ef;
    P.ncell = ncell;
    P.mask = ncell - 1;
    P.dt_dx = dt_over_dx;
    P.qm_dt = qm_dt;
    P.kick = kick;
    P.wscale = ldexpf(1.0f, s_w);
    P.rho = reinterpret_cast<unsigned long long*>(rho_fx);
    P.status = status;
    P.walls = boundary == PE_BOUNDARY_ABSORBING;
    P.w_out = w;
    if (sample) {
        P.E0f = sample->E0f;
        P.tau_dx = sample->tau * sample->inv_dx;
        P.qm_tau = sample->qm * sample->tau;
        P.pscale = ldexpf(1.0f, sample->s_p);
        P.bin_shift = sample->bin_shift;
        P.samp_n = reinterpret_cast<unsigned long long*>(sample->sample_fx);
        P.samp_m = P.samp_n + (ncell >> P.bin_shift);
        if (sample->n_v > 0) {
            P.nv = sample->n_v;
            P.vmin = sample->v_min;
            P.inv_dv = sample->inv_dv;
            P.tent_scale = ldexpf(1.0f, 24 - P.bin_shift);
            if (sample->x_tent) return launch_particles<kPushSamplePSW>(P, (cudaStream_t)stream, zero);
            return launch_particles<kPushSamplePS>(P, (cudaStream_t)stream, zero);
        }
        if (sample->second_moment) {  // rows [3][ncell >> bin_shift]
            P.samp_e = P.samp_n + 2 * (size_t)(ncell >> P.bin_shift);
            P.escale = ldexpf(1.0f, sample->s_e);
            if (P.bin_shift > 0) return launch_particles<kPushSampleBinnedE>(P, (cudaStream_t)stream, zero);
            return launch_particles<kPushSampleE>(P, (cudaStream_t)stream, zero);
        }
        if (P.bin_shift > 0) return launch_particles<kPushSampleBinned>(P, (cudaStream_t)stream, zero);
        return launch_particles<kPushSample>(P, (cudaStream_t)stream, zero);
    }
    return launch_particles<kPush>(P, (cudaStream_t)stream, zero);
}

int sample_pass(const int32_t* cell, const float* theta, const float* v, const float* w, int64_t n, const float* Ef,
                int32_t ncell, float qm_dt, float kick, const pe_sample_args* sample, uint32_t* status, void* stream,
                bool zero)
{
    if (!is_pow2(ncell) || ncell < 8 || !Ef || !particles_ok(cell, theta, v, w, n) || !sample_ok(sample, ncell))
        return PE_EINVAL;
    PushParams P{};
    P.walls = sample->boundary == PE_BOUNDARY_ABSORBING;
    P.cell = const_cast<int32_t*>(cell);
    P.theta = const_cast<float*>(theta);
    P.v = const_cast<float*>(v);
    P.w = w;
    P.n = n;
    P.Ef = Ef;
    P.ncell = ncell;
    P.mask = ncell - 1;
    P.qm_dt = qm_dt;
    P.kick = kick;
    P.wscale = ldexpf(1.0f, sample->s_w);
    P.status = status;
    P.E0f = sample->E0f;
    P.tau_dx = sample->tau * sample->inv_dx;
    P.qm_tau = sample->qm * sample->tau;
    P.pscale = ldexpf(1.0f, sample->s_p);
    P.bin_shift = sample->bin_shift;
    P.samp_n = reinterpret_cast<unsigned long long*>(sample->sample_fx);
    P.samp_m = P.samp_n + (ncell >> P.bin_shift);
    if (sample->n_v > 0) {
        P.nv = sample->n_v;
        P.vmin = sample->v_min;
        P.inv_dv = sample->inv_dv;
        P.tent_scale = ldexpf(1.0f, 24 - P.bin_shift);
        if (sample->x_tent) return launch_particles<kSamplePSW>(P, (cudaStream_t)stream, zero);
        return launch_particles<kSamplePS>(P, (cudaStream_t)stream, zero);
    }
    if (sample->second_moment) {  // rows [3][ncell >> bin_shift]
        P.samp_e = P.samp_n + 2 * (size_t)(ncell >> P.bin_shift);
        P.escale = ldexpf(1.0f, sample->s_e);
        if (P.bin_shift > 0) return launch_particles<kSampleBinnedE>(P, (cudaStream_t)stream, zero);
        return launch_particles<kSampleE>(P, (cudaStream_t)stream, zero);
    }
    if (P.bin_shift > 0) return launch_particles<kSampleBinned>(P, (cudaStream_t)stream, zero);
    return launch_particles<kSample>(P, (cudaStream_t)stream, zero);
}

}  // namespace pe

extern "C" PE_API int pe_push_ex(int32_t* cell, float* theta, float* v, float* w, int64_t n, const float* Ef,
                                 int32_t ncell, float dt_over_dx, float qm_dt, float kick, int32_t s_w,
                                 int32_t boundary, int64_t* rho_fx, const pe_sample_args* sample, uint32_t* status,
                                 void* stream)
{
    return push_pass(cell, theta, v, w, n, Ef, ncell, dt_over_dx, qm_dt, kick, s_w, boundary, rho_fx, sample, status,
                     stream, true);
}

extern "C" PE_API int pe_push(int32_t* cell, float* theta, float* v, const float* w, int64_t n, const float* Ef,
                              int32_t ncell, float dt_over_dx, float qm_dt, float kick, int32_t s_w, int64_t* rho_fx,
                              const pe_sample_args* sample, uint32_t* status, void* stream)
{
    if (sample && sample->boundary != PE_BOUNDARY_PERIODIC) return PE_EINVAL;
    // periodic: the weights are only read
    return pe_push_ex(cell, theta, v, const_cast<float*>(w), n, Ef, ncell, dt_over_dx, qm_dt, kick, s_w,
                      PE_BOUNDARY_PERIODIC, rho_fx, sample, status, stream);
}

extern "C" PE_API int pe_sample(const int32_t* cell, const float* theta, const float* v, const float* w, int64_t n,
                                const float* Ef, int32_t ncell, float qm_dt, float kick, const pe_sample_args* sample,
                                uint32_t* status, void* stream)
{
    return sample_pass(cell, theta, v, w, n, Ef, ncell, qm_dt, kick, sample, status, stream, true);
}

// Appendix C's loading of the slots [first, first + n); prof_t != NULL loads at the local
// temperature instead of v_th.
static int quiet_start_launch(int32_t* cell, float* theta, float* v, float* w, int64_t first, int64_t n,
                              int64_t n_total, int32_t ncell, const float* prof_n, const float* prof_u,
                              const float* prof_t, float v_th, uint64_t seed, int32_t s_w, int64_t* rho_fx,
                              uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !prof_n || !prof_u || !particles_ok(cell, theta, v, w, n)) return PE_EINVAL;
    if (n_total % ncell != 0 || n_total == 0 || n_total >= (int64_t(1) << 32)) return PE_EINVAL;
    if (first < 0 || n < 1 || first > n_total - n) return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    LoadParams P{};
    P.first = first;
    P.cell = cell;
    P.theta = theta;
    P.v = v;
    P.w = w;
    P.n = n;
    P.ppc = (uint32_t)(n_total / ncell);
    P.log2ppc = is_pow2(P.ppc) ? ilog2(P.ppc) : -1;
    P.ncell = ncell;
    P.mask = ncell - 1;
    P.inv_ppc = 1.0f / (float)P.ppc;
    P.two_ppc = 2.0f * (float)P.ppc;
    P.inv_two_ppc = 1.0f / P.two_ppc;
    P.prof_n = prof_n;
    P.prof_u = prof_u;
    P.prof_t = prof_t;
    P.v_th = v_th;
    P.wscale = ldexpf(1.0f, s_w);
    P.half = (uint32_t)(2147483648.0 / (double)n_total);
    // splitmix64 (Steele, Lea, Flood 2014) of the seed; its upper half is the shift
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    P.shift = (uint32_t)(z >> 32);
    P.rho = reinterpret_cast<unsigned long long*>(rho_fx);
    P.rho_width = rho_fx ? (ncell <= kRhoWindowNodes ? ncell : kRhoWindowNodes) : 0;
    P.status = status;
    const int block = 256;
    size_t smem = kSmemGridWords * sizeof(uint32_t) * (size_t)P.rho_width;
    const void* k = prof_t ? (const void*)k_quiet_start<true> : (const void*)k_quiet_start<false>;
    if (ensure_smem(k, smem) != PE_OK) return PE_ECUDA;
    int grid = particle_grid(k, block, smem, n, &P.chunk);
    if (rho_fx && cudaMemsetAsync(rho_fx, 0, sizeof(int64_t) * (size_t)ncell, s) != cudaSuccess) return PE_ECUDA;
    if (prof_t)
        k_quiet_start<true><<<grid, block, smem, s>>>(P);
    else
        k_quiet_start<false><<<grid, block, smem, s>>>(P);
    return launch_status();
}

extern "C" PE_API int pe_quiet_start_slice(int32_t* cell, float* theta, float* v, float* w, int64_t first,
                                           int64_t n, int64_t n_total, int32_t ncell, const float* prof_n,
                                           const float* prof_u, float v_th, uint64_t seed, int32_t s_w, int64_t* rho_fx,
                                           uint32_t* status, void* stream)
{
    return quiet_start_launch(cell, theta, v, w, first, n, n_total, ncell, prof_n, prof_u, nullptr, v_th, seed, s_w,
                              rho_fx, status, stream);
}

extern "C" PE_API int pe_quiet_start_thermal(int32_t* cell, float* theta, float* v, float* w, int64_t n,
                                             int32_t ncell, const float* prof_n, const float* prof_u,
                                             const float* prof_T, uint64_t seed, int32_t s_w, int64_t* rho_fx,
                                             uint32_t* status, void* stream)
{
    if (!prof_T) return PE_EINVAL;
    return quiet_start_launch(cell, theta, v, w, 0, n, n, ncell, prof_n, prof_u, prof_T, 0.0f, seed, s_w, rho_fx,
                              status, stream);
}

extern "C" PE_API int pe_quiet_start(int32_t* cell, float* theta, float* v, float* w, int64_t n, int32_t ncell,
                                     const float* prof_n, const float* prof_u, float v_th, uint64_t seed, int32_t s_w,
                                     int64_t* rho_fx, uint32_t* status, void* stream)
{
    return pe_quiet_start_slice(cell, theta, v, w, 0, n, n, ncell, prof_n, prof_u, v_th, seed, s_w, rho_fx, status,
                                stream);
}

extern "C" PE_API int pe_quiet_start_equal(int32_t* cell, float* theta, float* v, float* w, int64_t n, int32_t ncell,
                                           const float* prof_n, const float* prof_u, float wall_factor, float v_th,
                                           uint64_t seed, int32_t s_w, void* scratch, int64_t* rho_fx,
                                           uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !prof_n || !prof_u || !scratch || !particles_ok(cell, theta, v, w, n))
        return PE_EINVAL;
    if (n == 0 || n >= (int64_t(1) << 32) || ((uintptr_t)scratch & 15u) || !(wall_factor >= 0.0f))
        return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int ncl = ncell - 1;
    double* C = static_cast<double*>(scratch);
    long long* first = reinterpret_cast<long long*>(C + ncl + 1);
    double* MoN = reinterpret_cast<double*>(first + ncl + 1);
    k_eq_table<float><<<1, kEqThreads, 0, s>>>(prof_n, ncell, wall_factor, n, C, first, MoN, status);
    EqParams P{};
    P.cell = cell;
    P.theta = theta;
    P.v = v;
    P.w = w;
    P.n = n;
    P.ncell = ncell;
    P.mask = ncell - 1;
    P.wall_factor = wall_factor;
    P.prof_n = prof_n;
    P.prof_u = prof_u;
    P.tab = EqTable{C, first, MoN};
    P.v_th = v_th;
    P.wscale = ldexpf(1.0f, s_w);
    P.half = (uint32_t)(2147483648.0 / (double)n);
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL;  // splitmix64 of the seed: the shift is its upper half
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    P.shift = (uint32_t)(z >> 32);
    P.rho = reinterpret_cast<unsigned long long*>(rho_fx);
    P.rho_width = rho_fx ? (ncell <= kRhoWindowNodes ? ncell : kRhoWindowNodes) : 0;
    P.status = status;
    const int block = 256;
    const size_t smem = kSmemGridWords * sizeof(uint32_t) * (size_t)P.rho_width;
    const void* k = (const void*)k_quiet_start_equal;
    if (ensure_smem(k, smem) != PE_OK) return PE_ECUDA;
    const int grid = particle_grid(k, block, smem, n, &P.chunk);
    if (rho_fx && cudaMemsetAsync(rho_fx, 0, sizeof(int64_t) * (size_t)ncell, s) != cudaSuccess) return PE_ECUDA;
    k_quiet_start_equal<<<grid, block, smem, s>>>(P);
    return launch_status(2);
}

// Device address of g_sort_static in the current context. Looked up on every call (the lookup
// allocates nothing): a cached address could go stale when another context becomes current
// or after cudaDeviceReset reloads the module, and a cache shared by threads would need
// synchronisation.
static unsigned* sort_static_ptr()
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sort_static) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<unsigned*>(p);
}

extern "C" PE_API int pe_sort_noalloc(const int32_t* cell, const float* theta, const float* v, const float* w,
                                      int64_t n, int32_t ncell, int32_t* out_cell, float* out_theta, float* out_v,
                                      float* out_w, uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || ncell > PE_SORT_STATIC_MAX_CELLS) return PE_EINVAL;
    unsigned* scratch = sort_static_ptr();
    if (!scratch) return PE_ECUDA;
    return pe_sort(cell, theta, v, w, n, ncell, out_cell, out_theta, out_v, out_w, reinterpret_cast<int32_t*>(scratch),
                   status, stream);
}

extern "C" PE_API int pe_sort(const int32_t* cell, const float* theta, const float* v, const float* w, int64_t n,
                              int32_t ncell, int32_t* out_cell, float* out_theta, float* out_v, float* out_w,
                              int32_t* scratch, uint32_t* status, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !scratch || !particles_ok(cell, theta, v, w, n) ||
        !particles_ok(out_cell, out_theta, out_v, out_w, n))
        return PE_EINVAL;
    if ((size_t)ncell * 2 * sizeof(unsigned) > (size_t)max_smem_optin()) return PE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* counts = reinterpret_cast<unsigned*>(scratch);
    unsigned* cursor = counts + ncell;
    if (cudaMemsetAsync(counts, 0, sizeof(unsigned) * (size_t)ncell, s) != cudaSuccess) return PE_ECUDA;
    if (n == 0) return PE_OK;
    const int block = 512;
    int64_t chunk = 0;
    size_t smem1 = sizeof(unsigned) * (size_t)ncell, smem2 = 2 * smem1;
    if (ensure_smem((const void*)k_sort_count, smem1) != PE_OK ||
        ensure_smem((const void*)k_sort_scatter, smem2) != PE_OK)
        return PE_ECUDA;
    int grid = particle_grid((const void*)k_sort_scatter, block, smem2, n, &chunk);
    k_sort_count<<<grid, block, smem1, s>>>(cell, n, chunk, ncell, counts, status);
    k_sort_scan<<<1, 1024, 0, s>>>(counts, cursor, ncell);
    k_sort_scatter<<<grid, block, smem2, s>>>(cell, theta, v, w, n, chunk, ncell, cursor, out_cell, out_theta, out_v,
                                              out_w);
    return launch_status(3);
}
