// Blackwell tensor-core GEMM building blocks (sm_100 family, compiled for sm_103a): mbarriers,
// TMA tile loads with the 128-byte swizzle, tcgen05.mma with the accumulator in tensor memory
// (TMEM), and a single-CTA kernel C[M][N] = A[M][K] B[N][K]^T for BF16 operands stored with K
// contiguous, FP32 accumulation, and an epilogue functor applied to each row of the tile.
//
// Tile: 128 rows (the MMA's M) x BN columns (64 or 128) x 64 K per stage (one 128-byte swizzle
// row of BF16), four stages. One thread issues the TMA loads and the MMAs (kind::f16, K = 16
// per instruction, four per stage); a stage is reloaded once the MMAs that read it have
// signalled its empty barrier (tcgen05.commit). After the last MMA the four warps read their
// 32 TMEM lanes (tile rows) 32 columns at a time (tcgen05.ld 32x32b.x32).
//
// Every wait on an mbarrier is bounded by a clock budget (about one second); on expiry the
// kernel sets PE_FLAG_TIMEOUT in the status word, skips the remaining MMAs and the epilogue,
// and still frees its TMEM, so the context stays usable.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pepic.h"

namespace pe {
namespace tc {

constexpr int kBM = 128;       // tile rows = MMA M
constexpr int kBK = 64;        // K per stage: 64 BF16 = one 128-byte swizzle row
constexpr int kStages = 4;
constexpr int kThreads = 128;  // four warps: one per 32 TMEM lanes in the epilogue
constexpr long long kWaitBudget = 2000000000LL;  // clock cycles (about one second)

template <int BN>
struct TileCfg {
    static_assert(BN == 64 || BN == 128, "tile width");
    static constexpr int kABytes = kBM * kBK * 2;
    static constexpr int kBBytes = BN * kBK * 2;
    static constexpr int kStageBytes = kABytes + kBBytes;
    // stages (1024-byte aligned for the swizzle), then 2 kStages + 1 mbarriers and the TMEM slot
    static constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 8 * (2 * kStages + 1) + 16;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; false once the budget is spent.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitBudget) return false;
    return true;
}

// TMA: box {64 (K), rows} of a 2D BF16 tensor map at element (c0 = k, c1 = row) into dst,
// completing `bytes` on bar.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(saddr(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)  // one whole warp
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)  // the allocating warp
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte swizzle layout:
// rows of 128 bytes, groups of 8 rows 1024 bytes apart (stride byte offset), version 1,
// swizzle mode 2 (128 B). The leading byte offset is not used by this layout.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives once on bar when every MMA this thread issued so far has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of TMEM lane (lane base of taddr + thread's lane) into v.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    // the registers are valid only after the wait: tie them to it so no use moves above it
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// C tile (blockIdx.y, blockIdx.x) of A[M][K] B[N][K]^T; ta / tb: tensor maps of A (dims {K, M},
// box {64, 128}) and B (dims {K, N}, box {64, BN}), 128-byte swizzle, zero fill beyond the
// extents (ragged M and K). epi(row, col0, v) receives 32 columns col0.. of one row (the row
// may be >= M: the functor checks); every thread then calls epi.finish() (block-wide
// reductions of the epilogue). N % BN == 0.
template <int BN, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int K, Epi epi,
              uint32_t* status)
{
    using Cfg = TileCfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * Cfg::kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int ktiles = (K + kBK - 1) / kBK;
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);
    (void)M;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        fence_mbar_init();
        s_fail = 0;
    }
    if (warp == 0) tmem_alloc(tmem_slot, BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        auto load = [&](int t) {
            const int s = t % kStages;
            uint8_t* a = smem + s * Cfg::kStageBytes;
            mbar_expect_tx(&full[s], Cfg::kStageBytes);
            tma_load_2d(a, &ta, &full[s], t * kBK, m0);
            tma_load_2d(a + Cfg::kABytes, &tb, &full[s], t * kBK, n0);
        };
        const int pro = ktiles < kStages ? ktiles : kStages;
        for (int t = 0; t < pro; ++t) load(t);
        int issued = pro, consumed = 0;
        bool ok = true;
        for (int kt = 0; kt < ktiles; ++kt) {
            const int s = kt % kStages;
            if (!mbar_wait(&full[s], (uint32_t)((kt / kStages) & 1))) {
                ok = false;
                break;
            }
            consumed = kt + 1;
            tc_fence_after();
            const uint32_t a0 = saddr(smem + s * Cfg::kStageBytes), b0 = a0 + Cfg::kABytes;
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)  // K = 16 per MMA: 32 bytes along the swizzled row
                umma_bf16(tmem, sw128_desc(a0 + 32 * k), sw128_desc(b0 + 32 * k), idesc, (kt | k) ? 1u : 0u);
            umma_commit(&empty[s]);
            // refill the stage of the previous tile once its MMAs are done (this tile's MMAs are queued)
            const int t = kt - 1 + kStages;
            if (kt >= 1 && t < ktiles) {
                if (!mbar_wait(&empty[(kt - 1) % kStages], (uint32_t)(((kt - 1) / kStages) & 1))) {
                    ok = false;
                    break;
                }
                load(t);
                ++issued;
            }
        }
        umma_commit(done);
        if (!ok) {
            s_fail = 1;
            // let the tile loads still in flight land (bounded) before the block may exit
            for (int t = consumed; t < issued; ++t) mbar_wait(&full[t % kStages], (uint32_t)((t / kStages) & 1));
        }
    }
    __syncthreads();
    bool ok = mbar_wait(done, 0u) && !s_fail;
    ok = __all_sync(0xFFFFFFFFu, ok);
    if (!ok && lane == 0) atomicOr(status, PE_FLAG_TIMEOUT);
    tc_fence_after();
    Epi e = epi;
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t t_row = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            float v[32];
            tmem_ld32(t_row + (uint32_t)c, v);
            e(row, n0 + c, v);
        }
    }
    e.finish();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, BN);
}

}  // namespace tc
}  // namespace pe
