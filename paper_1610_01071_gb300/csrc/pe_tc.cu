// Host side of the tensor-core GEMM (pe_tc.cuh): TMA tensor maps of BF16 operands and the
// plain product C = A B^T (FP32 out), the entry point the GEMM tests call.
#include <cudaTypedefs.h>

#include <mutex>

#include "pe_ctx.h"
#include "pe_internal.h"
#include "pe_tc.cuh"

namespace pe {

static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

int tc_operand_map(CUtensorMap* map, const void* base, int64_t rows, int64_t K, int64_t ld, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn) return PE_ECUDA;
    if (!base || ((uintptr_t)base & 15u) || rows < 1 || K < 1 || ld < K || (ld * 2) % 16 != 0) return PE_EINVAL;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)tc::kBK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? PE_OK : PE_EINVAL;
}

namespace {
struct EpiStoreF32 {
    float* C;
    int M;
    int64_t ldc;
    __device__ __forceinline__ void operator()(int row, int col0, const float* v) const
    {
        if (row >= M) return;
        float4* d = reinterpret_cast<float4*>(C + (size_t)row * ldc + col0);
#pragma unroll
        for (int j = 0; j < 8; ++j) d[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
    __device__ __forceinline__ void finish() {}
};

template <int BN>
int launch_plain(const CUtensorMap& ma, const CUtensorMap& mb, int M, int N, int K, EpiStoreF32 epi,
                 uint32_t* status, cudaStream_t s)
{
    const void* k = (const void*)tc::k_tc_gemm<BN, EpiStoreF32>;
    if (ensure_smem(k, tc::TileCfg<BN>::kSmemBytes) != PE_OK) return PE_ECUDA;
    dim3 grid(N / BN, (M + tc::kBM - 1) / tc::kBM);
    tc::k_tc_gemm<BN, EpiStoreF32><<<grid, tc::kThreads, tc::TileCfg<BN>::kSmemBytes, s>>>(ma, mb, M, K, epi, status);
    return launch_status();
}
}  // namespace

}  // namespace pe

using namespace pe;

extern "C" PE_API int pe_tc_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc,
                                      int32_t M, int32_t N, int32_t K, uint32_t* status, void* stream)
{
    if (!A || !B || !C || !status || M < 1 || N < 64 || N % 64 != 0 || K < 1 || ldc < N || ldc % 4 != 0 ||
        ((uintptr_t)C & 15u))
        return PE_EINVAL;
    const int bn = (N % 128 == 0) ? 128 : 64;
    CUtensorMap ma, mb;
    PE_TRY(tc_operand_map(&ma, A, M, K, lda, tc::kBM));
    PE_TRY(tc_operand_map(&mb, B, N, K, ldb, bn));
    EpiStoreF32 epi{C, M, ldc};
    cudaStream_t s = (cudaStream_t)stream;
    return bn == 128 ? launch_plain<128>(ma, mb, M, N, K, epi, status, s)
                     : launch_plain<64>(ma, mb, M, N, K, epi, status, s);
}
