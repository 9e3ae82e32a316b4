// Learned coarse-derivative surrogate: a multilayer perceptron c -> dc/dt trained on the
// least-squares slopes that resolved bursts measure (Section 3.3, Eq. (leastsquares)),
// with BF16 tensor-core GEMMs accumulating in FP32, GELU hidden layers, MSE loss and
// Adam. Every layer's forward, data-gradient and weight-gradient product is one launch of
// the tcgen05 GEMM of pe_tc.cuh (TMEM accumulator, TMA-staged operands) with the bias,
// activation, loss or GELU' factor fused into its epilogue. That kernel takes both operands
// with K contiguous, so the products that contract over another index read transposed
// copies kept alongside: the BF16 weights' transposes (rewritten with the mirror by Adam),
// and the activations' and gradients' transposes (written by the epilogues that produce them).
//
// Storage (caller-owned arena, see pe_mlp_layout_for): FP32 master parameters (the flat
// vector W_1 [d1][d0], b_1, W_2, ...), their BF16 mirror and its per-layer transposes used by
// the GEMMs, FP32 gradients, Adam moments, per-component z-score statistics, and a batch
// workspace.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pe_common.cuh"
#include "pe_ctx.h"
#include "pe_internal.h"
#include "pe_tc.cuh"
#include "pepic.h"

namespace pe {
namespace {

constexpr int kNormBlocks = 64;    // row blocks of the z-score statistics
constexpr int kLossSlots = 4096;

enum Epi { kEpiHidden = 0, kEpiOutInfer = 1, kEpiOutTrain = 2, kEpiDgrad = 3, kEpiWgrad = 4 };

__device__ __forceinline__ float warp_sum_f(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int M, N, K, lda, ldb;
    const float* bias;     // [N] (hidden / output epilogues)
    float* Z;              // hidden: pre-activation out [M][N]; dgrad: pre-activation in
    __nv_bfloat16* Aout;   // hidden: GELU(z) out; train / dgrad: gradient out [M][N] (BF16)
    const float* T;        // train: normalised target [M][N]
    float* Y;              // output: FP32 out [M][N] (infer: de-normalised unless Y64 set)
    double* Y64;           // infer: de-normalised FP64 out
    const float* mu;       // infer: output mean [N]
    const float* sd;       // infer: output deviation [N]
    float* loss_part;      // train: one partial per block
    float gscale;          // train: 2 / (B D)
};

// Epilogue of the tensor-core GEMM for row m, columns n0 .. n0 + 31 of C = A B^T (FP32 from
// TMEM): the bias + GELU of a hidden layer (Z, Aout and its transpose AoutT), the
// de-normalised output (inference), the loss and output gradient (training; Y optional, G and
// its transpose), the data gradient times GELU'(Z) (G and its transpose), or the FP32 weight
// gradient. Rows beyond M are not stored. finish() folds the training loss of the block into
// loss_part[block] (every thread calls it).
template <int EPI>
struct TcEpi {
    GemmArgs g;
    __nv_bfloat16* AoutT;  // transposed BF16 output [N][ldT]
    int ldT;
    float lsum;

    __device__ __forceinline__ void operator()(int m, int n0, const float* v)
    {
        if (m >= g.M) return;
        const size_t o = (size_t)m * g.N + n0;
        if (EPI == kEpiWgrad) {
            float4* d = reinterpret_cast<float4*>(g.Y + o);
#pragma unroll
            for (int j = 0; j < 8; ++j) d[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            return;
        }
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            const int n = n0 + j;
            float v0 = v[j], v1 = v[j + 1];
            if (EPI == kEpiHidden) {
                v0 += g.bias[n];
                v1 += g.bias[n + 1];
                *reinterpret_cast<float2*>(g.Z + o + j) = make_float2(v0, v1);
                const __nv_bfloat162 a = __floats2bfloat162_rn(gelu_f(v0), gelu_f(v1));
                *reinterpret_cast<__nv_bfloat162*>(g.Aout + o + j) = a;
                AoutT[(size_t)n * ldT + m] = a.x;
                AoutT[(size_t)(n + 1) * ldT + m] = a.y;
            } else if (EPI == kEpiOutInfer) {
                v0 += g.bias[n];
                v1 += g.bias[n + 1];
                const float y0 = fmaf(v0, g.sd[n], g.mu[n]), y1 = fmaf(v1, g.sd[n + 1], g.mu[n + 1]);
                if (g.Y64) {
                    g.Y64[o + j] = (double)y0;
                    g.Y64[o + j + 1] = (double)y1;
                } else {
                    *reinterpret_cast<float2*>(g.Y + o + j) = make_float2(y0, y1);
                }
            } else if (EPI == kEpiOutTrain) {
                v0 += g.bias[n];
                v1 += g.bias[n + 1];
                const float2 t = *reinterpret_cast<const float2*>(g.T + o + j);
                const float d0 = v0 - t.x, d1 = v1 - t.y;
                lsum = fmaf(d0, d0, fmaf(d1, d1, lsum));
                if (g.Y) *reinterpret_cast<float2*>(g.Y + o + j) = make_float2(v0, v1);
                const __nv_bfloat162 gr = __floats2bfloat162_rn(g.gscale * d0, g.gscale * d1);
                *reinterpret_cast<__nv_bfloat162*>(g.Aout + o + j) = gr;
                AoutT[(size_t)n * ldT + m] = gr.x;
                AoutT[(size_t)(n + 1) * ldT + m] = gr.y;
            } else if (EPI == kEpiDgrad) {
                const float2 z = *reinterpret_cast<const float2*>(g.Z + o + j);
                const __nv_bfloat162 gr = __floats2bfloat162_rn(v0 * gelu_grad_f(z.x), v1 * gelu_grad_f(z.y));
                *reinterpret_cast<__nv_bfloat162*>(g.Aout + o + j) = gr;
                AoutT[(size_t)n * ldT + m] = gr.x;
                AoutT[(size_t)(n + 1) * ldT + m] = gr.y;
            }
        }
    }

    __device__ __forceinline__ void finish()
    {
        if (EPI != kEpiOutTrain) return;
        __shared__ float sloss[tc::kThreads / 32];
        const float w = warp_sum_f(lsum);
        if ((threadIdx.x & 31) == 0) sloss[threadIdx.x >> 5] = w;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int k = 0; k < tc::kThreads / 32; ++k) t += sloss[k];
            g.loss_part[blockIdx.y * gridDim.x + blockIdx.x] = t;
        }
    }
};

// ------------------------------------------------------------------ small kernels

// Weight blocks of the flat parameter vector: layer l's W [rows = d_{l+1}][cols = d_l] at off;
// its BF16 transpose [d_l][d_{l+1}] sits at the same offset of the transposed mirror.
struct WeightTable {
    int64_t off[PE_MLP_MAX_LAYERS];
    int rows[PE_MLP_MAX_LAYERS], cols[PE_MLP_MAX_LAYERS];
    int L;
};

// Writes the BF16 value of flat parameter i into the mirror and, for a weight, into the
// transposed mirror.
__device__ __forceinline__ void put_bf16(const WeightTable& wt, int64_t i, float w, __nv_bfloat16* __restrict__ pb,
                                         __nv_bfloat16* __restrict__ pbT)
{
    const __nv_bfloat16 b = __float2bfloat16_rn(w);
    pb[i] = b;
    for (int l = 0; l < wt.L; ++l) {
        const int64_t r = i - wt.off[l];
        if (r >= 0 && r < (int64_t)wt.rows[l] * wt.cols[l]) {
            const int row = (int)(r / wt.cols[l]), col = (int)(r - (int64_t)row * wt.cols[l]);
            pbT[wt.off[l] + (int64_t)col * wt.rows[l] + row] = b;
            break;
        }
    }
}

struct ParamSeg {
    int64_t off, n;
    float bound;  // weight init bound (0 for biases)
};
struct ParamTable {
    ParamSeg seg[2 * PE_MLP_MAX_LAYERS];
    int nseg;
};

__device__ __forceinline__ uint64_t splitmix64_seq(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// W = (2u - 1) a with u = (s_i >> 40) 2^-24 from the splitmix64 sequence (flat index i);
// biases 0. Writes the FP32 master and its BF16 mirror.
__global__ void k_mlp_init(ParamTable tab, WeightTable wt, uint64_t seed, float* __restrict__ p,
                           __nv_bfloat16* __restrict__ pb, __nv_bfloat16* __restrict__ pbT)
{
    for (int s = 0; s < tab.nseg; ++s) {
        const ParamSeg sg = tab.seg[s];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sg.n; i += (int64_t)gridDim.x * blockDim.x) {
            const int64_t idx = sg.off + i;
            float w = 0.0f;
            if (sg.bound > 0.0f) {
                const float u = (float)(splitmix64_seq(seed, (uint64_t)idx) >> 40) * 5.9604644775390625e-8f;
                w = (2.0f * u - 1.0f) * sg.bound;
            }
            p[idx] = w;
            put_bf16(wt, idx, w, pb, pbT);
        }
    }
}

// Per-component column sums of X [rows][D] over row block blockIdx.y (pass 0: sum x;
// pass 1: sum (x - mu)^2), FP64, fixed order; with period P > 0 component k is pooled
// with every k' = k (mod P)-position of its block of P (translation-invariant statistics).
template <typename T>
__global__ void k_norm_partial(const T* __restrict__ X, int64_t rows, int D, const double* __restrict__ mu,
                               double* __restrict__ part)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= D) return;
    const int64_t per = (rows + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = blockIdx.y * per, r1 = min(rows, r0 + per);
    double s = 0.0;
    const double m = mu ? mu[k] : 0.0;
    for (int64_t r = r0; r < r1; ++r) {
        const double x = (double)X[r * D + k];
        s += mu ? (x - m) * (x - m) : x;
    }
    part[(size_t)blockIdx.y * D + k] = s;
}

// Folds the row-block partials (and, with P > 0, the P positions of each block) into
// mean (pass 0) or deviation (pass 1, with the 1e-6 max floor) in FP64 and FP32.
__global__ void k_norm_final(const double* __restrict__ part, int nparts, int D, int P, int64_t rows, int pass,
                             double* __restrict__ acc64, float* __restrict__ out32)
{
    __shared__ double red[32];
    __shared__ double smax;
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
        double s = 0.0;
        int64_t cnt = rows;
        if (P > 0) {
            const int b0 = (k / P) * P;
            for (int j = 0; j < P; ++j)
                for (int q = 0; q < nparts; ++q) s += part[(size_t)q * D + b0 + j];
            cnt = rows * P;
        } else {
            for (int q = 0; q < nparts; ++q) s += part[(size_t)q * D + k];
        }
        acc64[D + k] = (pass == 0) ? s / (double)cnt : sqrt(s / (double)cnt);
    }
    __syncthreads();
    if (pass == 0) {
        for (int k = threadIdx.x; k < D; k += blockDim.x) {
            acc64[k] = acc64[D + k];
            out32[k] = (float)acc64[k];
        }
        return;
    }
    double mx = 0.0;
    for (int k = threadIdx.x; k < D; k += blockDim.x) mx = fmax(mx, acc64[D + k]);
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        smax = 1e-6 * fmax(m, 1e-30);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < D; k += blockDim.x) out32[k] = (float)fmax(acc64[D + k], smax);
}

// Batch rows and translation shifts for a training step, from the splitmix64 sequence of
// (seed, step): row = (h >> 32) npairs >> 32, shift = (h mod 2^32) P >> 32.
__global__ void k_sample_rows(uint64_t seed, const int64_t* __restrict__ step, int B, int64_t npairs, int P,
                              int32_t* __restrict__ rows, int32_t* __restrict__ shifts)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const uint64_t h = splitmix64_seq(seed, (uint64_t)(*step) * (uint64_t)B + (uint64_t)i);
    rows[i] = (int32_t)(((h >> 32) * (uint64_t)npairs) >> 32);
    shifts[i] = P > 0 ? (int32_t)(((h & 0xFFFFFFFFull) * (uint64_t)P) >> 32) : 0;
}

// Normalised BF16 inputs (and FP32 targets) of a batch: x'[k] = x[src(k)] with the
// circular shift s inside each block of P components, src(k) = b P + (j - s) mod P.
template <typename T>
__global__ void k_prep(const T* __restrict__ X, const float* __restrict__ Y, int B, int D, int Dout,
                       const int32_t* __restrict__ rows, const int32_t* __restrict__ shifts, int P,
                       const float* __restrict__ mu, const float* __restrict__ sd, const float* __restrict__ mu_o,
                       const float* __restrict__ sd_o, __nv_bfloat16* __restrict__ xz, __nv_bfloat16* __restrict__ xzT,
                       int ldT, float* __restrict__ tz)
{
    const int i = blockIdx.y;
    if (i >= B) return;
    const int64_t r = rows ? rows[i] : i;
    const int s = shifts ? shifts[i] : 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < max(D, Dout); k += gridDim.x * blockDim.x) {
        int src = k;
        if (P > 0) {
            const int j = k % P;
            src = k - j + (j - s + P) % P;
        }
        if (k < D) {
            const float x = (float)X[r * D + src];
            const __nv_bfloat16 b = __float2bfloat16_rn((x - mu[k]) / sd[k]);
            xz[(size_t)i * D + k] = b;
            if (xzT) xzT[(size_t)k * ldT + i] = b;
        }
        if (Y && k < Dout) tz[(size_t)i * Dout + k] = (Y[r * Dout + src] - mu_o[k]) / sd_o[k];
    }
}

// Bias gradient db[n] = sum_m G[m][n] from the transposed gradient GT [N][ldT] (row n holds
// G[0..M)[n] contiguously): one warp per n, lanes over m, FP32 partial sums folded in a
// fixed order (reproducible).
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ GT, int ldT, int M, int N, float* __restrict__ db)
{
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (n >= N) return;
    const __nv_bfloat16* row = GT + (size_t)n * ldT;
    float s = 0.0f;
    for (int m = lane; m < M; m += 32) s += __bfloat162float(row[m]);
    s = warp_sum_f(s);
    if (lane == 0) db[n] = s;
}

__global__ void k_loss_final(const float* __restrict__ part, int n, float* __restrict__ out, float scale)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)part[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = (float)(t * scale);
    }
}

// Adam with bias correction; the step counter lives on the device (graph replays
// advance it). theta, m, v FP32; the BF16 mirror is rewritten. The decay rates and their
// complements come in FP64 (0.999 is not a float) and the bias corrections are formed in
// FP64 once per thread.
__global__ void k_adam(float* __restrict__ p, __nv_bfloat16* __restrict__ pb, __nv_bfloat16* __restrict__ pbT,
                       WeightTable wt, const float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, int64_t* __restrict__ step, float lr, double b1, double b2, float eps)
{
    const int64_t t = *step + 1;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)t))), c2 = (float)(1.0 / (1.0 - pow(b2, (double)t)));
    const float fb1 = (float)b1, fb2 = (float)b2, ob1 = (float)(1.0 - b1), ob2 = (float)(1.0 - b2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = fmaf(fb1, m[i], ob1 * gi);
        const float vi = fmaf(fb2, v[i], ob2 * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float w = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = w;
        put_bf16(wt, i, w, pb, pbT);
    }
}

__global__ void k_step_advance(int64_t* step)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

}  // namespace
}  // namespace pe

// ------------------------------------------------------------------ host side

struct pe_mlp {
    int L;
    int dims[PE_MLP_MAX_LAYERS + 1];
    int dmax, max_batch;
    int64_t nparams;
    int64_t w_off[PE_MLP_MAX_LAYERS], b_off[PE_MLP_MAX_LAYERS];
    pe_mlp_layout lay;
    char* arena;
    cudaStream_t stream;
    float* p;
    __nv_bfloat16* pb;
    __nv_bfloat16* pbT;  // per-layer transposes of the BF16 weights (same offsets as pb)
    pe::WeightTable wt;
    float* grad;
    float* am;
    float* av;
    float* norm;        // [4][dmax]: mu_in, sd_in, mu_out, sd_out
    double* norm64;     // [2][dmax] scratch of the statistics
    double* normpart;   // [kNormBlocks][dmax]
    int64_t* step;      // Adam step counter (device)
    float* loss;        // last training loss (device)
    float* loss_part;   // [kLossSlots]
    int32_t* rows;
    int32_t* shifts;
    __nv_bfloat16* xz;  // [Bm][d0]
    float* z[PE_MLP_MAX_LAYERS];
    __nv_bfloat16* a[PE_MLP_MAX_LAYERS];
    float* y;           // [Bm][dL]
    float* tz;          // [Bm][dL]
    __nv_bfloat16* g[2];
    int ldT;             // row stride of the transposed batch arrays (max_batch rounded up to 64)
    __nv_bfloat16* xzT;  // [d0][ldT]
    __nv_bfloat16* aT[PE_MLP_MAX_LAYERS];  // [d_{l+1}][ldT]
    __nv_bfloat16* gT[2];                  // [dmax][ldT]
    uint32_t* status;    // device status word (PE_FLAG_TIMEOUT from the GEMM's bounded waits)
    int shift_period;   // period used by the statistics (for reference)
};

using namespace pe;

namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

int check_dims(int32_t nlayers, const int32_t* dims, int32_t max_batch)
{
    if (nlayers < 1 || nlayers > PE_MLP_MAX_LAYERS || !dims || max_batch < 1 || max_batch > 65536) return PE_EINVAL;
    for (int l = 0; l <= nlayers; ++l)
        if (dims[l] < 64 || dims[l] > 4096 || dims[l] % 64) return PE_EINVAL;
    return PE_OK;
}

struct WorkPlan {
    size_t rows, shifts, xz, z[PE_MLP_MAX_LAYERS], a[PE_MLP_MAX_LAYERS], y, tz, g0, g1, xzT, aT[PE_MLP_MAX_LAYERS],
        gT0, gT1, total;
};

int ld_transposed(int Bm) { return (Bm + 63) & ~63; }

WorkPlan plan_work(int L, const int32_t* dims, int Bm, int dmax)
{
    WorkPlan w;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += al256(bytes);
        return at;
    };
    w.rows = take(4 * (size_t)Bm);
    w.shifts = take(4 * (size_t)Bm);
    w.xz = take(2 * (size_t)Bm * dims[0]);
    for (int l = 0; l + 1 < L; ++l) {
        w.z[l] = take(4 * (size_t)Bm * dims[l + 1]);
        w.a[l] = take(2 * (size_t)Bm * dims[l + 1]);
    }
    w.y = take(4 * (size_t)Bm * dims[L]);
    w.tz = take(4 * (size_t)Bm * dims[L]);
    w.g0 = take(2 * (size_t)Bm * dmax);
    w.g1 = take(2 * (size_t)Bm * dmax);
    const size_t ldT = (size_t)ld_transposed(Bm);
    w.xzT = take(2 * ldT * dims[0]);
    for (int l = 0; l + 1 < L; ++l) w.aT[l] = take(2 * ldT * dims[l + 1]);
    w.gT0 = take(2 * ldT * dmax);
    w.gT1 = take(2 * ldT * dmax);
    w.total = o;
    return w;
}

// C[M][N] = A[M][K] B[N][K]^T on the tensor cores with the epilogue EPI; A and B stored
// with K contiguous (row strides lda, ldb). AoutT/ldT: transposed BF16 copy of the output.
// Returns the number of tiles (one loss partial each).
// Tile width: 128 columns, or 64 when N needs it or when 128-wide tiles would leave SMs idle.
int tile_n(int N, int M)
{
    if (N % 128 != 0) return 64;
    return (N / 128) * ((M + tc::kBM - 1) / tc::kBM) < sm_count() ? 64 : 128;
}

template <int EPI>
int tc_gemm(pe_mlp* h, const GemmArgs& g, __nv_bfloat16* AoutT, cudaStream_t s, int* tiles)
{
    const int bn = tile_n(g.N, g.M);
    CUtensorMap ma, mb;
    PE_TRY(tc_operand_map(&ma, g.A, g.M, g.K, g.lda, tc::kBM));
    PE_TRY(tc_operand_map(&mb, g.B, g.N, g.K, g.ldb, bn));
    TcEpi<EPI> e{g, AoutT, h->ldT, 0.0f};
    dim3 grid(g.N / bn, (g.M + tc::kBM - 1) / tc::kBM);
    if (tiles) *tiles = (int)(grid.x * grid.y);
    if (bn == 128) {
        const void* k = (const void*)tc::k_tc_gemm<128, TcEpi<EPI>>;
        if (ensure_smem(k, tc::TileCfg<128>::kSmemBytes) != PE_OK) return PE_ECUDA;
        tc::k_tc_gemm<128, TcEpi<EPI>><<<grid, tc::kThreads, tc::TileCfg<128>::kSmemBytes, s>>>(ma, mb, g.M, g.K, e,
                                                                                               h->status);
    } else {
        const void* k = (const void*)tc::k_tc_gemm<64, TcEpi<EPI>>;
        if (ensure_smem(k, tc::TileCfg<64>::kSmemBytes) != PE_OK) return PE_ECUDA;
        tc::k_tc_gemm<64, TcEpi<EPI>><<<grid, tc::kThreads, tc::TileCfg<64>::kSmemBytes, s>>>(ma, mb, g.M, g.K, e,
                                                                                             h->status);
    }
    return PE_OK;
}

// Loss partials of the output layer's GEMM (one per tile).
int loss_tiles(int Dout, int B) { return (Dout / tile_n(Dout, B)) * ((B + tc::kBM - 1) / tc::kBM); }

GemmArgs args0() { GemmArgs g; memset(&g, 0, sizeof(g)); return g; }

// Forward through every layer from h->xz (rows B). mode 0: inference, output into
// y32 / y64 de-normalised; mode 1: training, output compared with h->tz.
int forward(pe_mlp* h, int B, int train, float* y32, double* y64, int* launches)
{
    cudaStream_t s = h->stream;
    const __nv_bfloat16* in = h->xz;
    for (int l = 0; l < h->L; ++l) {
        GemmArgs g = args0();
        g.A = in;
        g.B = h->pb + h->w_off[l];
        g.M = B;
        g.N = h->dims[l + 1];
        g.K = h->dims[l];
        g.lda = h->dims[l];
        g.ldb = h->dims[l];
        g.bias = h->p + h->b_off[l];
        if (l + 1 < h->L) {
            g.Z = h->z[l];
            g.Aout = h->a[l];
            PE_TRY(tc_gemm<kEpiHidden>(h, g, h->aT[l], s, nullptr));
            in = h->a[l];
        } else if (!train) {
            g.Y = y32;
            g.Y64 = y64;
            g.mu = h->norm + 2 * h->dmax;
            g.sd = h->norm + 3 * h->dmax;
            PE_TRY(tc_gemm<kEpiOutInfer>(h, g, nullptr, s, nullptr));
        } else {
            g.T = h->tz;
            g.Y = h->y;
            g.Aout = h->g[(h->L - 1) & 1];
            g.loss_part = h->loss_part;
            g.gscale = 2.0f / ((float)B * (float)g.N);
            PE_TRY(tc_gemm<kEpiOutTrain>(h, g, h->gT[(h->L - 1) & 1], s, nullptr));
        }
        ++*launches;
    }
    return PE_OK;
}

// Backward from the output gradient in g[(L-1)&1]: weight and bias gradients of every
// layer into h->grad, data gradients (times GELU') down to layer 1.
int backward(pe_mlp* h, int B, int* launches)
{
    cudaStream_t s = h->stream;
    for (int l = h->L - 1; l >= 0; --l) {
        const __nv_bfloat16* gl = h->g[l & 1];
        GemmArgs w = args0();  // dW_l [d_{l+1}][d_l] = G_l^T act_{l-1}: both transposes, K = batch
        w.A = h->gT[l & 1];
        w.B = l ? h->aT[l - 1] : h->xzT;
        w.M = h->dims[l + 1];
        w.N = h->dims[l];
        w.K = B;
        w.lda = h->ldT;
        w.ldb = h->ldT;
        w.Y = h->grad + h->w_off[l];
        PE_TRY(tc_gemm<kEpiWgrad>(h, w, nullptr, s, nullptr));
        k_bias_grad<<<(h->dims[l + 1] + 7) / 8, 256, 0, s>>>(h->gT[l & 1], h->ldT, B, h->dims[l + 1],
                                                             h->grad + h->b_off[l]);
        *launches += 2;
        if (l == 0) break;
        GemmArgs d = args0();  // G_{l-1} = (G_l W_l) * GELU'(z_{l-1}): W_l read as its transpose
        d.A = gl;
        d.B = h->pbT + h->w_off[l];
        d.M = B;
        d.N = h->dims[l];
        d.K = h->dims[l + 1];
        d.lda = h->dims[l + 1];
        d.ldb = h->dims[l + 1];
        d.Z = h->z[l - 1];
        d.Aout = h->g[(l - 1) & 1];
        PE_TRY(tc_gemm<kEpiDgrad>(h, d, h->gT[(l - 1) & 1], s, nullptr));
        ++*launches;
    }
    return PE_OK;
}

int grad_pass(pe_mlp* h, const float* X, const float* Y, int64_t npairs, const int32_t* rows, const int32_t* shifts,
              int B, int P, int* launches)
{
    cudaStream_t s = h->stream;
    const int D = h->dims[0], Dout = h->dims[h->L];
    dim3 pg((std::max(D, Dout) + 255) / 256, B);
    k_prep<float><<<pg, 256, 0, s>>>(X, Y, B, D, Dout, rows, shifts, P, h->norm, h->norm + h->dmax,
                                     h->norm + 2 * h->dmax, h->norm + 3 * h->dmax, h->xz, h->xzT, h->ldT, h->tz);
    ++*launches;
    PE_TRY(forward(h, B, 1, nullptr, nullptr, launches));
    const int nblk = loss_tiles(Dout, B);
    k_loss_final<<<1, 256, 0, s>>>(h->loss_part, nblk, h->loss, 1.0f / ((float)B * (float)Dout));
    ++*launches;
    return backward(h, B, launches);
}

}  // namespace

extern "C" PE_API int pe_mlp_layout_for(int32_t nlayers, const int32_t* dims, int32_t max_batch, pe_mlp_layout* out)
{
    if (!out) return PE_EINVAL;
    PE_TRY(check_dims(nlayers, dims, max_batch));
    memset(out, 0, sizeof(*out));
    int64_t np = 0;
    int dmax = 0;
    for (int l = 0; l < nlayers; ++l) np += (int64_t)dims[l + 1] * dims[l] + dims[l + 1];
    for (int l = 0; l <= nlayers; ++l) dmax = std::max(dmax, (int)dims[l]);
    out->nparams = np;
    out->bytes[PE_MLP_PARAMS] = 4 * (size_t)np;
    out->bytes[PE_MLP_PARAMS_BF16] = 2 * 2 * (size_t)np;  // the mirror, then its per-layer transposes
    out->bytes[PE_MLP_GRADS] = 4 * (size_t)np;
    out->bytes[PE_MLP_ADAM_M] = 4 * (size_t)np;
    out->bytes[PE_MLP_ADAM_V] = 4 * (size_t)np;
    out->bytes[PE_MLP_NORM] = 4 * 4 * (size_t)dmax + 8 * 2 * (size_t)dmax + 8 * (size_t)kNormBlocks * dmax + 256 +
                              4 * (size_t)kLossSlots;
    out->bytes[PE_MLP_WORK] = plan_work(nlayers, dims, max_batch, dmax).total;
    size_t off = 0;
    for (int b = 0; b < PE_MLP_NBUF; ++b) {
        out->offset[b] = off;
        off += al256(out->bytes[b]);
    }
    out->total_bytes = off;
    return PE_OK;
}

extern "C" PE_API int pe_mlp_create(int32_t nlayers, const int32_t* dims, int32_t max_batch, void* arena,
                                    size_t arena_bytes, void* stream, pe_mlp** out)
{
    if (!out) return PE_EINVAL;
    *out = nullptr;
    pe_mlp_layout lay;
    PE_TRY(pe_mlp_layout_for(nlayers, dims, max_batch, &lay));
    if (!arena || ((uintptr_t)arena & 255u) || arena_bytes < lay.total_bytes) return PE_EINVAL;
    pe_mlp* h = (pe_mlp*)calloc(1, sizeof(pe_mlp));
    if (!h) return PE_EINVAL;
    h->L = nlayers;
    h->dmax = 0;
    for (int l = 0; l <= nlayers; ++l) {
        h->dims[l] = dims[l];
        h->dmax = std::max(h->dmax, (int)dims[l]);
    }
    h->max_batch = max_batch;
    h->nparams = lay.nparams;
    int64_t o = 0;
    for (int l = 0; l < nlayers; ++l) {
        h->w_off[l] = o;
        o += (int64_t)dims[l + 1] * dims[l];
        h->b_off[l] = o;
        o += dims[l + 1];
    }
    h->lay = lay;
    h->arena = (char*)arena;
    h->stream = (cudaStream_t)stream;
    h->p = (float*)(h->arena + lay.offset[PE_MLP_PARAMS]);
    h->pb = (__nv_bfloat16*)(h->arena + lay.offset[PE_MLP_PARAMS_BF16]);
    h->pbT = h->pb + h->nparams;
    h->wt.L = nlayers;
    for (int l = 0; l < nlayers; ++l) {
        h->wt.off[l] = h->w_off[l];
        h->wt.rows[l] = dims[l + 1];
        h->wt.cols[l] = dims[l];
    }
    h->grad = (float*)(h->arena + lay.offset[PE_MLP_GRADS]);
    h->am = (float*)(h->arena + lay.offset[PE_MLP_ADAM_M]);
    h->av = (float*)(h->arena + lay.offset[PE_MLP_ADAM_V]);
    char* nb = h->arena + lay.offset[PE_MLP_NORM];
    h->norm = (float*)nb;
    nb += 4 * 4 * (size_t)h->dmax;
    h->norm64 = (double*)nb;
    nb += 8 * 2 * (size_t)h->dmax;
    h->normpart = (double*)nb;
    nb += 8 * (size_t)kNormBlocks * h->dmax;
    h->step = (int64_t*)nb;
    h->loss = (float*)(nb + 8);
    h->status = (uint32_t*)(nb + 16);
    h->loss_part = (float*)(nb + 256);
    const WorkPlan w = plan_work(nlayers, dims, max_batch, h->dmax);
    char* wb = h->arena + lay.offset[PE_MLP_WORK];
    h->rows = (int32_t*)(wb + w.rows);
    h->shifts = (int32_t*)(wb + w.shifts);
    h->xz = (__nv_bfloat16*)(wb + w.xz);
    for (int l = 0; l + 1 < nlayers; ++l) {
        h->z[l] = (float*)(wb + w.z[l]);
        h->a[l] = (__nv_bfloat16*)(wb + w.a[l]);
    }
    h->y = (float*)(wb + w.y);
    h->tz = (float*)(wb + w.tz);
    h->g[0] = (__nv_bfloat16*)(wb + w.g0);
    h->g[1] = (__nv_bfloat16*)(wb + w.g1);
    h->ldT = ld_transposed(max_batch);
    h->xzT = (__nv_bfloat16*)(wb + w.xzT);
    for (int l = 0; l + 1 < nlayers; ++l) h->aT[l] = (__nv_bfloat16*)(wb + w.aT[l]);
    h->gT[0] = (__nv_bfloat16*)(wb + w.gT0);
    h->gT[1] = (__nv_bfloat16*)(wb + w.gT1);
    *out = h;
    return PE_OK;
}

extern "C" PE_API void pe_mlp_destroy(pe_mlp* h) { free(h); }

extern "C" PE_API int pe_mlp_init(pe_mlp* h, uint64_t seed)
{
    if (!h) return PE_EINVAL;
    ParamTable tab;
    memset(&tab, 0, sizeof(tab));
    for (int l = 0; l < h->L; ++l) {
        const bool last = l == h->L - 1;
        tab.seg[2 * l] = {h->w_off[l], (int64_t)h->dims[l + 1] * h->dims[l],
                          (float)sqrt((last ? 3.0 : 6.0) / h->dims[l])};
        tab.seg[2 * l + 1] = {h->b_off[l], h->dims[l + 1], 0.0f};
    }
    tab.nseg = 2 * h->L;
    cudaStream_t s = h->stream;
    k_mlp_init<<<2 * sm_count(), 256, 0, s>>>(tab, h->wt, seed, h->p, h->pb, h->pbT);
    const size_t nb = 4 * (size_t)h->nparams;
    if (cudaMemsetAsync(h->am, 0, nb, s) != cudaSuccess || cudaMemsetAsync(h->av, 0, nb, s) != cudaSuccess ||
        cudaMemsetAsync(h->grad, 0, nb, s) != cudaSuccess || cudaMemsetAsync(h->step, 0, 32, s) != cudaSuccess)
        return PE_ECUDA;
    // identity normalisation until pe_mlp_fit_norm
    std::vector<float> id(4 * (size_t)h->dmax, 0.0f);
    for (int k = 0; k < h->dmax; ++k) id[h->dmax + k] = id[3 * h->dmax + k] = 1.0f;
    if (cudaMemcpyAsync(h->norm, id.data(), 4 * id.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) return PE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PE_ECUDA;  // host vector goes out of scope
    return launch_status(1);
}

extern "C" PE_API int pe_mlp_fit_norm(pe_mlp* h, const float* X, const float* Y, int64_t npairs, int32_t period)
{
    if (!h || !X || !Y || npairs < 1) return PE_EINVAL;
    const int D[2] = {h->dims[0], h->dims[h->L]};
    for (int q = 0; q < 2; ++q)
        if (period < 0 || (period > 0 && D[q] % period)) return PE_EINVAL;
    cudaStream_t s = h->stream;
    const int nparts = (int)std::min<int64_t>(kNormBlocks, npairs);
    for (int q = 0; q < 2; ++q) {
        const float* src = q ? Y : X;
        float* mu32 = h->norm + (2 * q) * h->dmax;
        float* sd32 = h->norm + (2 * q + 1) * h->dmax;
        dim3 grid((D[q] + 255) / 256, nparts);
        k_norm_partial<float><<<grid, 256, 0, s>>>(src, npairs, D[q], nullptr, h->normpart);
        k_norm_final<<<1, 1024, 0, s>>>(h->normpart, nparts, D[q], period, npairs, 0, h->norm64, mu32);
        k_norm_partial<float><<<grid, 256, 0, s>>>(src, npairs, D[q], h->norm64, h->normpart);
        k_norm_final<<<1, 1024, 0, s>>>(h->normpart, nparts, D[q], period, npairs, 1, h->norm64, sd32);
    }
    h->shift_period = period;
    return launch_status(8);
}

extern "C" PE_API int pe_mlp_forward(pe_mlp* h, const void* x, int32_t x_is_f64, int32_t B, void* y, int32_t y_is_f64)
{
    if (!h || !x || !y || B < 1 || B > h->max_batch) return PE_EINVAL;
    cudaStream_t s = h->stream;
    const int D = h->dims[0];
    dim3 pg((D + 255) / 256, B);
    if (x_is_f64)
        k_prep<double><<<pg, 256, 0, s>>>((const double*)x, nullptr, B, D, 0, nullptr, nullptr, 0, h->norm,
                                          h->norm + h->dmax, nullptr, nullptr, h->xz, nullptr, h->ldT, nullptr);
    else
        k_prep<float><<<pg, 256, 0, s>>>((const float*)x, nullptr, B, D, 0, nullptr, nullptr, 0, h->norm,
                                         h->norm + h->dmax, nullptr, nullptr, h->xz, nullptr, h->ldT, nullptr);
    int launches = 1;
    PE_TRY(forward(h, B, 0, y_is_f64 ? nullptr : (float*)y, y_is_f64 ? (double*)y : nullptr, &launches));
    return launch_status(launches);
}

extern "C" PE_API int pe_mlp_grad(pe_mlp* h, const float* X, const float* Y, int64_t npairs, const int32_t* rows,
                                  int32_t B, float* loss)
{
    if (!h || !X || !Y || B < 32 || B % 32 || B > h->max_batch || (!rows && npairs < B)) return PE_EINVAL;
    if (loss_tiles(h->dims[h->L], B) > kLossSlots) return PE_EINVAL;
    int launches = 0;
    PE_TRY(grad_pass(h, X, Y, npairs, rows, nullptr, B, 0, &launches));
    if (loss && cudaMemcpyAsync(loss, h->loss, 4, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess) return PE_ECUDA;
    return launch_status(launches);
}

extern "C" PE_API int pe_mlp_adam(pe_mlp* h, double lr, double beta1, double beta2, double eps)
{
    if (!h || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return PE_EINVAL;
    cudaStream_t s = h->stream;
    k_adam<<<2 * sm_count(), 256, 0, s>>>(h->p, h->pb, h->pbT, h->wt, h->grad, h->am, h->av, h->nparams, h->step,
                                          (float)lr, beta1, beta2, (float)eps);
    k_step_advance<<<1, 32, 0, s>>>(h->step);
    return launch_status(2);
}

extern "C" PE_API int pe_mlp_train(pe_mlp* h, const float* X, const float* Y, int64_t npairs, int32_t B,
                                   int32_t shift_period, uint64_t seed, int32_t nsteps, float lr, float* loss)
{
    if (!h || !X || !Y || npairs < 1 || npairs >= (int64_t(1) << 31) || nsteps < 0 || B < 32 || B % 32 ||
        B > h->max_batch || !(lr >= 0.0f))
        return PE_EINVAL;
    const int D = h->dims[0], Dout = h->dims[h->L];
    if (shift_period < 0 || (shift_period > 0 && (D % shift_period || Dout % shift_period))) return PE_EINVAL;
    if (loss_tiles(Dout, B) > kLossSlots) return PE_EINVAL;
    cudaStream_t s = h->stream;
    const int nsm = sm_count();  // cached before any capture
    int launches = 0;
    auto one_step = [&]() {
        k_sample_rows<<<(B + 255) / 256, 256, 0, s>>>(seed, h->step, B, npairs, shift_period, h->rows, h->shifts);
        grad_pass(h, X, Y, npairs, h->rows, h->shifts, B, shift_period, &launches);
        k_adam<<<2 * nsm, 256, 0, s>>>(h->p, h->pb, h->pbT, h->wt, h->grad, h->am, h->av, h->nparams, h->step, lr,
                                       0.9, 0.999, 1e-8f);
        k_step_advance<<<1, 32, 0, s>>>(h->step);
        launches += 3;
    };
    // One step captured as a graph and replayed (the step counter on the device advances the
    // sampling and the bias correction); on the legacy default stream the steps run eagerly.
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool captured = false;
    if (s != nullptr && nsteps > 1 && cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        one_step();
        if (cudaStreamEndCapture(s, &graph) == cudaSuccess && graph &&
            cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
            captured = true;
        else
            cudaGetLastError();
    }
    const int per_step = launches;
    if (captured) {
        for (int i = 0; i < nsteps; ++i)
            if (cudaGraphLaunch(exec, s) != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                cudaGraphDestroy(graph);
                return PE_ECUDA;
            }
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        note_launches(per_step * nsteps);
    } else {
        if (graph) cudaGraphDestroy(graph);
        launches = 0;
        for (int i = 0; i < nsteps; ++i) one_step();
        if (cudaGetLastError() != cudaSuccess) return PE_ECUDA;
        note_launches(launches);
    }
    if (loss && cudaMemcpyAsync(loss, h->loss, 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return PE_ECUDA;
    return PE_OK;
}

extern "C" PE_API int pe_mlp_sync_status(pe_mlp* h)
{
    if (!h) return PE_EINVAL;
    uint32_t st = 0;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PE_ECUDA;
    if (cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return PE_ECUDA;
    if (cudaMemset(h->status, 0, sizeof(st)) != cudaSuccess) return PE_ECUDA;
    return (st & PE_FLAG_TIMEOUT) ? PE_ETIMEOUT : PE_OK;
}

extern "C" PE_API int pe_mlp_info(const pe_mlp* h, int64_t* nparams, int64_t* steps_device_ptr, void** params,
                                  void** grads)
{
    if (!h) return PE_EINVAL;
    if (nparams) *nparams = h->nparams;
    if (steps_device_ptr) *steps_device_ptr = (int64_t)(uintptr_t)h->step;
    if (params) *params = h->p;
    if (grads) *grads = h->grad;
    return PE_OK;
}

// ------------------------------------------------------------------ gated surrogate step

namespace pe {
namespace {

using GateResult = pe_gate_result;

// Probe slope s_p and standard error sigma_i of every coefficient (line fit of the samples
// c_0..c_Ks at t_p = p dt), the gate decision, and on acceptance the leap
// c <- c_Ks + (dT - Ks dt) s_mlp (slope <- s_mlp). The estimated error is the relative change
// of the projected state, e = leap ||s_mlp - s_p|| / ||c_Ks||, accepted when
// e <= max(tol, nsig leap ||sigma|| / ||c_Ks||). One block, fixed summation order.
__global__ void __launch_bounds__(1024) k_gate(const double* __restrict__ cs, int Ks, int n, double dt, double dT,
                                              const double* __restrict__ s_mlp, double tol, double nsig,
                                              double* __restrict__ coarse, double* __restrict__ slope,
                                              GateResult* __restrict__ res)
{
    __shared__ double red[4][32];
    __shared__ int acc;
    const double tbar = 0.5 * Ks * dt;
    const double leap = dT - Ks * dt;
    double sxx = 0.0;
    for (int p = 0; p <= Ks; ++p) sxx += (p * dt - tbar) * (p * dt - tbar);
    double e2 = 0.0, n2 = 0.0, v2 = 0.0, c2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double ybar = 0.0;
        for (int p = 0; p <= Ks; ++p) ybar += cs[(size_t)p * n + i];
        ybar /= (double)(Ks + 1);
        double sxy = 0.0;
        for (int p = 0; p <= Ks; ++p) sxy += (p * dt - tbar) * (cs[(size_t)p * n + i] - ybar);
        const double sp = sxy / sxx;
        double r2 = 0.0;
        for (int p = 0; p <= Ks; ++p) {
            const double r = cs[(size_t)p * n + i] - (ybar + sp * (p * dt - tbar));
            r2 += r * r;
        }
        const double d = s_mlp[i] - sp;
        const double cl = cs[(size_t)Ks * n + i];
        e2 += d * d;
        n2 += sp * sp;
        v2 += r2 / (double)(Ks - 1) / sxx;
        c2 += cl * cl;
    }
    e2 = warp_sum(e2);
    n2 = warp_sum(n2);
    v2 = warp_sum(v2);
    c2 = warp_sum(c2);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][w] = e2;
        red[1][w] = n2;
        red[2][w] = v2;
        red[3][w] = c2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += red[0][k];
            b += red[1][k];
            c += red[2][k];
            d += red[3][k];
        }
        const double cn = sqrt(d);
        GateResult r;
        r.err = cn > 0.0 ? leap * sqrt(a) / cn : INFINITY;
        r.floor = fmax(tol, cn > 0.0 ? nsig * leap * sqrt(c) / cn : 0.0);
        r.norm = sqrt(b);
        r.sigma = sqrt(c);
        r.accepted = (r.err <= r.floor) ? 1 : 0;
        r.pad = 0;
        *res = r;
        acc = r.accepted;
    }
    __syncthreads();
    if (acc) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            coarse[i] = fma(leap, s_mlp[i], cs[(size_t)Ks * n + i]);
            slope[i] = s_mlp[i];
        }
    }
}

__global__ void k_to_f32(const double* __restrict__ src, int n, float* __restrict__ dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

}  // namespace
}  // namespace pe

extern "C" PE_API int pe_step_surrogate(pe_ctx* ctx, pe_mlp* h, const pe_gate_cfg* gc, pe_gate_stats* out)
{
    NvtxRange nvtx("pe_step_surrogate");
    if (!ctx || !h || !gc || !out) return PE_EINVAL;
    pe_ctx* x = ctx;
    const pe_config& c = x->cfg;
    const int n = 2 * x->nc, Ks = gc->K_probe;
    if (x->ps || x->pres) return PE_EINVAL;  // the surrogate maps the density and momentum coefficients
    if (x->te_active) return PE_EINVAL;  // an accepted leap would not project the electrons' energy
    if (h->dims[0] != n || h->dims[h->L] != n || Ks < 2 || Ks >= x->K_cur || !(gc->tol >= 0.0) ||
        !(gc->noise_sigmas >= 0.0))
        return PE_EINVAL;
    char* buf = x->arena + x->lay.offset[PE_BUF_SURROGATE];
    double* s_mlp = (double*)buf;
    GateResult* res = (GateResult*)(buf + al256(8 * (size_t)n));
    // the learned slope from the coarse state at the start of the step, on the context stream
    const cudaStream_t saved = h->stream;
    h->stream = x->stream;
    const int rc = pe_mlp_forward(h, x->coarse, 1, 1, s_mlp, 1);
    h->stream = saved;
    PE_TRY(rc);
    if (!x->fresh) PE_TRY(pe_lift(x));
    PE_TRY(pe_ctx_burst_range(x, 0, Ks, 1));
    PE_TRY(pe_coarsen(x->samples, Ks + 1, c.ncell, x->s_w, x->s_p, c.wavelet, x->nc, x->bin_shift, x->csamples,
                      x->stream));
    PE_TRY(pe_gate(x->csamples, Ks, n, c.dt, x->dT_cur, s_mlp, gc->tol, gc->noise_sigmas, x->coarse, x->slope, res,
                   x->stream));
    GateResult r;
    if (cudaMemcpyAsync(&r, res, sizeof(r), cudaMemcpyDeviceToHost, x->stream) != cudaSuccess ||
        cudaStreamSynchronize(x->stream) != cudaSuccess)
        return PE_ECUDA;
    memset(out, 0, sizeof(*out));
    out->accepted = r.accepted;
    out->err = r.err;
    out->floor = r.floor;
    out->norm = r.norm;
    out->sigma = r.sigma;
    if (r.accepted) {
        out->fine_steps = Ks;
        x->macro_steps += 1;
        x->coarse_state = 1;
        x->time += x->dT_cur;
        x->fresh = 0;
        return PE_OK;
    }
    out->fine_steps = x->K_cur;
    PE_TRY(pe_ctx_burst_range(x, Ks, x->K_cur, 1));
    PE_TRY(pe_restrict(x));
    return pe_project(x);
}

extern "C" PE_API int pe_gate(const double* samples, int32_t K_probe, int32_t ncoef, double dt, double dT,
                               const double* s_mlp, double tol, double noise_sigmas, double* coarse, double* slope,
                               pe_gate_result* result, void* stream)
{
    if (!samples || !s_mlp || !coarse || !slope || !result || K_probe < 2 || ncoef < 1 || !(dt > 0.0) ||
        !(tol >= 0.0) || !(noise_sigmas >= 0.0))
        return PE_EINVAL;
    k_gate<<<1, 1024, 0, (cudaStream_t)stream>>>(samples, K_probe, ncoef, dt, dT, s_mlp, tol, noise_sigmas, coarse,
                                                 slope, result);
    return launch_status(1);
}

extern "C" PE_API int pe_export_f32(pe_ctx* ctx, int32_t what, float* out)
{
    if (!ctx || !out || (what != 0 && what != 1)) return PE_EINVAL;
    const int n = (int)ctx->ncoef;
    k_to_f32<<<(n + 255) / 256, 256, 0, ctx->stream>>>(what ? ctx->slope : ctx->coarse, n, out);
    return launch_status(1);
}

namespace pe {
namespace {
__global__ void k_set_params(const float* __restrict__ src, int64_t n, float* __restrict__ p,
                             __nv_bfloat16* __restrict__ pb, __nv_bfloat16* __restrict__ pbT, WeightTable wt)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float w = src[i];
        p[i] = w;
        put_bf16(wt, i, w, pb, pbT);
    }
}
}  // namespace
}  // namespace pe

extern "C" PE_API int pe_mlp_set_params(pe_mlp* h, const float* params)
{
    if (!h || !params) return PE_EINVAL;
    k_set_params<<<2 * sm_count(), 256, 0, h->stream>>>(params, h->nparams, h->p, h->pb, h->pbT, h->wt);
    return launch_status(1);
}
