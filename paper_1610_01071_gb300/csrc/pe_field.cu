// Field solve: the nonlinear Poisson-Boltzmann equation of Section 3.3 (Eq.
// poisson2rescaled with lambda = n_0 = 1) on the nodes,
//   -(phi_{j+1} - 2 phi_j + phi_{j-1}) / dx^2 + g(phi_j) = n_j,   g = exp or 1 + phi,
// by Newton's method, followed by the centred field E_j = -(phi_{j+1} - phi_{j-1}) / (2 dx).
// Periodic grids wrap; bounded grids (Section 4.2's slab expansion) have walls at nodes 0
// and ncell-1 with phi' = 0 there (mirror ghosts phi_{-1} = phi_1, phi_{ncell} = phi_{ncell-2},
// hence E = 0 on the walls), and a wall node's density is twice its deposit (its CIC
// control volume is the half cell inside the domain).
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "pe_common.cuh"
#include "pe_internal.h"

namespace cg = cooperative_groups;

namespace pe {

constexpr int kClusterMinCells = 512;  // grids at least this large use the multi-SM solver

// ---------------------------------------------------------------------------------
// Production solver: one thread-block cluster of G blocks (G = 1 for small grids, up to
// 16 for large ones, one block per SM); block g owns the B = ncell / G nodes
// [g B, (g+1) B), one node per thread.
//
// Precision: phi, exp(phi), the Newton residual and the update are FP64; the Jacobian
// correction J d = -F is solved in FP32 on periodic grids. This is Newton's method with an
// inexact linear solve (mixed-precision iterative refinement): the FP64 residual drives the
// iteration, so it converges to the FP64 solution of the discrete equation, while the
// FP32 solve only bounds the final contraction rate (~ cond(J) 2^-24 per iteration).
// Bounded grids with vacuum regions have exp(phi) ~ 1e-6 there and cond(J) ~ 1e7: the FP32
// solve still contracts, but slowly (7 Newton iterations instead of 3 on an 8192-node slab from
// a warm start), so their linear solve runs in FP64 (template parameter T).
// On this GPU a dependent FP64 instruction costs ~100 cycles and the FP64 pipe retires
// ~2 lanes per cycle per SM, so FP64 is used only for per-node work, spread over many
// warps and SMs, and kept off the serial chains of the tridiagonal elimination.
//
// Linear solve (SPIKE-style partition): each block solves its B rows, with the two
// couplings to the neighbouring blocks moved to the right-hand side, by parallel
// cyclic reduction with three right-hand sides, x = y - g X_left - h X_right. The
// blocks' first and last unknowns then satisfy a cyclic block-tridiagonal system with
// 2x2 blocks; every block gathers it through distributed shared memory and solves it
// by block cyclic reduction. exp(phi) is evaluated once per solve and then carried
// multiplicatively, exp(phi + s d) = exp(phi) exp(s d), with a Taylor polynomial.

constexpr int kClusterMax = 16;

// exp(x) for |x| <= 2^-5 by its Taylor polynomial to degree 8 (relative error < 1e-18).
__device__ __forceinline__ double exp_small(double x)
{
    double p = 1.0 / 40320.0;
    p = fma(p, x, 1.0 / 5040.0);
    p = fma(p, x, 1.0 / 720.0);
    p = fma(p, x, 1.0 / 120.0);
    p = fma(p, x, 1.0 / 24.0);
    p = fma(p, x, 1.0 / 6.0);
    p = fma(p, x, 0.5);
    p = fma(p, x, 1.0);
    return fma(p, x, 1.0);
}

// Reciprocal for the elimination (and the 2x2 inverses of the boundary system): the fast FP32
// reciprocal (__fdividef, within 2 ulp for the diagonal magnitudes that occur here), or in
// FP64 two Newton-Raphson steps r <- r (2 - x r) from it (each step squares the relative
// error, 2^-22 -> 2^-44 -> 2^-88), which avoids the long division sequences on the
// reductions' serial chains. The FP32 solve is the inexact linear solve of a Newton
// iteration whose residual is FP64, so a 2-ulp reciprocal only changes its contraction rate.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x)
{
    double r = (double)__fdividef(1.0f, (float)x);
    r = r * fma(-x, r, 2.0);
    return r * fma(-x, r, 2.0);
}

template <typename T>
struct M2 {
    T a, b, c, d;  // [[a, b], [c, d]]
};
template <typename T>
__device__ __forceinline__ M2<T> mmul(M2<T> x, M2<T> y)
{
    return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
template <typename T>
__device__ __forceinline__ M2<T> msub(M2<T> x, M2<T> y)
{
    return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d};
}
template <typename T>
__device__ __forceinline__ M2<T> minv(M2<T> x)
{
    const T r = recip(x.a * x.d - x.b * x.c);
    return {x.d * r, -x.b * r, -x.c * r, x.a * r};
}
template <typename T>
__device__ __forceinline__ void mvec(M2<T> x, T v0, T v1, T* o0, T* o1)
{
    *o0 = x.a * v0 + x.b * v1;
    *o1 = x.c * v0 + x.d * v1;
}

// Block cyclic reduction of the G block rows (thread k < G owns row k) stored as full
// 2x2 matrices: L3[k] = {Mk(4), Dk(4), Pk(4), rk(2)}, row k: Mk z_{k-1} + Dk z_k + Pk z_{k+1} = rk.
// After the steps with stride G/2 every row couples only to itself. zsol gets z. (On a
// bounded grid the corner blocks M_0 and P_{G-1} are zero, so the wrap adds nothing.)
// The steps alternate between L3 and L3n, one barrier per step.
template <typename T>
__device__ void block_pcr(T* L3, T* L3n, T* zsol, int G)
{
    const int k = threadIdx.x;
    auto ld = [](const T* p) { return M2<T>{p[0], p[1], p[2], p[3]}; };
    auto st = [](T* p, M2<T> m) {
        p[0] = m.a;
        p[1] = m.b;
        p[2] = m.c;
        p[3] = m.d;
    };
    for (int s = 1; s <= G / 2; s <<= 1) {
        if (k < G) {
            const T* c = L3 + 14 * k;
            const T* lm = L3 + 14 * ((k - s + G) % G);
            const T* lp = L3 + 14 * ((k + s) % G);
            const M2<T> al = mmul(ld(c), minv(ld(lm + 4)));      // Mk D_{k-s}^-1
            const M2<T> ga = mmul(ld(c + 8), minv(ld(lp + 4)));  // Pk D_{k+s}^-1
            T* o = L3n + 14 * k;
            const M2<T> nM = mmul(al, ld(lm));
            const M2<T> nP = mmul(ga, ld(lp + 8));
            st(o, M2<T>{-nM.a, -nM.b, -nM.c, -nM.d});
            st(o + 8, M2<T>{-nP.a, -nP.b, -nP.c, -nP.d});
            st(o + 4, msub(msub(ld(c + 4), mmul(al, ld(lm + 8))), mmul(ga, ld(lp))));
            T ra0, ra1, rg0, rg1;
            mvec(al, lm[12], lm[13], &ra0, &ra1);
            mvec(ga, lp[12], lp[13], &rg0, &rg1);
            o[12] = c[12] - ra0 - rg0;
            o[13] = c[13] - ra1 - rg1;
        }
        __syncthreads();  // the next step reads L3n and overwrites L3, whose reads are done
        T* t = L3;
        L3 = L3n;
        L3n = t;
    }
    if (k < G) {
        const T* c = L3 + 14 * k;
        M2<T> Dt = ld(c + 4);
        const M2<T> Mm = ld(c), Pm = ld(c + 8);
        Dt = M2<T>{Dt.a + Mm.a + Pm.a, Dt.b + Mm.b + Pm.b, Dt.c + Mm.c + Pm.c, Dt.d + Mm.d + Pm.d};
        T z0, z1;
        mvec(minv(Dt), c[12], c[13], &z0, &z1);
        zsol[2 * k] = z0;
        zsol[2 * k + 1] = z1;
    }
    __syncthreads();
}

// Parameters of one field solve (one realisation).
struct FieldDesc {
    const long long* rho;
    double* phi;
    double* E;
    float* Ef;
    int* diag;
    uint32_t* status;
    double dx, nscale, tol;
    int ncell, mode, maxit, walls;  // walls: 1 for a bounded grid
    // Newton start: phi_prev (may be null) keeps the solution before the current one; with
    // extrap the start is the linear extrapolation 2 phi - phi_prev (solves one fine step apart)
    double* phi_prev;
    int extrap, pad2;
};

// Solver body for the realisation of this cluster: B = ncell / G nodes per block, one per
// thread; threads at or beyond B (a batched launch sized for a larger grid) only take
// part in the barriers. T is the precision of the linear solve.
template <typename T>
__device__ __forceinline__ void newton_body(const FieldDesc& d, cg::cluster_group& cluster)
{
    extern __shared__ double sh[];
    const int G = (int)cluster.num_blocks();
    const int g = (int)cluster.block_rank();
    const int ncell = d.ncell;
    const int B = ncell / G;
    const int i = threadIdx.x;
    const bool act = i < B;
    const long long* rho = d.rho;
    double* phi = d.phi;
    const double dx = d.dx, nscale = d.nscale, tol = d.tol;
    const int mode = d.mode, maxit = d.maxit;
    double* ph = sh;                             // [B + 2]
    double* mymax = ph + B + 2;                  // [1]
    // two sets of the seven row arrays (A, Bd, C, D, Gs, Hs, Rb: sub-, main and super-diagonal,
    // right-hand side, the two coupling columns, reciprocal of the diagonal); the reduction
    // steps alternate between them
    T* rows = reinterpret_cast<T*>(mymax + 1);   // [2][7][B]
    T* red = rows + 14 * B;  // [32]
    T* mine = red + 32;  // [6]
    T* L3 = mine + 8;    // [G][14]
    T* L3n = L3 + 14 * G;
    T* zsol = L3n + 14 * G;  // [2G]

    const int mask = ncell - 1;
    const int j = g * B + (act ? i : 0);
    const bool walls = d.walls != 0;
    const bool wl = walls && j == 0, wr = walls && j == ncell - 1;  // this thread's node is a wall
    const double inv_dx2 = 1.0 / (dx * dx);
    const T o = (T)(-inv_dx2);
    const bool boltz = (mode == PE_POISSON_BOLTZMANN);
    const double nj = act ? (double)__ldg(rho + j) * nscale * ((wl || wr) ? 2.0 : 1.0) : 0.0;
    double pj = act ? phi[j] : 0.0;
    if (d.phi_prev && act) {
        const double pp = d.phi_prev[j];
        d.phi_prev[j] = pj;
        if (d.extrap) {
            pj = 2.0 * pj - pp;
            phi[j] = pj;
        }
    }
    if (d.phi_prev && d.extrap) {  // extrapolated starts visible to the neighbouring blocks' halos
        __threadfence();
        cluster.sync();
    }
    double gj = boltz ? exp(pj) : 1.0 + pj;
    // Halo ph[0], ph[B + 1]: the neighbouring blocks' boundary nodes, read once and then
    // advanced here with the same damped updates their owners apply (the boundary unknowns of
    // the reduced system, known to every block), so they stay bit-identical to the owners'
    // values. Only threads 0 and B - 1 read and write them.
    if (act && i == 0) ph[0] = phi[(g * B - 1) & mask];
    if (act && i == B - 1) ph[B + 1] = phi[(g * B + B) & mask];

    int it = 0;
    bool converged = false;
    for (it = 0; it < maxit; ++it) {
        // ---- FP64 residual with the halo from the neighbouring blocks (mirror ghosts at walls)
        if (act) ph[i + 1] = pj;
        __syncthreads();
        T* A = rows;
        T* Bd = A + B;
        T* C = Bd + B;
        T* D = C + B;
        T* Gs = D + B;
        T* Hs = Gs + B;
        T* Rb = Hs + B;
        if (act) {
            const double pl = wl ? ph[i + 2] : ph[i], pr = wr ? ph[i] : ph[i + 2];
            const double lap = (pl - 2.0 * pj + pr) * inv_dx2;
            A[i] = (i == 0) ? T(0) : (wr ? T(2) * o : o);
            C[i] = (i == B - 1) ? T(0) : (wl ? T(2) * o : o);
            Bd[i] = (T)(2.0 * inv_dx2 + (boltz ? gj : 1.0));
            Rb[i] = recip(Bd[i]);
            D[i] = (T)(lap - gj + nj);  // -F_j
            Gs[i] = (i == 0 && !wl) ? o : T(0);
            Hs[i] = (i == B - 1 && !wr) ? o : T(0);
        }
        __syncthreads();
        // ---- parallel cyclic reduction of the block rows, three right-hand sides; step s reads
        // one row set and writes the other, so one barrier per step separates the steps
        for (int s = 1; s < B; s <<= 1) {
            T* nx = (A == rows) ? rows + 7 * B : rows;  // the other row set
            const int im = act ? i - s : -1, ip = act ? i + s : B;
            const T al = (im >= 0) ? A[i] * Rb[im] : T(0);
            const T ga = (ip < B) ? C[i] * Rb[ip] : T(0);
            const T nA = (im >= 0) ? -al * A[im] : T(0);
            const T nC = (ip < B) ? -ga * C[ip] : T(0);
            T nB = act ? Bd[i] : T(0), nD = act ? D[i] : T(0), nG = act ? Gs[i] : T(0), nH = act ? Hs[i] : T(0);
            if (im >= 0) {
                nB -= al * C[im];
                nD -= al * D[im];
                nG -= al * Gs[im];
                nH -= al * Hs[im];
            }
            if (ip < B) {
                nB -= ga * A[ip];
                nD -= ga * D[ip];
                nG -= ga * Gs[ip];
                nH -= ga * Hs[ip];
            }
            A = nx;
            Bd = nx + B;
            C = nx + 2 * B;
            D = nx + 3 * B;
            Gs = nx + 4 * B;
            Hs = nx + 5 * B;
            Rb = nx + 6 * B;
            if (act) {
                A[i] = nA;
                C[i] = nC;
                Bd[i] = nB;
                Rb[i] = recip(nB);
                D[i] = nD;
                Gs[i] = nG;
                Hs[i] = nH;
            }
            __syncthreads();
        }
        const T rb = act ? Rb[i] : T(0);
        const T y = act ? D[i] * rb : T(0), gsp = act ? Gs[i] * rb : T(0),
                hsp = act ? Hs[i] * rb : T(0);  // x = y - g X_left - h X_right
        if (i == 0) {
            mine[0] = y;
            mine[1] = gsp;
            mine[2] = hsp;
        }
        if (i == B - 1) {
            mine[3] = y;
            mine[4] = gsp;
            mine[5] = hsp;
        }
        cluster.sync();  // #1: every block's boundary rows are visible
        // ---- cyclic block-tridiagonal system of the blocks' (first, last) unknowns
        if (i < G) {
            const T* rem = cluster.map_shared_rank(mine, i);
            T* r = L3 + 14 * i;
            // F_k + g0 L_{k-1} + h0 F_{k+1} = y0 ;  L_k + gB L_{k-1} + hB F_{k+1} = yB
            r[0] = T(0); r[1] = rem[1]; r[2] = T(0); r[3] = rem[4];     // M: picks L_{k-1}
            r[4] = T(1); r[5] = T(0);   r[6] = T(0); r[7] = T(1);       // D = I
            r[8] = rem[2]; r[9] = T(0); r[10] = rem[5]; r[11] = T(0);   // P: picks F_{k+1}
            r[12] = rem[0]; r[13] = rem[3];
        }
        __syncthreads();
        block_pcr<T>(L3, L3n, zsol, G);
        const T Xl = zsol[2 * ((g - 1 + G) % G) + 1];  // previous block's last unknown
        const T Xr = zsol[2 * ((g + 1) % G)];          // next block's first unknown
        // the block's own first and last unknowns are those of the reduced system (equal to
        // y - g X_left - h X_right up to rounding), so that the neighbours' halos follow them
        const T dlt = (i == 0) ? zsol[2 * g] : ((i == B - 1) ? zsol[2 * g + 1] : y - gsp * Xl - hsp * Xr);
        // ---- global max |update| (damping and convergence)
        T mloc = act ? (dlt < T(0) ? -dlt : dlt) : T(0);
        for (int off = 16; off > 0; off >>= 1) {
            const T oth = __shfl_xor_sync(0xffffffffu, mloc, off);
            mloc = oth > mloc ? oth : mloc;
        }
        if ((i & 31) == 0) red[i >> 5] = mloc;
        __syncthreads();
        if (i < 32) {
            T v = (i < ((blockDim.x + 31) >> 5)) ? red[i] : T(0);
            for (int off = 16; off > 0; off >>= 1) {
                const T oth = __shfl_xor_sync(0xffffffffu, v, off);
                v = oth > v ? oth : v;
            }
            if (i == 0) *mymax = (double)v;
        }
        // #2: block maxima visible; level-3 rows no longer read. The next iteration rewrites
        // mine and mymax only after its barrier #1, which every block reaches after reading them.
        cluster.sync();
        double m = 0.0;
        for (int k = 0; k < G; ++k) m = fmax(m, *cluster.map_shared_rank(mymax, k));
        const double scale = (m > 2.0) ? 2.0 / m : 1.0;
        const double x = act ? scale * (double)dlt : 0.0;
        pj += x;
        if (act) phi[j] = pj;
        if (act && i == 0) ph[0] += scale * (double)Xl;
        if (act && i == B - 1) ph[B + 1] += scale * (double)Xr;
        if (boltz)
            gj = (fabs(x) <= 0.03125) ? gj * exp_small(x) : exp(pj);
        else
            gj = 1.0 + pj;
        if (m < tol) {
            converged = true;
            ++it;
            break;
        }
    }
    if (act) ph[i + 1] = pj;
    __syncthreads();
    if (act) {
        const double e = (wl || wr) ? 0.0 : -(ph[i + 2] - ph[i]) * (0.5 / dx);
        d.E[j] = e;
        d.Ef[j] = (float)e;
    }
    if (g == 0 && i == 0) {
        if (d.diag) {
            d.diag[0] = it;
            d.diag[1] = converged ? 1 : 0;
            d.diag[2] = G;
            d.diag[3] = B;
        }
        if (!converged) raise_flag(d.status, PE_FLAG_NOCONV);
    }
    cluster.sync();  // no block leaves while another may still read its mymax
}

template <typename T>
__global__ void __launch_bounds__(1024) k_newton_cluster(FieldDesc d)
{
    cg::cluster_group cluster = cg::this_cluster();
    newton_body<T>(d, cluster);
}

// One cluster per realisation: cluster c solves descs[c]; extrap applies to every realisation.
template <typename T>
__global__ void __launch_bounds__(1024) k_newton_batch(const FieldDesc* descs, int extrap)
{
    cg::cluster_group cluster = cg::this_cluster();
    FieldDesc d = descs[blockIdx.x / cluster.num_blocks()];
    d.extrap = extrap;
    newton_body<T>(d, cluster);
}

static int cluster_size_for(int ncell)
{
    // largest cluster (<= 16) the device accepts for this kernel; 0 if none
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        cudaFuncSetAttribute((const void*)k_newton_cluster<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute((const void*)k_newton_cluster<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kClusterMax;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(kClusterMax);
        cfg.blockDim = dim3(512);
        cfg.dynamicSmemBytes = 16 * 1024;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int size = 0;
        if (cudaOccupancyMaxPotentialClusterSize(&size, (const void*)k_newton_cluster<float>, &cfg) != cudaSuccess)
            size = 8;
        cudaGetLastError();
        int p = 1;
        while (p * 2 <= size && p * 2 <= kClusterMax) p *= 2;
        cached[dev] = p;
    }
    int G = cached[dev];
    while (G > 1 && ncell / G < 32) G >>= 1;  // at least 32 nodes per block
    if (ncell < kClusterMinCells) G = 1;
    while (ncell / G > 1024) G <<= 1;          // at most 1024 nodes (threads) per block
    return G <= kClusterMax ? G : 0;
}

size_t newton_smem_bytes(int B, int G, bool fp64)
{
    const size_t t = fp64 ? sizeof(double) : sizeof(float);
    return sizeof(double) * ((size_t)B + 3) + t * (14 * (size_t)B + 32 + 8 + 30 * (size_t)G) + 16;
}

static cudaLaunchConfig_t cluster_config(cudaLaunchAttribute* attr, int G, int nclusters, int block, size_t smem,
                                         cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(G * nclusters);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

static int launch_newton_cluster(int G, const long long* rho, int ncell, double dx, double nscale, int mode,
                                 int walls, double tol, int maxit, double* phi, double* E, float* Ef, int* diag,
                                 uint32_t* status, double* phi_prev, int extrap, cudaStream_t s)
{
    const int B = ncell / G;  // one node per thread
    if (B > 1024 || B < 2) return PE_EINVAL;
    const bool fp64 = walls != 0;
    const size_t smem = newton_smem_bytes(B, G, fp64);
    const void* k = fp64 ? (const void*)k_newton_cluster<double> : (const void*)k_newton_cluster<float>;
    if (ensure_smem(k, smem) != PE_OK) return PE_ECUDA;
    FieldDesc d{rho, phi, E, Ef, diag, status, dx, nscale, tol, ncell, mode, maxit, walls ? 1 : 0, phi_prev,
                extrap ? 1 : 0, 0};
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(attr, G, 1, B, smem, s);
    const cudaError_t e = fp64 ? cudaLaunchKernelEx(&cfg, k_newton_cluster<double>, d)
                               : cudaLaunchKernelEx(&cfg, k_newton_cluster<float>, d);
    if (e != cudaSuccess) return PE_ECUDA;
    return launch_status();
}

int newton_cluster_size(int ncell) { return cluster_size_for(ncell); }

// Batched field solves: descs[R] on the device, every grid with the same cluster size G;
// fp64: the linear solves run in FP64 (needed when any grid is bounded).
int launch_newton_batch(const void* descs, int R, int G, int max_ncell, bool fp64, bool extrap, cudaStream_t s)
{
    const int B = max_ncell / G;
    if (B > 1024 || B < 2 || R < 1) return PE_EINVAL;
    const size_t smem = newton_smem_bytes(B, G, fp64);
    const void* k = fp64 ? (const void*)k_newton_batch<double> : (const void*)k_newton_batch<float>;
    if (ensure_smem(k, smem) != PE_OK) return PE_ECUDA;
    static bool nonportable[2][64] = {{false}};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PE_ECUDA;
    if (G > 8 && !nonportable[fp64][dev]) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            return PE_ECUDA;
        nonportable[fp64][dev] = true;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(attr, G, R, B, smem, s);
    const FieldDesc* dd = static_cast<const FieldDesc*>(descs);
    const int ex = extrap ? 1 : 0;
    const cudaError_t e = fp64 ? cudaLaunchKernelEx(&cfg, k_newton_batch<double>, dd, ex)
                               : cudaLaunchKernelEx(&cfg, k_newton_batch<float>, dd, ex);
    if (e != cudaSuccess) return PE_ECUDA;
    return launch_status();
}

size_t field_desc_size() { return sizeof(FieldDesc); }

void make_field_desc(void* out, const int64_t* rho, int ncell, double dx, int s_w, int mode, int walls, double tol,
                     int maxit, double* phi, double* E, float* Ef, int32_t* diag, uint32_t* status, double* phi_prev)
{
    FieldDesc d{reinterpret_cast<const long long*>(rho), phi, E, Ef, diag, status, dx, ldexp(1.0, -(s_w + 24)), tol,
                ncell, mode, maxit, walls ? 1 : 0, phi_prev, 0, 0};
    memcpy(out, &d, sizeof(d));
}

}  // namespace pe

using namespace pe;

namespace pe {
// Field solve with a Newton start from the solution history (context path): phi_prev keeps the
// solution before the current one, extrap selects the extrapolated start.
int field_solve_history(const int64_t* rho_fx, int ncell, double dx, int s_w, int mode, int boundary, double tol,
                        int maxit, double* phi, double* E, float* Ef, int32_t* diag, uint32_t* status,
                        double* phi_prev, int extrap, cudaStream_t s)
{
    if (!is_pow2(ncell) || ncell < 8 || !rho_fx || !phi || !E || !Ef || !(dx > 0.0) || maxit < 0) return PE_EINVAL;
    if (mode != PE_POISSON_BOLTZMANN && mode != PE_POISSON_LINEARIZED) return PE_EINVAL;
    if (boundary != PE_BOUNDARY_PERIODIC && boundary != PE_BOUNDARY_ABSORBING) return PE_EINVAL;
    const double nscale = ldexp(1.0, -(s_w + 24));
    if (ncell > kFullGridMax) return PE_EINVAL;
    const int G = cluster_size_for(ncell);
    if (G < 1) return PE_EINVAL;
    return launch_newton_cluster(G, reinterpret_cast<const long long*>(rho_fx), ncell, dx, nscale, mode,
                                 boundary == PE_BOUNDARY_ABSORBING, tol, maxit, phi, E, Ef, diag, status, phi_prev,
                                 extrap, s);
}
}  // namespace pe

// ---------------------------------------------------------------------------------
// Kinetic electrons (Section 4.1's two-species bursts): periodic Poisson equation for the
// net charge, one block of 256 threads; thread t owns the m = ncell / 256 (at least 1)
// consecutive nodes j0 = t m ... The net charge and then the face fields and potentials live
// in shared memory; every sum runs node by node within a thread, then lane by lane and warp
// by warp, in a fixed order. FP64 throughput of one SM bounds this kernel, so each node costs
// a handful of FP64 operations and the block-wide sums run over 256 partial sums.

constexpr int kPoissonThreads = 256;

// Exclusive prefix sum over the block of one value per thread, and the block total.
// wsum: 32 shared slots. Every thread of the block calls it.
template <typename V>
__device__ __forceinline__ V block_exclusive_scan(V x, V* total, V* wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    V incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        V s = lane < nw ? wsum[lane] : V(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const V y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const V base = w > 0 ? wsum[w - 1] : V(0);
    *total = wsum[nw - 1];
    __syncthreads();  // wsum is reused by the next call
    return base + incl - x;
}

__global__ void __launch_bounds__(kPoissonThreads) k_poisson_periodic(const long long* rho_i, const long long* rho_e,
                                                                      int n, double dx, double nscale, double* phi,
                                                                      double* E, float* Ef)
{
    extern __shared__ double psh[];
    double* F = psh;      // [n]: net charge, then the face fields F_{j+1/2}
    double* P = psh + n;  // [n]: potential before its mean is removed
    __shared__ double wd[32];
    const int t = threadIdx.x;
    const int m = n >= (int)blockDim.x ? n / (int)blockDim.x : 1;
    const int nt = n / m;  // threads that own nodes
    const int j0 = t * m;
    const bool act = t < nt;
    // net charge per node (the int64 difference of the deposits is exact), and its sum
    double s = 0.0;
    if (act)
        for (int k = 0; k < m; ++k) {
            const double q = (double)(__ldg(rho_i + j0 + k) - __ldg(rho_e + j0 + k));
            F[j0 + k] = q;
            s += q;
        }
    double tot;
    const double off = block_exclusive_scan(s, &tot, wd);
    // face fields before the gauge: F_{j+1/2} - F_{-1/2} = dx nscale (S_j - (j + 1) <S>)
    const double mean = tot / n, c = dx * nscale;
    double fs = 0.0;
    if (act) {
        double acc = off;
        for (int k = 0; k < m; ++k) {
            acc += F[j0 + k];
            const double f = c * (acc - (double)(j0 + k + 1) * mean);
            F[j0 + k] = f;
            fs += f;
        }
    }
    double ftot;
    (void)block_exclusive_scan(fs, &ftot, wd);
    const double gauge = ftot / n;  // the faces of a periodic phi sum to zero
    double ps = 0.0;
    if (act)
        for (int k = 0; k < m; ++k) {
            const double f = F[j0 + k] - gauge;
            F[j0 + k] = f;
            ps += f;
        }
    // phi_0 = 0, phi_{j+1} = phi_j - dx F_{j+1/2}
    double ptot;
    const double poff = block_exclusive_scan(ps, &ptot, wd);
    double psum = 0.0;
    if (act) {
        double p = -dx * poff;
        for (int k = 0; k < m; ++k) {
            P[j0 + k] = p;
            psum += p;
            p -= dx * F[j0 + k];
        }
    }
    double pt;
    (void)block_exclusive_scan(psum, &pt, wd);  // its barriers also publish F to the neighbours
    const double pmean = pt / n;
    if (act)
        for (int k = 0; k < m; ++k) {
            const int j = j0 + k;
            const double e = 0.5 * (F[j] + F[j > 0 ? j - 1 : n - 1]);  // E_j = (F_{j+1/2} + F_{j-1/2}) / 2
            E[j] = e;
            Ef[j] = (float)e;
            phi[j] = P[j] - pmean;
        }
}

__global__ void k_boltzmann_profile(const double* phi, const long long* mom, int n, double vscale, float* nprof,
                                    float* uprof)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        nprof[j] = (float)exp(phi[j]);
        if (uprof) {
            float u = 0.0f;
            if (mom) {  // V_e = V_i: the ions' momentum over their density at the node
                const long long d = mom[j], m = mom[n + j];
                if (d > 0) u = (float)((double)m / (double)d * vscale);
            }
            uprof[j] = u;
        }
    }
}

extern "C" PE_API int pe_field_kinetic(const int64_t* rho_i, const int64_t* rho_e, int32_t ncell, double dx,
                                       int32_t s_w, double* phi, double* E, float* Ef, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || ncell > kFullGridMax || !rho_i || !rho_e || !phi || !E || !Ef ||
        !(dx > 0.0))
        return PE_EINVAL;
    const size_t smem = 2 * sizeof(double) * (size_t)ncell;
    if (ensure_smem((const void*)k_poisson_periodic, smem) != PE_OK) return PE_ECUDA;
    k_poisson_periodic<<<1, kPoissonThreads, smem, (cudaStream_t)stream>>>(
        reinterpret_cast<const long long*>(rho_i), reinterpret_cast<const long long*>(rho_e), ncell, dx,
        ldexp(1.0, -(s_w + 24)), phi, E, Ef);
    return launch_status();
}

extern "C" PE_API int pe_boltzmann_profile(const double* phi, const int64_t* ion_moments, int32_t s_w, int32_t s_p,
                                           int32_t ncell, float* n_prof, float* u_prof, void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || ncell > kFullGridMax || !phi || !n_prof || (ion_moments && !u_prof))
        return PE_EINVAL;
    k_boltzmann_profile<<<(ncell + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        phi, reinterpret_cast<const long long*>(ion_moments), ncell, ldexp(1.0, s_w - s_p), n_prof, u_prof);
    return launch_status();
}

extern "C" PE_API int pe_field_ex(const int64_t* rho_fx, int32_t ncell, double dx, int32_t s_w, int32_t mode,
                                  int32_t boundary, double tol, int32_t maxit, double* phi, double* E, float* Ef,
                                  int32_t* diag, uint32_t* status, void* stream)
{
    return field_solve_history(rho_fx, ncell, dx, s_w, mode, boundary, tol, maxit, phi, E, Ef, diag, status, nullptr,
                               0, (cudaStream_t)stream);
}

extern "C" PE_API int pe_field(const int64_t* rho_fx, int32_t ncell, double dx, int32_t s_w, int32_t mode, double tol,
                               int32_t maxit, double* phi, double* E, float* Ef, int32_t* diag, uint32_t* status,
                               void* stream)
{
    return pe_field_ex(rho_fx, ncell, dx, s_w, mode, PE_BOUNDARY_PERIODIC, tol, maxit, phi, E, Ef, diag, status,
                       stream);
}
