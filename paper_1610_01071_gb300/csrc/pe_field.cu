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
// a warm start); it remains the faster solve (kWallsJacobianFP64 selects the FP64 elimination,
// template parameter T).
// On this GPU a dependent FP64 instruction costs ~100 cycles and the FP64 pipe retires
// ~2 lanes per cycle per SM, so FP64 is used only for per-node work, spread over many
// warps and SMs, and kept off the serial chains of the tridiagonal elimination.
//
// Linear solve (nested separators, scalar tridiagonal systems only): the last row of every
// warp is a separator, and the last row of every block is a separator of the cluster. Each
// warp solves its other rows (its interior) by parallel cyclic reduction with register
// shuffles, with the couplings to the two separators around it moved to two extra right-hand
// sides (x = y - g S_left - h S_right). Substituting the interiors next to a separator into
// its row leaves a scalar tridiagonal system over the separators: one warp of the block solves
// the block's warp separators in terms of the two block separators around them, and one warp
// of every block solves the cyclic system of the cluster's block separators, whose rows every
// block pushes into every other block's shared memory before the cluster barrier. exp(phi) is
// evaluated once per solve and then carried multiplicatively, exp(phi + s d) = exp(phi)
// exp(s d), with a Taylor polynomial.
//
// Stopping: besides max |update| < tol, the iteration stops before a linear solve when the
// residual already bounds the next update below tol. The Jacobian J = L + diag(g'(phi)) has
// L symmetric with zero row sums and non-positive off-diagonals (periodic or mirror-wall
// rows), so J is an M-matrix with row sums g'(phi_j) and ||J^-1||_inf <= 1 / min_j g'(phi_j):
// the next Newton update is at most max|F| / min g' in every component.

constexpr int kClusterMax = 16;
constexpr int kNewtonMaxThreads = 512;  // nodes (threads) per block: 16 blocks cover the largest grid

// exp(x) for |x| <= 2^-5 by its Taylor polynomial to degree 8 (relative error < 1e-18),
// evaluated by Estrin's scheme: a dependent FP64 operation costs ~100 cycles here, and the
// scheme's dependency depth is 5 instead of the 9 of Horner's rule.
__device__ __forceinline__ double exp_small(double x)
{
    const double x2 = x * x, x4 = x2 * x2;
    const double p01 = 1.0 + x, p23 = fma(x, 1.0 / 6.0, 0.5), p45 = fma(x, 1.0 / 120.0, 1.0 / 24.0),
                 p67 = fma(x, 1.0 / 5040.0, 1.0 / 720.0);
    const double lo = fma(x2, p23, p01), hi = fma(x2, p67, p45);
    return fma(x4, fma(x4, 1.0 / 40320.0, hi), lo);
}

// exp(x) for |x| <= 2^-10 to degree 4 (relative error < 1e-17), dependency depth 3.
__device__ __forceinline__ double exp_tiny(double x)
{
    const double x2 = x * x;
    return fma(x2, fma(x2, 1.0 / 24.0, fma(x, 1.0 / 6.0, 0.5)), 1.0 + x);
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

// Parallel cyclic reduction of a scalar tridiagonal system held by lanes 0 .. n-1 of the
// calling warp (n a power of two, <= 32; all 32 lanes call it; a lane without a row holds the
// identity row). Row k: a x_{k-1} + b x_k + c x_{k+1} = r (three right-hand sides r0, r1,
// r2). cyclic: rows couple to (k +- 1) mod n; else the chain ends at 0 and n - 1. Returns
// x_k for each right-hand side (after the last step of a cyclic system its remaining
// couplings reach the row itself and are folded into the diagonal).
template <typename T>
__device__ __forceinline__ void warp_scalar_pcr(T a, T b, T c, T r0, T r1, T r2, int n, bool cyclic, T& x0, T& x1,
                                                T& x2)
{
    const int k = threadIdx.x & 31;
    for (int s = 1; s < n; s <<= 1) {
        const int km = (k - s + n) % n, kp = (k + s) % n;
        const T am = __shfl_sync(0xFFFFFFFFu, a, km), bm = __shfl_sync(0xFFFFFFFFu, b, km);
        const T cm = __shfl_sync(0xFFFFFFFFu, c, km), q0m = __shfl_sync(0xFFFFFFFFu, r0, km);
        const T q1m = __shfl_sync(0xFFFFFFFFu, r1, km), q2m = __shfl_sync(0xFFFFFFFFu, r2, km);
        const T ap = __shfl_sync(0xFFFFFFFFu, a, kp), bp = __shfl_sync(0xFFFFFFFFu, b, kp);
        const T cp = __shfl_sync(0xFFFFFFFFu, c, kp), q0p = __shfl_sync(0xFFFFFFFFu, r0, kp);
        const T q1p = __shfl_sync(0xFFFFFFFFu, r1, kp), q2p = __shfl_sync(0xFFFFFFFFu, r2, kp);
        const bool hm = k < n && (cyclic || k >= s), hp = k < n && (cyclic || k + s < n);
        const T al = hm ? a * recip(bm) : T(0);
        const T ga = hp ? c * recip(bp) : T(0);
        a = -al * am;
        c = -ga * cp;
        b = b - al * cm - ga * ap;
        r0 = r0 - al * q0m - ga * q0p;
        r1 = r1 - al * q1m - ga * q1p;
        r2 = r2 - al * q2m - ga * q2p;
    }
    const T bt = cyclic ? a + b + c : b;
    const T rb = recip(bt);
    x0 = r0 * rb;
    x1 = r1 * rb;
    x2 = r2 * rb;
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

// Parallel cyclic reduction of the 32 rows held by the calling warp (one per lane; a lane
// without a row holds the identity row). Row i: a x_{i-1} + b x_i + c x_{i+1} = d, with the
// couplings to rows outside the warp already moved to the columns gc (left) and hc (right).
// On return every row is decoupled: b x_i = d - gc X_left - hc X_right.
template <typename T>
__device__ __forceinline__ void warp_pcr(T& a, T& b, T& c, T& d, T& gc, T& hc)
{
    const int lane = threadIdx.x & 31;
    T rb = recip(b);
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const T am = __shfl_up_sync(0xFFFFFFFFu, a, s), cm = __shfl_up_sync(0xFFFFFFFFu, c, s);
        const T dm = __shfl_up_sync(0xFFFFFFFFu, d, s), gm = __shfl_up_sync(0xFFFFFFFFu, gc, s);
        const T hm = __shfl_up_sync(0xFFFFFFFFu, hc, s), rm = __shfl_up_sync(0xFFFFFFFFu, rb, s);
        const T ap = __shfl_down_sync(0xFFFFFFFFu, a, s), cp = __shfl_down_sync(0xFFFFFFFFu, c, s);
        const T dp = __shfl_down_sync(0xFFFFFFFFu, d, s), gp = __shfl_down_sync(0xFFFFFFFFu, gc, s);
        const T hp = __shfl_down_sync(0xFFFFFFFFu, hc, s), rp = __shfl_down_sync(0xFFFFFFFFu, rb, s);
        const T al = (lane >= s) ? a * rm : T(0);
        const T ga = (lane + s < 32) ? c * rp : T(0);
        a = -al * am;
        c = -ga * cp;
        b = b - al * cm - ga * ap;
        d = d - al * dm - ga * dp;
        gc = gc - al * gm - ga * gp;
        hc = hc - al * hm - ga * hp;
        rb = recip(b);
    }
    d *= rb;
    gc *= rb;
    hc *= rb;
}

// Values every block pushes into every block's shared memory before the first cluster barrier
// of a Newton iteration (slot k holds block k's): its first interior row and its last interior
// row in terms of the block separators around it (x = y - g s_{k-1} - h s_k), its separator
// row (a, b, c, d of row s_k), and its residual bound (max |F|, min g').
constexpr int kPush = 12;

// A block's first interior row from its pushed values, given the separators around the block
// (the owner and its left neighbour evaluate this same function, so the neighbour's halo stays
// bit-identical to the owner's node).
template <typename T>
__device__ __forceinline__ T edge_row(const T* r, T s_left, T s_right)
{
    return r[0] - r[1] * s_left - r[2] * s_right;
}

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
    const int i = threadIdx.x, lane = i & 31, w = i >> 5;
    const int W = (B + 31) >> 5;  // warps holding rows
    const bool act = i < B;
    const long long* rho = d.rho;
    double* phi = d.phi;
    const double dx = d.dx, nscale = d.nscale, tol = d.tol;
    const int mode = d.mode, maxit = d.maxit;
    double* ph = sh;                              // [B + 2] phi with the halo
    T* recv = reinterpret_cast<T*>(ph + B + 2);   // [G][kPush] rows pushed by every block
    T* recvm = recv + kPush * G;                  // [G] every block's max |update|
    T* wedge = recvm + G;                         // [W][8]: warp w's first interior row (y, g, h),
                                                  // last interior row (y, g, h), max|F|, min g'
    T* wsep = wedge + 8 * W;                      // [W][4]: warp w's separator row (a, b, c, d)
    T* lev2 = wsep + 4 * W;                       // [W][3]: S_w = Y - Gc s_{k-1} - Hc s_k
    T* svals = lev2 + 3 * W;                      // [G]: every block separator s_k
    T* wmax = svals + G;                          // [32]: per-warp max |update|
    T* flag = wmax + 32;                          // [1]: converged by the residual bound

    const int mask = ncell - 1;
    const int j = g * B + (act ? i : 0);
    const bool walls = d.walls != 0;
    const bool wl = walls && j == 0, wr = walls && j == ncell - 1;  // this thread's node is a wall
    const double inv_dx2 = 1.0 / (dx * dx);
    const T o = (T)(-inv_dx2);
    const bool boltz = (mode == PE_POISSON_BOLTZMANN);
    const double nj = act ? (double)__ldg(rho + j) * nscale * ((wl || wr) ? 2.0 : 1.0) : 0.0;
    // Newton start: phi, or with extrap the extrapolation 2 phi - phi_prev of the last two
    // solutions. Nothing is written to phi or phi_prev before the first cluster barrier, so the
    // halo nodes below (the neighbouring blocks' boundary nodes) are read unchanged and
    // extrapolated here with the owners' arithmetic.
    const bool hist = d.phi_prev != nullptr, ex = hist && d.extrap;
    const double p_old = act ? phi[j] : 0.0;
    double pj = (act && ex) ? 2.0 * p_old - d.phi_prev[j] : p_old;
    double gj = boltz ? exp(pj) : 1.0 + pj;
    // Halo ph[0], ph[B + 1]: read once and then advanced here with the same damped updates their
    // owners apply (values of the reduced systems, known to every block), so they stay
    // bit-identical to the owners' values. Only threads 0 and B - 1 read and write them.
    if (act && (i == 0 || i == B - 1)) {
        const int h = (i == 0) ? ((g * B - 1) & mask) : ((g * B + B) & mask);
        const double v = phi[h];
        ph[i == 0 ? 0 : B + 1] = ex ? 2.0 * v - d.phi_prev[h] : v;
    }
    bool hist_written = false;
    const int sep = (w == W - 1) ? ((B - 1) & 31) : 31;  // this warp's separator lane

    int it = 0;
    bool converged = false;
    for (it = 0; it < maxit; ++it) {
        // ---- FP64 residual with the halo from the neighbouring blocks (mirror ghosts at walls)
        if (act) ph[i + 1] = pj;
        __syncthreads();
        T a = T(0), b = T(1), c = T(0), rhs = T(0), gc = T(0), hc = T(0);
        float fabs_r = 0.f, gmin = 3.0e38f;
        T sa = T(0), sb = T(1), sc = T(0), sd = T(0);  // the separator's row (lane sep)
        if (act) {
            const double pl = wl ? ph[i + 2] : ph[i], pr = wr ? ph[i] : ph[i + 2];
            const double lap = (pl - 2.0 * pj + pr) * inv_dx2;
            const double r = lap - gj + nj;  // -F_j
            fabs_r = (float)fabs(r);
            gmin = boltz ? (float)gj : 1.0f;
            const T lo = wr ? T(2) * o : o, up = wl ? T(2) * o : o;  // mirror ghosts double a wall row's coupling
            const T bd = (T)(2.0 * inv_dx2 + (boltz ? gj : 1.0));
            if (lane == sep) {  // separator: an identity row in the warp's reduction
                sa = wl ? T(0) : lo;
                sb = bd;
                sc = wr ? T(0) : up;
                sd = (T)r;
            } else {
                b = bd;
                rhs = (T)r;
                // couplings to the separators around the interior become extra right-hand sides
                if (lane == 0) gc = wl ? T(0) : lo;
                else a = lo;
                if (lane == sep - 1) hc = wr ? T(0) : up;
                else c = up;
            }
        }
        // ---- warp interiors: x = rhs - gc S_left - hc S_right
        warp_pcr(a, b, c, rhs, gc, hc);
        float fr = fabs_r, gm = gmin;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            fr = fmaxf(fr, __shfl_xor_sync(0xFFFFFFFFu, fr, off));
            gm = fminf(gm, __shfl_xor_sync(0xFFFFFFFFu, gm, off));
        }
        if (w < W) {
            T* e = wedge + 8 * w;
            if (lane == 0) {
                e[0] = rhs;
                e[1] = gc;
                e[2] = hc;
                e[6] = (T)fr;
                e[7] = (T)gm;
            }
            if (lane == sep - 1) {
                e[3] = rhs;
                e[4] = gc;
                e[5] = hc;
            }
            if (lane == sep) {
                wsep[4 * w] = sa;
                wsep[4 * w + 1] = sb;
                wsep[4 * w + 2] = sc;
                wsep[4 * w + 3] = sd;
            }
        }
        __syncthreads();
        // ---- warp 0: the block's warp separators S_0 .. S_{W-2} in terms of the block
        // separators s_{k-1} (left) and s_k (right), then the block's rows for the cluster system
        if (w == 0) {
            // row q = lane < W - 1: separator of warp q, between warp q's last interior row and
            // warp q+1's first interior row
            T la = T(0), lb = T(1), lc = T(0), r0 = T(0), r1 = T(0), r2 = T(0);
            if (lane < W - 1) {
                const T* ep = wedge + 8 * lane;        // warp q
                const T* en = wedge + 8 * (lane + 1);  // warp q + 1
                const T* sr = wsep + 4 * lane;
                la = -sr[0] * ep[4];
                lb = sr[1] - sr[0] * ep[5] - sr[2] * en[1];
                lc = -sr[2] * en[2];
                r0 = sr[3] - sr[0] * ep[3] - sr[2] * en[0];
                if (lane == 0) {  // S_{-1} = s_{k-1}
                    r1 = la;
                    la = T(0);
                }
                if (lane == W - 2) {  // S_{W-1} = s_k
                    r2 = lc;
                    lc = T(0);
                }
            }
            T Y = T(0), Gc = T(0), Hc = T(0);
            warp_scalar_pcr(la, lb, lc, r0, r1, r2, W, false, Y, Gc, Hc);
            if (lane < W - 1) {
                lev2[3 * lane] = Y;
                lev2[3 * lane + 1] = Gc;
                lev2[3 * lane + 2] = Hc;
            }
            // the block's first interior row (warp 0, lane 0) and last interior row (warp W-1,
            // lane sep-1), each in terms of s_{k-1} and s_k
            const T* e0 = wedge;
            const T* eL = wedge + 8 * (W - 1);
            const T Y0 = __shfl_sync(0xFFFFFFFFu, Y, 0), G0 = __shfl_sync(0xFFFFFFFFu, Gc, 0),
                    H0 = __shfl_sync(0xFFFFFFFFu, Hc, 0);
            const int ql = W >= 2 ? W - 2 : 0;
            const T YL = __shfl_sync(0xFFFFFFFFu, Y, ql), GL = __shfl_sync(0xFFFFFFFFu, Gc, ql),
                    HL = __shfl_sync(0xFFFFFFFFu, Hc, ql);
            T row[kPush];
            if (W > 1) {  // first row: x = y - g s_{k-1} - h S_0; last row: x = y - g S_{W-2} - h s_k
                row[0] = e0[0] - e0[2] * Y0;
                row[1] = e0[1] - e0[2] * G0;
                row[2] = -e0[2] * H0;
                row[3] = eL[3] - eL[4] * YL;
                row[4] = -eL[4] * GL;
                row[5] = eL[5] - eL[4] * HL;
            } else {
                row[0] = e0[0];
                row[1] = e0[1];
                row[2] = e0[2];
                row[3] = eL[3];
                row[4] = eL[4];
                row[5] = eL[5];
            }
            const T* sL = wsep + 4 * (W - 1);  // the block separator s_k
            row[6] = sL[0];
            row[7] = sL[1];
            row[8] = sL[2];
            row[9] = sL[3];
            // residual bound of the block
            T fb = lane < W ? wedge[8 * lane + 6] : T(0), gb = lane < W ? wedge[8 * lane + 7] : T(3.0e38f);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T f2 = __shfl_xor_sync(0xFFFFFFFFu, fb, off), g2 = __shfl_xor_sync(0xFFFFFFFFu, gb, off);
                fb = f2 > fb ? f2 : fb;
                gb = g2 < gb ? g2 : gb;
            }
            row[10] = fb;
            row[11] = gb;
            if (lane < G) {  // lane r pushes the block's rows into block r's shared memory
                T* dst = cluster.map_shared_rank(recv, lane) + kPush * g;
#pragma unroll
                for (int c2 = 0; c2 < kPush; ++c2) dst[c2] = row[c2];
            }
        }
        cluster.sync();  // #1: every block's pushed rows are visible in every block
        if (hist && !hist_written) {  // every block has read its halo: the history may move on
            if (act) d.phi_prev[j] = p_old;
            hist_written = true;
        }
        // ---- warp 0: the cyclic system of the block separators s_0 .. s_{G-1}, and the residual bound
        if (w == 0) {
            T la = T(0), lb = T(1), lc = T(0), r0 = T(0);
            T fb = T(0), gb = T(3.0e38f);
            if (lane < G) {
                // row of s_k: a x_last(k) + b s_k + c x_first(k+1) = d
                const T* rk = recv + kPush * lane;
                const T* rn = recv + kPush * ((lane + 1) % G);
                la = -rk[6] * rk[4];
                lb = rk[7] - rk[6] * rk[5] - rk[8] * rn[1];
                lc = -rk[8] * rn[2];
                r0 = rk[9] - rk[6] * rk[3] - rk[8] * rn[0];
                fb = rk[10];
                gb = rk[11];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T f2 = __shfl_xor_sync(0xFFFFFFFFu, fb, off), g2 = __shfl_xor_sync(0xFFFFFFFFu, gb, off);
                fb = f2 > fb ? f2 : fb;
                gb = g2 < gb ? g2 : gb;
            }
            T sk, u1, u2;
            warp_scalar_pcr(la, lb, lc, r0, T(0), T(0), G, true, sk, u1, u2);
            if (lane < G) svals[lane] = sk;
            // the residual bounds the next update below tol: phi is converged (the same decision
            // in every block: the same pushed values reduced in the same order)
            if (lane == 0) flag[0] = (it > 0 && (double)fb < tol * (double)gb) ? T(1) : T(0);
        }
        __syncthreads();
        if (flag[0] != T(0)) {
            converged = true;
            break;
        }
        const T Sl = svals[(g - 1 + G) % G], Sr = svals[g];  // s_{k-1}, s_k
        // ---- back substitution: the warp's separators, then its row
        T dlt = T(0);
        if (act) {
            const T Sw_l = (w == 0) ? Sl : lev2[3 * (w - 1)] - lev2[3 * (w - 1) + 1] * Sl - lev2[3 * (w - 1) + 2] * Sr;
            const T Sw_r = (w == W - 1) ? Sr : lev2[3 * w] - lev2[3 * w + 1] * Sl - lev2[3 * w + 2] * Sr;
            if (lane == sep) dlt = Sw_r;
            else if (i == 0)  // the block's first row: the form the left neighbour uses for its halo
                dlt = edge_row(recv + kPush * g, Sl, Sr);
            else
                dlt = rhs - gc * Sw_l - hc * Sw_r;
        }
        // ---- global max |update| (damping and convergence): pushed to every block
        T mloc = dlt < T(0) ? -dlt : dlt;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const T oth = __shfl_xor_sync(0xFFFFFFFFu, mloc, off);
            mloc = oth > mloc ? oth : mloc;
        }
        if (lane == 0) wmax[w] = mloc;
        __syncthreads();
        if (w == 0) {
            T v = (lane < ((int)(blockDim.x + 31) >> 5)) ? wmax[lane] : T(0);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T oth = __shfl_xor_sync(0xFFFFFFFFu, v, off);
                v = oth > v ? oth : v;
            }
            v = __shfl_sync(0xFFFFFFFFu, v, 0);
            if (lane < G) cluster.map_shared_rank(recvm, lane)[g] = v;
        }
        // #2: every block's maximum is visible; the pushed rows are no longer read. The next
        // iteration pushes again only after its barrier #1, which every block reaches after
        // reading these.
        cluster.sync();
        T mm = T(0);
        for (int k = 0; k < G; ++k) mm = recvm[k] > mm ? recvm[k] : mm;
        const double m = (double)mm;
        const double scale = (m > 2.0) ? 2.0 / m : 1.0;
        const double x = act ? scale * (double)dlt : 0.0;
        pj += x;
        if (act) phi[j] = pj;
        if (act && i == 0) ph[0] += scale * (double)Sl;  // the previous block's last node is s_{k-1}
        if (act && i == B - 1) {  // the next block's first row, as its owner computes it
            ph[B + 1] += scale * (double)edge_row(recv + kPush * ((g + 1) % G), Sr, svals[(g + 1) % G]);
        }
        if (boltz) {  // |x| <= scale m for every node: the degree follows the cluster-wide bound
            if (scale * m <= 0.0009765625)
                gj *= exp_tiny(x);
            else
                gj = (fabs(x) <= 0.03125) ? gj * exp_small(x) : exp(pj);
        } else {
            gj = 1.0 + pj;
        }
        if (m < tol) {
            converged = true;
            ++it;
            break;
        }
    }
    if (hist && !hist_written) {  // no iteration ran (maxit 0): the start is the solution
        cluster.sync();           // every block has read its halo
        if (act) {
            d.phi_prev[j] = p_old;
            phi[j] = pj;
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
    cluster.sync();  // no block leaves while another may still push into it
}

template <typename T>
__global__ void __launch_bounds__(kNewtonMaxThreads, 1) k_newton_cluster(FieldDesc d)
{
    cg::cluster_group cluster = cg::this_cluster();
    newton_body<T>(d, cluster);
}

// One cluster per realisation: cluster c solves descs[c]; extrap applies to every realisation.
template <typename T>
__global__ void __launch_bounds__(kNewtonMaxThreads, 1) k_newton_batch(const FieldDesc* descs, int extrap)
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
    while (ncell / G > kNewtonMaxThreads) G <<= 1;  // at most kNewtonMaxThreads nodes (threads) per block
    return G <= kClusterMax ? G : 0;
}

size_t newton_smem_bytes(int B, int G, bool fp64)
{
    const size_t t = fp64 ? sizeof(double) : sizeof(float);
    const size_t W = ((size_t)B + 31) / 32;
    return sizeof(double) * ((size_t)B + 2) + t * ((kPush + 2) * (size_t)G + 15 * W + 33) + 16;
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
    if (B > kNewtonMaxThreads || B < 2) return PE_EINVAL;
    const bool fp64 = walls != 0 && kWallsJacobianFP64;
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

// Cluster size of a realisation's solve inside a batched launch: as few blocks as hold the grid
// at kNewtonMaxThreads nodes each. A lone solve spreads its nodes over up to 16 SMs to cut the
// latency of the FP64 work; an ensemble fills the GPU with many solves at once, and clusters of
// 16 for small grids left most of them waiting for SMs in later waves.
int newton_batch_cluster_size(int ncell)
{
    const int gmax = cluster_size_for(kNewtonMaxThreads * kClusterMax);  // the device's largest
    int G = 1;
    while (ncell / G > kNewtonMaxThreads) G <<= 1;
    return G <= gmax ? G : 0;
}

// Batched field solves: descs[R] on the device, every grid with the same cluster size G;
// fp64: the linear solves run in FP64 (bounded grids with kWallsJacobianFP64).
int launch_newton_batch(const void* descs, int R, int G, int max_ncell, bool fp64, bool extrap, cudaStream_t s)
{
    const int B = max_ncell / G;
    if (B > kNewtonMaxThreads || B < 2 || R < 1) return PE_EINVAL;
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
