// Field solve: the nonlinear Poisson-Boltzmann equation of Section 3.3,
//   -(phi_{j+1} - 2 phi_j + phi_{j-1}) / dx^2 + g(phi_j) = n_j,   g = exp or 1 + phi,
// by Newton's method in FP64 on one block, followed by the centred field
// E_j = -(phi_{j+1} - phi_{j-1}) / (2 dx).
//
// Each Newton update solves the cyclic tridiagonal Jacobian system with a partition
// method: thread t owns the contiguous segment of M = ncell / T nodes. A downward
// and an upward elimination sweep inside the segment express every interior node
// through the segment's first (F) and last (L) node; the 2T boundary unknowns form a
// cyclic tridiagonal system (order F_0, L_0, F_1, L_1, ...) solved by parallel cyclic
// reduction in shared memory; the interior nodes follow by back-substitution.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pe_common.cuh"
#include "pe_internal.h"

namespace pe {

constexpr int kNewtonThreads = 512;

__device__ __forceinline__ double block_max(double v, double* red)
{
    v = warp_max(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double r = (lane < nw) ? red[lane] : 0.0;
    return warp_max(r);
}

__global__ void __launch_bounds__(kNewtonThreads) k_newton(const long long* rho, int ncell, double dx, double nscale,
                                                           int mode, double tol, int maxit, double* phi, double* E,
                                                           float* Ef, int* diag, uint32_t* status)
{
    extern __shared__ double sh[];
    __shared__ double red[32];
    const int T = blockDim.x;
    const int M = ncell / T;
    const int mask = ncell - 1;
    double* CH = sh;  // [M][T] sweep coefficients: coupling to L (upward) / right neighbour
    double* AH = CH + (size_t)M * T;  // coupling to F
    double* DH = AH + (size_t)M * T;  // right-hand side
    double* RA = DH + (size_t)M * T;  // reduced system [2T]
    double* RB = RA + 2 * T;
    double* RC = RB + 2 * T;
    double* RD = RC + 2 * T;
    const int t = threadIdx.x;
    const int j0 = t * M;
    const double inv_dx2 = 1.0 / (dx * dx);
    const double o = -inv_dx2;  // off-diagonal of the Jacobian
    const int nred = 2 * T;

    int it = 0;
    bool converged = false;
    for (it = 0; it < maxit; ++it) {
        // ---- residual, Jacobian diagonal and downward sweep over the segment
        double b0 = 0.0, d0 = 0.0;
        double phm = phi[(j0 - 1) & mask], phj = phi[j0];
        for (int i = 0; i < M; ++i) {
            const int j = j0 + i;
            const double php = phi[(j + 1) & mask];
            const double g = (mode == PE_POISSON_BOLTZMANN) ? exp(phj) : 1.0 + phj;
            const double gp = (mode == PE_POISSON_BOLTZMANN) ? g : 1.0;
            const double nj = (double)__ldg(rho + j) * nscale;
            const double b = 2.0 * inv_dx2 + gp;
            const double d = (phm - 2.0 * phj + php) * inv_dx2 - g + nj;  // -F_j
            if (i == 0) {
                b0 = b;
                d0 = d;
            } else if (i == 1) {
                const double rr = 1.0 / b;
                CH[T + t] = o * rr;
                AH[T + t] = o * rr;
                DH[T + t] = d * rr;
            } else {
                const double cp = CH[(i - 1) * T + t], ap = AH[(i - 1) * T + t], dp = DH[(i - 1) * T + t];
                const double rr = 1.0 / (b - o * cp);
                CH[i * T + t] = o * rr;
                AH[i * T + t] = -o * ap * rr;
                DH[i * T + t] = (d - o * dp) * rr;
            }
            phm = phj;
            phj = php;
        }
        // ---- upward sweep: rows M-3 .. 1 in terms of the segment's last node
        for (int i = M - 3; i >= 1; --i) {
            const double ct = CH[i * T + t], at = AH[i * T + t], dt = DH[i * T + t];
            const double cn = CH[(i + 1) * T + t], an = AH[(i + 1) * T + t], dn = DH[(i + 1) * T + t];
            CH[i * T + t] = -ct * cn;
            AH[i * T + t] = at - ct * an;
            DH[i * T + t] = dt - ct * dn;
        }
        // ---- reduced rows of this segment
        if (M >= 3) {
            RA[2 * t] = o;
            RB[2 * t] = b0 - o * AH[T + t];
            RC[2 * t] = -o * CH[T + t];
            RD[2 * t] = d0 - o * DH[T + t];
        } else {
            RA[2 * t] = o;
            RB[2 * t] = b0;
            RC[2 * t] = o;
            RD[2 * t] = d0;
        }
        RA[2 * t + 1] = AH[(M - 1) * T + t];
        RB[2 * t + 1] = 1.0;
        RC[2 * t + 1] = CH[(M - 1) * T + t];
        RD[2 * t + 1] = DH[(M - 1) * T + t];
        __syncthreads();
        // ---- parallel cyclic reduction on the 2T boundary unknowns
        for (int s = 1; s < nred / 2; s <<= 1) {
            double na[2], nb[2], nc[2], nd[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int r = 2 * t + q;
                const int rm = (r - s) & (nred - 1), rp = (r + s) & (nred - 1);
                const double al = RA[r] / RB[rm];
                const double ga = RC[r] / RB[rp];
                na[q] = -al * RA[rm];
                nc[q] = -ga * RC[rp];
                nb[q] = RB[r] - al * RC[rm] - ga * RA[rp];
                nd[q] = RD[r] - al * RD[rm] - ga * RD[rp];
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int r = 2 * t + q;
                RA[r] = na[q];
                RB[r] = nb[q];
                RC[r] = nc[q];
                RD[r] = nd[q];
            }
            __syncthreads();
        }
        {  // rows r and r + T now couple only to each other
            const int r = t, q = t + T;
            const double er = RA[r] + RC[r], eq = RA[q] + RC[q];
            const double xr = (RD[r] * RB[q] - er * RD[q]) / (RB[r] * RB[q] - er * eq);
            const double xq = (RD[q] - eq * xr) / RB[q];
            __syncthreads();
            RD[r] = xr;
            RD[q] = xq;
        }
        __syncthreads();
        // ---- back-substitution and damped update
        const double xF = RD[2 * t], xL = RD[2 * t + 1];
        double mloc = fmax(fabs(xF), fabs(xL));
        for (int i = 1; i < M - 1; ++i) {
            const double x = DH[i * T + t] - CH[i * T + t] * xL - AH[i * T + t] * xF;
            DH[i * T + t] = x;
            mloc = fmax(mloc, fabs(x));
        }
        const double m = block_max(mloc, red);
        const double scale = (m > 2.0) ? 2.0 / m : 1.0;
        phi[j0] += scale * xF;
        phi[j0 + M - 1] += scale * xL;
        for (int i = 1; i < M - 1; ++i) phi[j0 + i] += scale * DH[i * T + t];
        __syncthreads();
        if (m < tol) {
            converged = true;
            ++it;
            break;
        }
    }
    // ---- centred field
    const double inv_2dx = 0.5 / dx;
    for (int i = 0; i < M; ++i) {
        const int j = j0 + i;
        const double e = -(phi[(j + 1) & mask] - phi[(j - 1) & mask]) * inv_2dx;
        E[j] = e;
        Ef[j] = (float)e;
    }
    if (t == 0) {
        if (diag) {
            diag[0] = it;
            diag[1] = converged ? 1 : 0;
        }
        if (!converged) raise_flag(status, PE_FLAG_NOCONV);
    }
}

}  // namespace pe

using namespace pe;

extern "C" PE_API int pe_field(const int64_t* rho_fx, int32_t ncell, double dx, int32_t s_w, int32_t mode, double tol,
                               int32_t maxit, double* phi, double* E, float* Ef, int32_t* diag, uint32_t* status,
                               void* stream)
{
    if (!is_pow2(ncell) || ncell < 8 || !rho_fx || !phi || !E || !Ef || !(dx > 0.0) || maxit < 0) return PE_EINVAL;
    if (mode != PE_POISSON_BOLTZMANN && mode != PE_POISSON_LINEARIZED) return PE_EINVAL;
    const int T = ncell / 2 < kNewtonThreads ? ncell / 2 : kNewtonThreads;
    const size_t smem = sizeof(double) * (3 * (size_t)ncell + 8 * (size_t)T);
    if (smem > (size_t)max_smem_optin()) return PE_EINVAL;
    if (ensure_smem((const void*)k_newton, smem) != PE_OK) return PE_ECUDA;
    const double nscale = ldexp(1.0, -(s_w + 24));
    k_newton<<<1, T, smem, (cudaStream_t)stream>>>(reinterpret_cast<const long long*>(rho_fx), ncell, dx, nscale, mode,
                                                   tol, maxit, phi, E, Ef, diag, status);
    return launch_status();
}
