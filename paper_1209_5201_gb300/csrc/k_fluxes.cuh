// Stress and heat flux of the distribution behind f~ (Sec. II).
//
// The stored state is post-collision f~*; the pre-collision f~ of the next
// step is what the pull of a step produces (Eq. (5) streaming with the Eq. (12)
// wall), so this kernel pulls exactly like k_step_direct and, instead of
// colliding, evaluates in FP64
//   f = (f~ + h f^eq) / (1 + h),  h = dt / (2 tau)      (definition of f~)
//   sigma_ij = sum (c_i - u_i)(c_j - u_j) f - rho T delta_ij
//   q_i      = 1/2 sum |c - u|^2 (c_i - u_i) f
// with T = 1 in an isothermal run.  Diagnostic read-out, not on the step path.
#pragma once

#include "k_aux.cuh"
#include "k_step_direct.cuh"

namespace lbm {

constexpr int kFluxThreads = 128;

template <int Q, int PREC>
__global__ void __launch_bounds__(kFluxThreads)
k_fluxes(const typename Store<PREC>::S *__restrict__ fin, const float *__restrict__ rin,
         const __grid_constant__ KConsts<typename Store<PREC>::C> k,
         const __grid_constant__ KConsts<double> kd, double *sxx, double *sxy, double *syy,
         double *qx, double *qy) {
    using L = Lat<Q>;
    using C = typename Store<PREC>::C;
    __shared__ double s_min[kFluxThreads + 6];
    const int j = blockIdx.y;
    const int x0 = blockIdx.x * kFluxThreads;
    const int x = x0 + threadIdx.x;
    const bool bot = j < L::N, top = j >= k.Ny - L::N;
    if (bot || top) {
        wall_prologue<Q, PREC, kFluxThreads>(fin, rin, k, bot ? 0 : 1, x0,
                                             min(kFluxThreads, k.Nx - x0) + 6, s_min);
        __syncthreads();
    }
    if (x >= k.Nx) return;

    C fc[Q];
    const typename Store<PREC>::S *src = fin + col_index(k, j, x);
    const float *rsrc = Store<PREC>::dev ? rin + rho_index(k, j, x) : nullptr;
    if (bot || top) pull<Q, PREC, true, 0>(fin, rin, src, rsrc, k, x, j, s_min, fc);
    else pull<Q, PREC, false, 0>(fin, rin, src, rsrc, k, x, j, s_min, fc);

    double f[Q];
    double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        f[a] = (double)fc[a] + (Store<PREC>::shifted ? kd.w[a] : 0.0);
        rho += f[a];
        jx += (double)L::ex(a) * f[a];
        jy += (double)L::ey(a) * f[a];
    }
    const double ux = kd.r * jx / rho, uy = kd.r * jy / rho;
    double T = 1.0;
    if (kd.thermal) {
        double e = 0.0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double cx = kd.r * L::ex(a) - ux, cy = kd.r * L::ey(a) - uy;
            e += (cx * cx + cy * cy) * f[a];
        }
        T = e / (2.0 * rho);
    }
    // tau / dt exactly as the collision forms it
    double taul;
    if (kd.const_tau) taul = kd.tau_lat;
    else if (kd.mu_is_one || !kd.thermal) taul = kd.K / rho;
    else taul = kd.K / rho * pow(T, kd.mu_m1);
    const double h = 0.5 / taul;

    double feq[Q];
    equilibrium_all<Q, double, false>(rho, rho - 1.0, ux, uy, T, kd, feq);
    double pxx = 0.0, pxy = 0.0, pyy = 0.0, hx = 0.0, hy = 0.0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const double fa = (f[a] + h * feq[a]) / (1.0 + h);
        const double cx = kd.r * L::ex(a) - ux, cy = kd.r * L::ey(a) - uy;
        const double c2 = cx * cx + cy * cy;
        pxx += cx * cx * fa;
        pxy += cx * cy * fa;
        pyy += cy * cy * fa;
        hx += 0.5 * c2 * cx * fa;
        hy += 0.5 * c2 * cy * fa;
    }
    const long long c = (long long)j * k.Nx + x;
    if (sxx) sxx[c] = pxx - rho * T;
    if (sxy) sxy[c] = pxy;
    if (syy) syy[c] = pyy - rho * T;
    if (qx) qx[c] = hx;
    if (qy) qy[c] = hy;
}

}  // namespace lbm
