// Device-side building blocks of the step kernels: compile-time lattice
// descriptors, storage formats, Eq. (3) moments, Eq. (4) equilibrium in the
// per-shell polynomial form, Eq. (5) relaxation and the Eq. (12) wall fill.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice_tables.h"
#include "lbm_internal.h"

namespace lbm {

// ---- compile-time lattice descriptors --------------------------------------
template <int Q> struct Lat;

#define LBM_DEFINE_LAT(QQ, NSHELL, EX, EY, SH)                                        \
    template <> struct Lat<QQ> {                                                      \
        static constexpr int Q = QQ, NSH = NSHELL, N = 3;                             \
        __host__ __device__ static constexpr int ex(int a) { constexpr int t[] = EX; return t[a]; } \
        __host__ __device__ static constexpr int ey(int a) { constexpr int t[] = EY; return t[a]; } \
        __host__ __device__ static constexpr int sh(int a) { constexpr int t[] = SH; return t[a]; } \
        __host__ __device__ static constexpr int e2(int a) { return ex(a) * ex(a) + ey(a) * ey(a); } \
        /* |e|^2 of shell s: that of its first member */                              \
        __host__ __device__ static constexpr int shell_e2(int s) {                     \
            for (int a = 0; a < Q; ++a) if (sh(a) == s) return e2(a);                  \
            return 0;                                                                   \
        }                                                                               \
    };

LBM_DEFINE_LAT(17, 5, LBM_Q17_EX, LBM_Q17_EY, LBM_Q17_SH)
LBM_DEFINE_LAT(25, 6, LBM_Q25_EX, LBM_Q25_EY, LBM_Q25_SH)
LBM_DEFINE_LAT(37, 8, LBM_Q37_EX, LBM_Q37_EY, LBM_Q37_SH)

// ---- storage formats ---------------------------------------------------------
template <int PREC> struct Store;
// dev:     stored d_a = f~*_a - w_a rho with rho the cell's own density,
//          kept in an FP32 plane (BF16DEV); values are converted back to f~.
// shifted: stored d_a = f~*_a - w_a (the rest weights as rounded to the
//          compute type); the collision runs on the deviations, so FP32
//          round-off scales with |d| instead of |f|.
template <> struct Store<LBM_FP64> {
    using S = double; using C = double;
    static constexpr bool dev = false, shifted = false;
};
template <> struct Store<LBM_FP32> {
    using S = float; using C = float;
    static constexpr bool dev = false, shifted = true;
};
template <> struct Store<LBM_BF16DEV> {
    using S = __nv_bfloat16; using C = float;
    static constexpr bool dev = true, shifted = false;
};

__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ double to_c(double v) { return v; }

template <class S> __device__ __forceinline__ S from_c(float v);
template <> __device__ __forceinline__ float from_c<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <class S> __device__ __forceinline__ S from_c(double v);
template <> __device__ __forceinline__ double from_c<double>(double v) { return v; }

// ---- stochastic rounding of the BF16 store -----------------------------------
// 16 pseudo-random bits per (step, cell, velocity): one counter-based integer
// hash per cell ("lowbias32", C. Wellons, hash-prospector, 2018) of the cell's
// index mixed with the step count, then per velocity the top 16 bits of its
// product with an odd multiplier that depends on the velocity (one multiply
// per population instead of a hash).
__device__ __forceinline__ uint32_t sr_cell(uint32_t step, uint32_t cell) {
    uint32_t x = cell ^ (step * 0x9E3779B9u);
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ uint32_t sr_bits(uint32_t hcell, int a) {
    return (hcell * (0x9E3779B9u * (2u * (uint32_t)a + 1u))) >> 16;
}
// The value to store: BF16 keeps the top 16 bits of the FP32 pattern; adding
// 16 random bits below them first rounds up with probability equal to the
// dropped fraction (unbiased), so the fixed point of the rounded iteration
// carries no systematic round-off.  FP32 / FP64 values are stored as they are.
template <class S> __device__ __forceinline__ S store_rounded(float v, uint32_t bits);
template <> __device__ __forceinline__ float store_rounded<float>(float v, uint32_t) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 store_rounded<__nv_bfloat16>(float v,
                                                                               uint32_t bits) {
    uint32_t u = __float_as_uint(v);
    if ((u & 0x7f800000u) != 0x7f800000u) u += bits;   // bits < 2^16
    return __ushort_as_bfloat16((unsigned short)(u >> 16));
}
template <class S> __device__ __forceinline__ S store_rounded(double v, uint32_t);
template <> __device__ __forceinline__ double store_rounded<double>(double v, uint32_t) { return v; }

// Step count of this launch's source buffer; block 0 writes the count of the
// destination buffer (read by the next step only).
template <class C>
__device__ __forceinline__ uint32_t step_count(const void *fin, const KConsts<C> &k,
                                               bool first_thread) {
    if (k.sr == nullptr) return 0u;
    const int src = fin == k.f0 ? 0 : 1;
    const uint32_t n = k.sr[src];
    if (first_thread) k.sr[src ^ 1] = n + 1u;
    return n;
}

__device__ __forceinline__ int wrap(int v, int n) {
    int m = v % n;
    return m < 0 ? m + n : m;
}

// ---- Eq. (3)-(5): moments, relaxation factor, equilibrium coefficients --------
// g_a^eq of Eq. (4) for a velocity of shell k, with s = c_a . u, written as
//   w_k (A0_k + A1_k s + A2_k s^2 + A3 s^3 + A4 s^4)
// (D = 2, theta = T - 1, c2 = |c_a|^2):
//   order 2: A0 = 1 - u2/2 + theta (c2 - 2)/2,  A1 = 1,  A2 = 1/2
//   order 3: A1 += -u2/2 + theta (c2 - 4)/2,  A3 = 1/6
//   order 4: A0 += u2^2/8 - theta (c2 - 4) u2/4 + theta^2 (c2^2 - 8 c2 + 8)/8
//            A2 += -u2/4 + theta (c2 - 6)/4,  A4 = 1/24
// A velocity and its opposite share the even part E = A0 + A2 s^2 + A4 s^4 and
// have opposite odd parts O = s (A1 + A3 s^2).
// SHIFT: the inputs are deviations d_a = f_a - w_a and so are the outputs:
// rho = 1 + sum d, and w (rho g - 1) = rho w (g - 1 + drho / rho) replaces
// rho w g, i.e. A0 - 1 + drho / rho replaces A0 (no cancellation: the
// constant 1 of A0 is never formed).
template <int Q, class C, bool SHIFT = false>
struct Collision {
    using L = Lat<Q>;
    C omc;                  // 1 - omega
    C cw[L::NSH];           // omega rho w_k
    C A0[L::NSH], A1[L::NSH], A2[L::NSH];
    C A3, A4;
    C sx, sy;               // r u: s_a = e_ax sx + e_ay sy
    C rho;

    __device__ __forceinline__ void setup(const C (&f)[Q], const KConsts<C> &k) {
        // moments from the sums and differences of opposite pairs
        C r0 = f[0], jx = 0, jy = 0;
#pragma unroll
        for (int a = 1; a < Q; a += 2) {
            const C sum = f[a] + f[a + 1], dif = f[a] - f[a + 1];
            r0 += sum;
            if (L::ex(a) == 1) jx += dif;
            else if (L::ex(a) == -1) jx -= dif;
            else if (L::ex(a) != 0) jx += C(L::ex(a)) * dif;
            if (L::ey(a) == 1) jy += dif;
            else if (L::ey(a) == -1) jy -= dif;
            else if (L::ey(a) != 0) jy += C(L::ey(a)) * dif;
        }
        const C drho = r0;
        rho = SHIFT ? C(1) + r0 : r0;
        const C inv = C(1) / rho;
        const C ux = k.r * jx * inv, uy = k.r * jy * inv;
        const C u2 = ux * ux + uy * uy;
        C th = 0, T = 1;
        if (k.thermal) {
            C e2 = C(0);
#pragma unroll
            for (int a = 1; a < Q; a += 2) e2 += C(L::e2(a)) * (f[a] + f[a + 1]);
            if (SHIFT) {
                // deviations: 2 rho theta = (r^2 e2w - 2) + r^2 sum e^2 d - rho u^2
                // - 2 drho, every term small (no cancellation against 2)
                th = (k.th0 + k.r2 * e2 - rho * u2 - C(2) * drho) * (C(0.5) * inv);
                T = C(1) + th;
            } else {
                T = (k.r2 * e2 * inv - u2) * C(0.5);
                th = T - C(1);
            }
        }
        C taul;
        if (k.const_tau) taul = k.tau_lat;
        else if (k.mu_is_one || !k.thermal) taul = k.K * inv;
        else taul = k.K * inv * pow(T, k.mu_m1);
        const C om = C(1) / (taul + C(0.5));
        omc = C(1) - om;
        sx = k.r * ux;
        sy = k.r * uy;
        set_coefficients(u2, th, om * rho, drho * inv, k);
    }

    // A0 = a00 + a01 c2 + a02 c2^2, A1 = a10 + a11 c2, A2 = a20 + a21 c2: the
    // Eq. (4) coefficients above, collected in powers of c2 (D = 2)
    // orho = omega rho; drr = (rho - 1) / rho (used when SHIFT)
    __device__ __forceinline__ void set_coefficients(C u2, C th, C orho, C drr,
                                                     const KConsts<C> &k) {
        C p[8];
        powers(u2, th, drr, k, p);
#pragma unroll
        for (int s = 0; s < L::NSH; ++s) shell(p, orho, k, s, A0[s], A1[s], A2[s], cw[s]);
    }
    // the c2-independent factors a00, a01, a02, a10, a11, a20, a21 (and A3, A4)
    __device__ __forceinline__ void powers(C u2, C th, C drr, const KConsts<C> &k, C (&p)[8]) {
        const bool o3 = k.eq_order >= 3, o4 = k.eq_order >= 4;
        C a00 = (SHIFT ? drr : C(1)) - C(0.5) * u2 - th, a01 = C(0.5) * th, a02 = C(0);
        C a10 = C(1), a11 = C(0), a20 = C(0.5), a21 = C(0);
        if (o3) {
            a10 += C(-0.5) * u2 - C(2) * th;
            a11 = C(0.5) * th;
        }
        if (o4) {
            a00 += C(0.125) * u2 * u2 + th * u2 + th * th;
            a01 += C(-0.25) * th * u2 - th * th;
            a02 = C(0.125) * th * th;
            a20 += C(-0.25) * u2 - C(1.5) * th;
            a21 = C(0.25) * th;
        }
        A3 = o3 ? C(1) / C(6) : C(0);
        A4 = o4 ? C(1) / C(24) : C(0);
        p[0] = a00; p[1] = a01; p[2] = a02; p[3] = a10; p[4] = a11; p[5] = a20; p[6] = a21;
        p[7] = C(0);
    }
    // the coefficients of shell s
    __device__ __forceinline__ static void shell(const C (&p)[8], C orho, const KConsts<C> &k, int s,
                                                 C &A0s, C &A1s, C &A2s, C &cws) {
        const C c2 = k.c2sh[s];
        A0s = (p[2] * c2 + p[1]) * c2 + p[0];
        A1s = p[4] * c2 + p[3];
        A2s = p[6] * c2 + p[5];
        cws = orho * k.wsh[s];
    }

    // post-collision values of the rest velocity and of pair (a, a+1)
    __device__ __forceinline__ C rest(C f0) const { return omc * f0 + cw[0] * A0[0]; }
    template <int A>
    __device__ __forceinline__ void pair(C fa, C fb, C &oa, C &ob) const {
        constexpr int s = L::sh(A);
        const C sv = C(L::ex(A)) * sx + C(L::ey(A)) * sy;
        const C s2 = sv * sv;
        const C E = A0[s] + s2 * (A2[s] + A4 * s2);
        const C O = sv * (A1[s] + A3 * s2);
        const C P = cw[s] * E, R = cw[s] * O;
        oa = omc * fa + (P + R);
        ob = omc * fb + (P - R);
    }
};

// Re-emitted population of Eq. (12), M_in g^w_a / D_w, in FP64, returned in
// the form the collision takes (a deviation for shifted storage).
template <int PREC>
__device__ __forceinline__ typename Store<PREC>::C wall_fill(double m_in, double coef,
                                                             typename Store<PREC>::C w) {
    double v = m_in * coef;
    if constexpr (Store<PREC>::shifted) v -= (double)w;
    return (typename Store<PREC>::C)v;
}

// Eq. (9) with R = accom R_D + (1 - accom) R_S: the diffuse re-emission mixed
// with the specular one, `spec` being the mirrored population in the form the
// collision takes (a deviation for shifted storage; the mirror shares w_a).
template <int PREC>
__device__ __forceinline__ typename Store<PREC>::C wall_mix(double m_in, double coef,
                                                            typename Store<PREC>::C w,
                                                            double accom,
                                                            typename Store<PREC>::C spec) {
    using C = typename Store<PREC>::C;
    const C diffuse = wall_fill<PREC>(m_in, coef, w);
    return accom == 1.0 ? diffuse : (C)(accom * (double)diffuse + (1.0 - accom) * (double)spec);
}

// Specular partner of velocity a for fluid cell (x, j) next to a wall: the
// mirrored velocity b = (e_x, -e_y) reaching the ghost node from which a leaves
// came from the same row, 2 e_x columns back (periodic), in the collision's form.
template <int PREC>
__device__ __forceinline__ typename Store<PREC>::C
specular_source(const typename Store<PREC>::S *__restrict__ fin, const float *__restrict__ rin,
                const KConsts<typename Store<PREC>::C> &k, int a, int ex, int x, int j) {
    const int b = k.mirror[a];
    const long long ro = (long long)j * k.pitch + wrap(x - 2 * ex, k.Nx) + kPadL;
    auto v = to_c(fin[(long long)b * k.plane + ro]);
    if constexpr (Store<PREC>::dev) v += k.w[b] * rin[ro];
    return v;
}

// compile-time loop a = A, A + 1, ..., N - 1
template <int A, int N>
struct StaticFor {
    template <class F>
    __device__ __forceinline__ static void run(F &&fn) {
        if constexpr (A < N) {
            fn(std::integral_constant<int, A>{});
            StaticFor<A + 1, N>::run(fn);
        }
    }
};

// compile-time loop over the velocity pairs (a = 1, 3, 5, ...)
template <int A, int Q>
struct PairLoop {
    template <class F>
    __device__ __forceinline__ static void run(F &&fn) {
        if constexpr (A < Q) {
            fn(std::integral_constant<int, A>{});
            PairLoop<A + 2, Q>::run(fn);
        }
    }
};

// Store one population at logical column x of row j, and at every periodic
// image of x inside the padded row [-kPadL, Nx + kPadL).
template <class S>
__device__ __forceinline__ void store_with_images(S *__restrict__ row, int x, int Nx, S v) {
    row[x + kPadL] = v;
    if (x < kPadL || x >= Nx - kPadL) {
        for (int q = x - Nx; q >= -kPadL; q -= Nx) row[q + kPadL] = v;
        for (int q = x + Nx; q < Nx + kPadL; q += Nx) row[q + kPadL] = v;
    }
}

}  // namespace lbm
