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
// sr:      BF16 storage; the step kernels round the stored values
//          stochastically (FP32 and FP64 values are stored as computed).
template <> struct Store<LBM_FP64> {
    using S = double; using C = double;
    static constexpr bool dev = false, shifted = false, sr = false;
};
template <> struct Store<LBM_FP32> {
    using S = float; using C = float;
    static constexpr bool dev = false, shifted = true, sr = false;
};
template <> struct Store<LBM_BF16DEV> {
    using S = __nv_bfloat16; using C = float;
    static constexpr bool dev = true, shifted = false, sr = true;
};
// the FP32 format's deviations d_a = f~*_a - w_a held in BF16
template <> struct Store<LBM_BF16SHIFT> {
    using S = __nv_bfloat16; using C = float;
    static constexpr bool dev = false, shifted = true, sr = true;
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

// ---- addressing of the shifted streams ------------------------------------------
// A global access at byte offset b (signed) from the 64-bit base p, the
// offset a per-velocity constant of the solve: the address is one 64-bit add
// of a warp-uniform constant.  The loads use the read-only path (the source
// buffer is not written during a step) and ask L2 to fetch the 256-byte
// block around each 128-byte request: the next warp's shifted segment of the
// same plane row then hits L2 (about 1 % on the 4096 x 2048 step).
template <class S> __device__ __forceinline__ S ld_b(const S *p, long long b);
template <> __device__ __forceinline__ float ld_b<float>(const float *p, long long b) {
    float v;
    asm("{\n\t.reg .u64 a;\n\tadd.s64 a, %2, %1;\n\tld.global.nc.L2::256B.f32 %0, [a];\n\t}"
        : "=f"(v) : "l"(b), "l"(p));
    return v;
}
template <> __device__ __forceinline__ double ld_b<double>(const double *p, long long b) {
    double v;
    asm("{\n\t.reg .u64 a;\n\tadd.s64 a, %2, %1;\n\tld.global.nc.L2::256B.f64 %0, [a];\n\t}"
        : "=d"(v) : "l"(b), "l"(p));
    return v;
}
template <> __device__ __forceinline__ __nv_bfloat16 ld_b<__nv_bfloat16>(const __nv_bfloat16 *p,
                                                                       long long b) {
    unsigned short v;
    asm("{\n\t.reg .u64 a;\n\tadd.s64 a, %2, %1;\n\tld.global.nc.L2::256B.b16 %0, [a];\n\t}"
        : "=h"(v) : "l"(b), "l"(p));
    return __ushort_as_bfloat16(v);
}
// The same with a compile-time byte offset B (|B| < 2^23), folded into the
// access instruction: no address arithmetic per access.
template <class S, long long B> __device__ __forceinline__ S ld_i(const S *p);
template <class S, long long B> struct LdI;
template <long long B> struct LdI<float, B> {
    __device__ __forceinline__ static float go(const float *p) {
        float v;
        asm("ld.global.nc.L2::256B.f32 %0, [%1+%2];" : "=f"(v) : "l"(p), "n"(B));
        return v;
    }
};
template <long long B> struct LdI<double, B> {
    __device__ __forceinline__ static double go(const double *p) {
        double v;
        asm("ld.global.nc.L2::256B.f64 %0, [%1+%2];" : "=d"(v) : "l"(p), "n"(B));
        return v;
    }
};
template <long long B> struct LdI<__nv_bfloat16, B> {
    __device__ __forceinline__ static __nv_bfloat16 go(const __nv_bfloat16 *p) {
        unsigned short v;
        asm("ld.global.nc.L2::256B.b16 %0, [%1+%2];" : "=h"(v) : "l"(p), "n"(B));
        return __ushort_as_bfloat16(v);
    }
};
template <class S, long long B> __device__ __forceinline__ S ld_i(const S *p) { return LdI<S, B>::go(p); }
template <long long B, bool CS>
__device__ __forceinline__ void st_i(float *p, float v) {
    if constexpr (CS) asm volatile("st.global.cs.f32 [%0+%1], %2;" :: "l"(p), "n"(B), "f"(v) : "memory");
    else asm volatile("st.global.f32 [%0+%1], %2;" :: "l"(p), "n"(B), "f"(v) : "memory");
}
template <long long B, bool CS>
__device__ __forceinline__ void st_i(double *p, double v) {
    if constexpr (CS) asm volatile("st.global.cs.f64 [%0+%1], %2;" :: "l"(p), "n"(B), "d"(v) : "memory");
    else asm volatile("st.global.f64 [%0+%1], %2;" :: "l"(p), "n"(B), "d"(v) : "memory");
}
template <long long B, bool CS>
__device__ __forceinline__ void st_i(unsigned short *p, unsigned short v) {
    if constexpr (CS) asm volatile("st.global.cs.b16 [%0+%1], %2;" :: "l"(p), "n"(B), "h"(v) : "memory");
    else asm volatile("st.global.b16 [%0+%1], %2;" :: "l"(p), "n"(B), "h"(v) : "memory");
}

// stores; CS: streaming (evict-first) hint
template <bool CS>
__device__ __forceinline__ void st_b(float *p, long long b, float v) {
    if constexpr (CS)
        asm volatile("{\n\t.reg .u64 a;\n\tadd.s64 a, %1, %0;\n\tst.global.cs.f32 [a], %2;\n\t}"
                     :: "l"(b), "l"(p), "f"(v) : "memory");
    else
        asm volatile("{\n\t.reg .u64 a;\n\tadd.s64 a, %1, %0;\n\tst.global.f32 [a], %2;\n\t}"
                     :: "l"(b), "l"(p), "f"(v) : "memory");
}
template <bool CS>
__device__ __forceinline__ void st_b(double *p, long long b, double v) {
    if constexpr (CS)
        asm volatile("{\n\t.reg .u64 a;\n\tadd.s64 a, %1, %0;\n\tst.global.cs.f64 [a], %2;\n\t}"
                     :: "l"(b), "l"(p), "d"(v) : "memory");
    else
        asm volatile("{\n\t.reg .u64 a;\n\tadd.s64 a, %1, %0;\n\tst.global.f64 [a], %2;\n\t}"
                     :: "l"(b), "l"(p), "d"(v) : "memory");
}
template <bool CS>
__device__ __forceinline__ void st_b(unsigned short *p, long long b, unsigned short v) {
    if constexpr (CS)
        asm volatile("{\n\t.reg .u64 a;\n\tadd.s64 a, %1, %0;\n\tst.global.cs.b16 [a], %2;\n\t}"
                     :: "l"(b), "l"(p), "h"(v) : "memory");
    else
        asm volatile("{\n\t.reg .u64 a;\n\tadd.s64 a, %1, %0;\n\tst.global.b16 [a], %2;\n\t}"
                     :: "l"(b), "l"(p), "h"(v) : "memory");
}

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
// 32 random bits of the velocity pair led by odd A (and of the rest
// velocity, A = 0): the cell hash times an odd multiplier that depends on A,
// modulo 2^32.  An odd multiplier permutes the 32-bit words, so the product
// is uniform when the hash is; its lower half is a permutation of the hash's
// lower 16 bits and, for each of those, its upper half runs uniformly over
// the hash's upper 16 bits, so the two halves are uniform and independent.
// (The high word of the 64-bit product is not uniform: it stays below the
// multiplier, and its upper bits would round down more often than up.)
__device__ __forceinline__ uint32_t sr_word(uint32_t hcell, int A) {
    return hcell * (0x9E3779B9u * (2u * (uint32_t)A + 1u));
}
// 16 random bits of velocity a: the upper half of its pair's word for the
// rest velocity and the odd member a of a pair (a, a + 1), the lower half for
// the even member
__device__ __forceinline__ uint32_t sr_bits(uint32_t hcell, int a) {
    if (a == 0 || (a & 1)) return sr_word(hcell, a) >> 16;
    return sr_word(hcell, a - 1) & 0xffffu;
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
// Two values rounded to BF16 by one hardware stochastic-rounding conversion
// (cvt.rs.satfinite.bf16x2.f32): va to the upper half with the upper 16 bits
// of rbits, vb to the lower half with the lower 16.  For finite values below
// the BF16 maximum it adds those bits below the 16 kept ones and truncates,
// the same rounding as store_rounded with the same bits (checked on the
// device bit for bit over 2^20 random pairs), in one instruction for both.
__device__ __forceinline__ uint32_t bf16x2_rounded(float va, float vb, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(va), "f"(vb), "r"(rbits));
    return d;
}
// random bits of the pair (a, a + 1) for bf16x2_rounded: sr_bits(h, a) in the
// upper half, sr_bits(h, a + 1) in the lower (one multiply for both)
__device__ __forceinline__ uint32_t sr_bits_pair(uint32_t hcell, int a) { return sr_word(hcell, a); }

// ---- stochastic rounding of FP32 results (batched path) -----------------------
// f + t rounded to FP32 stochastically, from 32 random bits x: a uniform
// dither of one unit in the last place U of f, in [-U/2, U/2), is added to the
// small term before the final addition, so the result is the lower or the
// upper FP32 neighbour of the exact sum with probabilities that make it
// unbiased (Connolly, Higham & Mary, SIAM J. Sci. Comput. 43 (2021):
// stochastic rounding, mode 1).  Where the sum lies in f's binade or a lower
// one, U is a whole multiple of the sum's grid spacing and the rounding is
// exactly unbiased; t + dither is itself rounded on t's grid, which keeps it
// unbiased to within ~ulp(t) / 2 of a unit (exact where |t| << |f|, the case
// of a long relaxation time, where it matters most).  Round-to-nearest leaves
// the same round-off at every step of a steady state, a constant forcing
// that the slowest relaxation time amplifies (up to ~1e-4 U_w in u_x for tall
// or dense columns); stochastic rounding makes it zero-mean noise.
__device__ __forceinline__ float add_sr(float f, float t, uint32_t x) {
    // exponent bits of ulp(f) = 2^(E - 23) for f in [2^E, 2^(E+1)); clamped
    // to the smallest normal for |f| < 2^-103 (f = 0 included)
    const uint32_t e = max(__float_as_uint(f) & 0x7f800000u, 24u << 23) - (23u << 23);
    const float U = __uint_as_float(e);
    const float m = __uint_as_float(e | (x & 0x007fffffu));   // uniform in [U, 2U)
    return f + (t + fmaf(-1.5f, U, m));
}
// 32 random bits of velocity a from the cell's hash: the high word of its
// product with an odd multiplier that depends on a
__device__ __forceinline__ uint32_t sr_bits32(uint32_t hcell, int a) {
    return __umulhi(hcell, 0x9E3779B9u * (2u * (uint32_t)a + 1u));
}

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

// BF16DEV: f = d + w rho on the pull side and d = f - w rho on the store
// side, each with one rounding (an explicit FMA in every kernel, so that all
// of them round alike)
__device__ __forceinline__ float dev_to_f(float d, float w, float rho) { return __fmaf_rn(w, rho, d); }
__device__ __forceinline__ float f_to_dev(float f, float w, float rho) { return __fmaf_rn(-w, rho, f); }

__device__ __forceinline__ int wrap(int v, int n) {
    int m = v % n;
    return m < 0 ? m + n : m;
}

// ---- tiled storage (layout in KConsts) ----------------------------------------
// Element of velocity 0 of column x (0 <= x < Nx), row j, in a state buffer;
// velocity a sits a pitch further.  The density of (j, x) in the density plane.
template <class K>
__device__ __forceinline__ long long col_index(const K &k, int j, int x) {
    const int t = k.nt == 1 ? 0 : x / k.tw;
    return t * k.tile_elems + (long long)j * k.Q * k.pitch + (x - t * k.tw) + kPadL;
}
template <class K>
__device__ __forceinline__ long long rho_index(const K &k, int j, int x) {
    const int t = k.nt == 1 ? 0 : x / k.tw;
    return t * k.tile_rho + (long long)j * k.pitch + (x - t * k.tw) + kPadL;
}

// ---- explicit arithmetic --------------------------------------------------------
// The collision below is written with explicit fma / mul / add / sub, which
// the compiler never contracts or reorders, so every kernel that inlines it
// (one thread per cell, tile-staged, batched) executes the same roundings and
// their results agree bit for bit wherever they compute the same cell.
template <class V> struct Ar;
template <> struct Ar<float> {
    using S = float;
    __device__ __forceinline__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ __forceinline__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ __forceinline__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ __forceinline__ static float sub(float a, float b) { return __fsub_rn(a, b); }
    // FP32 reciprocal to within 2 ulp (one MUFU.RCP and a multiply): its
    // error, a relative 1e-7 in 1/rho and in omega, is far below what FP32
    // storage resolves, and every kernel evaluates the same expression
    __device__ __forceinline__ static float rcp(float a) { return __fdividef(1.0f, a); }
    __device__ __forceinline__ static float pw(float a, float e) { return powf(a, e); }
    __device__ __forceinline__ static float bc(float c) { return c; }
};
template <> struct Ar<double> {
    using S = double;
    __device__ __forceinline__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ __forceinline__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ __forceinline__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ __forceinline__ static double sub(double a, double b) { return __dsub_rn(a, b); }
    __device__ __forceinline__ static double rcp(double a) { return __drcp_rn(a); }
    __device__ __forceinline__ static double pw(double a, double e) { return pow(a, e); }
    __device__ __forceinline__ static double bc(double c) { return c; }
};

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
//
// Relaxation (Eq. (5)): f~* = f~ - omega (f~ - rho g) = f~ + (omega rho g - omega f~).
// In FP32 the factor 1 - omega is never formed: for a long relaxation time
// (omega ~ 1e-4 .. 1e-3 in tall, rarefied columns) fl(1 - omega) carries an
// absolute round-off of up to 2^-25, i.e. a systematic relative error of up to
// 2^-25 / omega in the effective omega of the f~ term, which moves the FP32
// steady state by about that relative amount.  FP64 keeps the form
// (1 - omega) f~ + omega rho g.
//
// V: float or double.
template <int Q, class V, bool SHIFT = false>
struct Collision {
    using L = Lat<Q>;
    using O = Ar<V>;
    using C = typename O::S;                // scalar type of the constants
    static constexpr bool kExactOmega = sizeof(C) == 4;
    V om;                   // omega
    V nom;                  // -omega (FP32)
    V omc;                  // 1 - omega (FP64)
    V cw[L::NSH];           // omega rho w_k
    V A0[L::NSH], A1[L::NSH], A2[L::NSH];
    V A3, A4;
    V sx, sy;               // r u: s_a = e_ax sx + e_ay sy
    V rho;

    __device__ __forceinline__ void setup(const V (&f)[Q], const KConsts<C> &k) {
        // moments from the sums and differences of opposite pairs
        V r0 = f[0], jx = O::bc(C(0)), jy = O::bc(C(0));
#pragma unroll
        for (int a = 1; a < Q; a += 2) {
            const V sum = O::add(f[a], f[a + 1]), dif = O::sub(f[a], f[a + 1]);
            r0 = O::add(r0, sum);
            if (L::ex(a) == 1) jx = O::add(jx, dif);
            else if (L::ex(a) == -1) jx = O::sub(jx, dif);
            else if (L::ex(a) != 0) jx = O::fma(O::bc(C(L::ex(a))), dif, jx);
            if (L::ey(a) == 1) jy = O::add(jy, dif);
            else if (L::ey(a) == -1) jy = O::sub(jy, dif);
            else if (L::ey(a) != 0) jy = O::fma(O::bc(C(L::ey(a))), dif, jy);
        }
        const V drho = r0;
        rho = SHIFT ? O::add(O::bc(C(1)), r0) : r0;
        const V inv = O::rcp(rho);
        const V ux = O::mul(O::mul(O::bc(k.r), jx), inv);
        const V uy = O::mul(O::mul(O::bc(k.r), jy), inv);
        const V u2 = O::fma(ux, ux, O::mul(uy, uy));
        V th = O::bc(C(0)), T = O::bc(C(1));
        if (k.thermal) {
            V e2 = O::bc(C(0));
#pragma unroll
            for (int a = 1; a < Q; a += 2)
                e2 = O::fma(O::bc(C(L::e2(a))), O::add(f[a], f[a + 1]), e2);
            if (SHIFT) {
                // deviations: 2 rho theta = (r^2 e2w - 2) + r^2 sum e^2 d - rho u^2
                // - 2 drho, every term small (no cancellation against 2)
                V t = O::fma(O::bc(k.r2), e2, O::bc(k.th0));
                t = O::sub(t, O::mul(rho, u2));
                t = O::fma(O::bc(C(-2)), drho, t);
                th = O::mul(t, O::mul(O::bc(C(0.5)), inv));
                T = O::add(O::bc(C(1)), th);
            } else {
                T = O::mul(O::sub(O::mul(O::mul(O::bc(k.r2), e2), inv), u2), O::bc(C(0.5)));
                th = O::sub(T, O::bc(C(1)));
            }
        }
        V taul;
        if (k.const_tau) taul = O::bc(k.tau_lat);
        else if (k.mu_is_one || !k.thermal) taul = O::mul(O::bc(k.K), inv);
        else taul = O::mul(O::mul(O::bc(k.K), inv), O::pw(T, k.mu_m1));
        set_omega(O::rcp(O::add(taul, O::bc(C(0.5)))));
        sx = O::mul(O::bc(k.r), ux);
        sy = O::mul(O::bc(k.r), uy);
        set_coefficients(u2, th, O::mul(om, rho), O::mul(drho, inv), k);
    }

    // A0 = a00 + a01 c2 + a02 c2^2, A1 = a10 + a11 c2, A2 = a20 + a21 c2: the
    // Eq. (4) coefficients above, collected in powers of c2 (D = 2)
    // orho = omega rho; drr = (rho - 1) / rho (used when SHIFT)
    __device__ __forceinline__ void set_coefficients(V u2, V th, V orho, V drr,
                                                     const KConsts<C> &k) {
        V p[8];
        powers(u2, th, drr, k, p);
#pragma unroll
        for (int s = 0; s < L::NSH; ++s) shell(p, orho, k, s, A0[s], A1[s], A2[s], cw[s]);
    }
    // the c2-independent factors a00, a01, a02, a10, a11, a20, a21 (and A3, A4)
    __device__ __forceinline__ void powers(V u2, V th, V drr, const KConsts<C> &k, V (&p)[8]) {
        const bool o3 = k.eq_order >= 3, o4 = k.eq_order >= 4;
        V a00 = O::sub(O::fma(O::bc(C(-0.5)), u2, SHIFT ? drr : O::bc(C(1))), th);
        V a01 = O::mul(O::bc(C(0.5)), th), a02 = O::bc(C(0));
        V a10 = O::bc(C(1)), a11 = O::bc(C(0)), a20 = O::bc(C(0.5)), a21 = O::bc(C(0));
        if (o3) {
            a10 = O::sub(O::fma(O::bc(C(-0.5)), u2, a10), O::mul(O::bc(C(2)), th));
            a11 = O::mul(O::bc(C(0.5)), th);
        }
        if (o4) {
            a00 = O::fma(O::mul(O::bc(C(0.125)), u2), u2, a00);
            a00 = O::fma(th, u2, a00);
            a00 = O::fma(th, th, a00);
            a01 = O::fma(O::mul(O::bc(C(-0.25)), th), u2, a01);
            a01 = O::sub(a01, O::mul(th, th));
            a02 = O::mul(O::mul(O::bc(C(0.125)), th), th);
            a20 = O::sub(O::fma(O::bc(C(-0.25)), u2, a20), O::mul(O::bc(C(1.5)), th));
            a21 = O::mul(O::bc(C(0.25)), th);
        }
        A3 = O::bc(o3 ? C(1) / C(6) : C(0));
        A4 = O::bc(o4 ? C(1) / C(24) : C(0));
        p[0] = a00; p[1] = a01; p[2] = a02; p[3] = a10; p[4] = a11; p[5] = a20; p[6] = a21;
        p[7] = O::bc(C(0));
    }
    // the coefficients of shell s
    __device__ __forceinline__ static void shell(const V (&p)[8], V orho, const KConsts<C> &k, int s,
                                                 V &A0s, V &A1s, V &A2s, V &cws) {
        const V c2 = O::bc(k.c2sh[s]);
        A0s = O::fma(O::fma(p[2], c2, p[1]), c2, p[0]);
        A1s = O::fma(p[4], c2, p[3]);
        A2s = O::fma(p[6], c2, p[5]);
        cws = O::mul(orho, O::bc(k.wsh[s]));
    }

    __device__ __forceinline__ void set_omega(V omega) {
        om = omega;
        nom = O::mul(O::bc(C(-1)), omega);
        omc = O::sub(O::bc(C(1)), omega);
    }
    // f + omega (g - f) given the equilibrium term omega rho g = eq
    __device__ __forceinline__ V relax(V f, V eq) const {
        if constexpr (kExactOmega) return O::add(f, O::fma(nom, f, eq));
        else return O::fma(omc, f, eq);
    }
    // s_a = c_a . u of velocity A
    template <int A>
    __device__ __forceinline__ V s_of() const {
        constexpr int ex = L::ex(A), ey = L::ey(A);
        if constexpr (ex == 0) return O::mul(O::bc(C(ey)), sy);
        else if constexpr (ey == 0) return O::mul(O::bc(C(ex)), sx);
        else return O::fma(O::bc(C(ex)), sx, O::mul(O::bc(C(ey)), sy));
    }
    // omega rho w g of the pair (A, A+1): the shared even part P and the odd part R
    template <int A>
    __device__ __forceinline__ void eq_pair(V &P, V &R) const {
        constexpr int s = L::sh(A);
        const V sv = s_of<A>();
        const V s2 = O::mul(sv, sv);
        const V E = O::fma(s2, O::fma(A4, s2, A2[s]), A0[s]);
        const V Od = O::mul(sv, O::fma(A3, s2, A1[s]));
        P = O::mul(cw[s], E);
        R = O::mul(cw[s], Od);
    }
    // post-collision values of the rest velocity and of pair (a, a+1)
    __device__ __forceinline__ V rest(V f0) const { return relax(f0, O::mul(cw[0], A0[0])); }
    template <int A>
    __device__ __forceinline__ void pair(V fa, V fb, V &oa, V &ob) const {
        V P, R;
        eq_pair<A>(P, R);
        oa = relax(fa, O::add(P, R));
        ob = relax(fb, O::sub(P, R));
    }
    // Relaxation of one FP32 cell whose increments t_a = omega (rho w g_a - f_a)
    // conserve mass, momentum and (thermal) energy as exactly as FP32 sums
    // allow, then added to f_a with stochastic rounding (add_sr).  In exact arithmetic
    // the BGK step conserves them (Sec. II: the equilibrium has the cell's rho,
    // u and T), so the correction below is zero; in FP32 the rounding of rho, u
    // and T and of the lattice constants leaves each collision a small source
    // of mass and momentum that is the same at every step of a steady state,
    // and the conserved quantities are the ones whose modes decay slowest, so
    // such a source moves the steady state by up to ~1e-5 U_w.  The sums M, Jx,
    // Jy, E of the increments are removed through the rest velocity (mass) and
    // the four unit velocities (1,0), (-1,0), (0,1), (0,-1) (velocities 1..4
    // of every lattice here): -J/2 and +J/2 on the two of an axis (momentum,
    // no mass or energy), -E/4 on each of the four (energy, no momentum), and
    // the remaining mass on the rest velocity.
    __device__ __forceinline__ void relax_conserving_sr(const float (&f)[Q], float (&o)[Q],
                                                        uint32_t hcell, bool thermal) const {
        static_assert(L::ex(1) == 1 && L::ey(1) == 0 && L::ex(2) == -1 && L::ey(2) == 0 &&
                          L::ex(3) == 0 && L::ey(3) == 1 && L::ex(4) == 0 && L::ey(4) == -1,
                      "velocities 1..4 must be the unit velocities");
        float M = 0.0f, Jx = 0.0f, Jy = 0.0f, E = 0.0f;
        float t1 = 0.0f, t2 = 0.0f, t3 = 0.0f, t4 = 0.0f;
        PairLoop<1, Q>::run([&](auto ic) {
            constexpr int A = decltype(ic)::value;
            float P, R;
            eq_pair<A>(P, R);
            const float ta = __fmaf_rn(nom, f[A], __fadd_rn(P, R));
            const float tb = __fmaf_rn(nom, f[A + 1], __fsub_rn(P, R));
            const float ts = __fadd_rn(ta, tb), td = __fsub_rn(ta, tb);
            M = __fadd_rn(M, ts);
            // e(A + 1) = -e(A): the pair's momentum is e(A) (ta - tb)
            if constexpr (L::ex(A) == 1) Jx = __fadd_rn(Jx, td);
            else if constexpr (L::ex(A) == -1) Jx = __fsub_rn(Jx, td);
            else if constexpr (L::ex(A) != 0) Jx = __fmaf_rn(float(L::ex(A)), td, Jx);
            if constexpr (L::ey(A) == 1) Jy = __fadd_rn(Jy, td);
            else if constexpr (L::ey(A) == -1) Jy = __fsub_rn(Jy, td);
            else if constexpr (L::ey(A) != 0) Jy = __fmaf_rn(float(L::ey(A)), td, Jy);
            if (thermal) E = __fmaf_rn(float(L::e2(A)), ts, E);
            if constexpr (A == 1) {
                t1 = ta;
                t2 = tb;
            } else if constexpr (A == 3) {
                t3 = ta;
                t4 = tb;
            } else {
                o[A] = add_sr(f[A], ta, sr_bits32(hcell, A));
                o[A + 1] = add_sr(f[A + 1], tb, sr_bits32(hcell, A + 1));
            }
        });
        float t0 = __fmaf_rn(nom, f[0], __fmul_rn(cw[0], A0[0]));
        M = __fadd_rn(M, t0);
        const float hx = __fmul_rn(0.5f, Jx), hy = __fmul_rn(0.5f, Jy);
        t1 = __fsub_rn(t1, hx);
        t2 = __fadd_rn(t2, hx);
        t3 = __fsub_rn(t3, hy);
        t4 = __fadd_rn(t4, hy);
        if (thermal) {
            const float q = __fmul_rn(0.25f, E);
            t1 = __fsub_rn(t1, q);
            t2 = __fsub_rn(t2, q);
            t3 = __fsub_rn(t3, q);
            t4 = __fsub_rn(t4, q);
            M = __fsub_rn(M, E);
        }
        t0 = __fsub_rn(t0, M);
        o[0] = add_sr(f[0], t0, sr_bits32(hcell, 0));
        o[1] = add_sr(f[1], t1, sr_bits32(hcell, 1));
        o[2] = add_sr(f[2], t2, sr_bits32(hcell, 2));
        o[3] = add_sr(f[3], t3, sr_bits32(hcell, 3));
        o[4] = add_sr(f[4], t4, sr_bits32(hcell, 4));
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
    const int xs = wrap(x - 2 * ex, k.Nx);
    auto v = to_c(fin[col_index(k, j, xs) + (long long)b * k.pitch]);
    if constexpr (Store<PREC>::dev) v = dev_to_f(v, k.w[b], rin[rho_index(k, j, xs)]);
    return v;
}

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

// The copies of column x (tile t, tile column xl of a tile of w columns) held
// in halos: with one tile its periodic images, else the slot in the previous
// tile's right halo (xl < kPadL) or the next tile's left halo (xl >= w -
// kPadL).  seg0: this row's segment of the velocity in tile 0; ts: tile stride.
template <class S, class K>
__device__ __forceinline__ void store_halo_copies(S *__restrict__ seg0, long long ts, const K &k,
                                                  int t, int xl, int w, S v) {
    if (k.nt == 1) {
        for (int q = xl - k.Nx; q >= -kPadL; q -= k.Nx) seg0[q + kPadL] = v;
        for (int q = xl + k.Nx; q < k.Nx + kPadL; q += k.Nx) seg0[q + kPadL] = v;
        return;
    }
    if (xl < kPadL) {
        const int tl = t == 0 ? k.nt - 1 : t - 1;
        seg0[tl * ts + tile_width(k, tl) + kPadL + xl] = v;
    }
    if (xl >= w - kPadL) {
        const int tr = t == k.nt - 1 ? 0 : t + 1;
        seg0[tr * ts + xl - w + kPadL] = v;
    }
}
// Population a of (j, x), its own slot and its halo copies.
template <class S, class K>
__device__ __forceinline__ void store_pop(S *__restrict__ f, const K &k, int a, int j, int x, S v) {
    const int t = k.nt == 1 ? 0 : x / k.tw, xl = x - t * k.tw;
    S *seg0 = f + ((long long)j * k.Q + a) * k.pitch;
    seg0[t * k.tile_elems + xl + kPadL] = v;
    store_halo_copies<S>(seg0, k.tile_elems, k, t, xl, tile_width(k, t), v);
}
// Density of (j, x) (BF16DEV), its own slot and its halo copies.
template <class K>
__device__ __forceinline__ void store_rho(float *__restrict__ r, const K &k, int j, int x, float v) {
    const int t = k.nt == 1 ? 0 : x / k.tw, xl = x - t * k.tw;
    float *seg0 = r + (long long)j * k.pitch;
    seg0[t * k.tile_rho + xl + kPadL] = v;
    store_halo_copies<float>(seg0, k.tile_rho, k, t, xl, tile_width(k, t), v);
}

}  // namespace lbm
