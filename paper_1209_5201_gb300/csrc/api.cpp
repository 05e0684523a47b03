// C ABI of the library (include/lbm.h): handles, parameter checks, device
// memory layout, and the host side of each call.  Every step of the method
// runs in the CUDA kernels this file launches.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "launchers.h"
#include "lbm_internal.h"

namespace lbm {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

size_t storage_elem_bytes(int precision) {
    return precision == LBM_FP64 ? 8 : (precision == LBM_FP32 ? 4 : 2);
}

int padded_pitch(int Nx, int precision) { return tile_layout(Nx, precision).pitch; }

TileLayout tile_layout(int Nx, int precision) {
    // one tile with a compact segment (kPadL | Nx columns | kPadL, rounded to
    // 128 bytes) for narrow grids; the smallest pitch class holding the row
    // once that is at most twice the row; past the widest class of the
    // precision, the fewest tiles of it, the columns spread evenly (every tile
    // but the last holds tw, the last the rest)
    const int per128 = (int)(128 / storage_elem_bytes(precision));
    const int n = Nx + 2 * kPadL;
    TileLayout t;
    t.nt = 1;
    t.tw = Nx;
    if (2 * n <= pitch_class(precision, 0)) {
        t.pitch = (n + per128 - 1) / per128 * per128;
        return t;
    }
    const int wide = widest_pitch_class(precision);
    for (int c = 0; c <= wide; ++c)
        if (n <= pitch_class(precision, c)) {
            t.pitch = pitch_class(precision, c);
            return t;
        }
    const int tp = pitch_class(precision, wide);
    const int cols = tp - 2 * kPadL;
    t.pitch = tp;
    t.nt = (Nx + cols - 1) / cols;
    t.tw = (Nx + t.nt - 1) / t.nt;
    if (Nx - (t.nt - 1) * t.tw < 2 * kPadL) ++t.nt, t.tw = (Nx + t.nt - 1) / t.nt;
    return t;
}

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t f_bytes, rho_bytes, stage_bytes, prev_bytes, red_bytes, total;
};

Layout layout_of(const LatticeHost &L, const lbm_params &p) {
    Layout lo;
    const TileLayout tl = tile_layout(p.Nx, p.precision);
    const size_t row = (size_t)tl.nt * tl.pitch;     // elements of one row of one velocity
    const size_t cells = (size_t)p.Nx * p.Ny;
    lo.f_bytes = align_up((size_t)L.Q * p.Ny * row * storage_elem_bytes(p.precision));
    lo.rho_bytes = p.precision == LBM_BF16DEV ? align_up((size_t)p.Ny * row * 4) : 0;
    lo.stage_bytes = align_up(5 * cells * 8);
    lo.prev_bytes = align_up(2 * cells * 8);
    lo.red_bytes = align_up((1024 * 8 + 64) * 8);
    lo.total = 2 * lo.f_bytes + 2 * lo.rho_bytes + lo.stage_bytes + lo.prev_bytes + lo.red_bytes;
    return lo;
}

int check_params(const LatticeHost &L, const lbm_params &p) {
    if (p.Nx < 1 || p.Ny < 2 * L.ghost_depth) {
        set_error("need Nx >= 1 and Ny >= 2 * ghost depth");
        return LBM_EINVAL;
    }
    if (p.Nx > (1 << 24)) {
        set_error("grid too large (Nx)");
        return LBM_EINVAL;
    }
    const TileLayout tl = tile_layout(p.Nx, p.precision);
    if ((long long)L.Q * p.Ny * tl.nt * tl.pitch > (1LL << 31) - 1) {
        set_error("grid too large (Q * Ny * padded row must fit in 31 bits)");
        return LBM_EINVAL;
    }
    if (p.eq_order < 2 || p.eq_order > 4) { set_error("eq_order must be 2, 3 or 4"); return LBM_EINVAL; }
    if (p.precision < LBM_FP64 || p.precision > LBM_BF16SHIFT) { set_error("bad precision"); return LBM_EINVAL; }
    if (!(p.tau > 0) && !(p.Kn > 0)) { set_error("need Kn > 0 or tau > 0"); return LBM_EINVAL; }
    if (!std::isfinite(p.Kn) || !std::isfinite(p.tau) || !std::isfinite(p.mu_exp) ||
        !std::isfinite(p.u_wall[0]) || !std::isfinite(p.u_wall[1]) ||
        !std::isfinite(p.T_wall[0]) || !std::isfinite(p.T_wall[1]) || !std::isfinite(p.rho0) ||
        !std::isfinite(p.noise_amp)) {
        set_error("non-finite parameter");
        return LBM_EINVAL;
    }
    if (p.thermal && (p.T_wall[0] <= 0 || p.T_wall[1] <= 0)) { set_error("T_wall must be > 0"); return LBM_EINVAL; }
    if (!(p.rho0 > 0)) { set_error("rho0 must be > 0"); return LBM_EINVAL; }
    if (p.kernel < LBM_KERNEL_AUTO || p.kernel > LBM_KERNEL_CELLWARP) { set_error("bad kernel"); return LBM_EINVAL; }
    if (p.kernel == LBM_KERNEL_STAGED && p.precision == LBM_BF16SHIFT) {
        set_error("the staged kernel is not built for LBM_BF16SHIFT");
        return LBM_EINVAL;
    }
    if (!(p.accom[0] >= 0 && p.accom[0] <= 1 && p.accom[1] >= 0 && p.accom[1] <= 1)) {
        set_error("accom must lie in [0, 1]");
        return LBM_EINVAL;
    }
    return LBM_OK;
}

// Host-side equilibrium of Eq. (4) at the wall (FP64), used only for the
// diffuse re-emission coefficients g^w_a / D_w of Eq. (11)-(12).
void wall_equilibrium(const LatticeHost &L, int order, double uw, double Tw, double *g) {
    const double th = Tw - 1.0, u2 = uw * uw;
    for (int a = 0; a < L.Q; ++a) {
        const double cx = L.r * L.ex[a], cy = L.r * L.ey[a];
        const double c2 = cx * cx + cy * cy, s = cx * uw;
        double A0 = 1 - 0.5 * u2 + 0.5 * th * (c2 - 2), A1 = 1, A2 = 0.5, A3 = 0, A4 = 0;
        if (order >= 3) { A1 += -0.5 * u2 + 0.5 * th * (c2 - 4); A3 = 1.0 / 6.0; }
        if (order >= 4) {
            A0 += 0.125 * u2 * u2 - 0.25 * th * (c2 - 4) * u2 + 0.125 * th * th * (c2 * c2 - 8 * c2 + 8);
            A2 += -0.25 * u2 + 0.25 * th * (c2 - 6);
            A4 = 1.0 / 24.0;
        }
        (void)cy;
        g[a] = L.w[a] * (A0 + s * (A1 + s * (A2 + s * (A3 + s * A4))));
    }
}

#define CU(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (cudaError_t)(call);                                      \
        if (e_ != cudaSuccess) {                                                   \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));         \
            return LBM_ECUDA;                                                      \
        }                                                                          \
    } while (0)

template <class F>
int dispatch_prec(int prec, F &&fn) {
    switch (prec) {
    case LBM_FP64: return fn(std::integral_constant<int, LBM_FP64>{});
    case LBM_FP32: return fn(std::integral_constant<int, LBM_FP32>{});
    case LBM_BF16SHIFT: return fn(std::integral_constant<int, LBM_BF16SHIFT>{});
    default: return fn(std::integral_constant<int, LBM_BF16DEV>{});
    }
}

int effective_kernel(const SolverImpl &s) {
    // the direct kernel is the faster one on every measured grid but the
    // smallest, where one warp per cell shortens the per-step latency chain;
    // the autotuner can still choose any kernel
    if (s.p.kernel != LBM_KERNEL_AUTO) return s.p.kernel;
    return (long long)s.p.Nx * s.p.Ny <= kCellwarpAutoCells ? LBM_KERNEL_CELLWARP : LBM_KERNEL_DIRECT;
}

// Error flags the staged kernel raises when a bounded wait runs out.
int check_device_error(SolverImpl &s) {
    int flag = 0;
    CU(cudaMemcpyAsync(&flag, s.derr, sizeof(int), cudaMemcpyDeviceToHost, s.stream));
    CU(cudaStreamSynchronize(s.stream));
    if (flag) {
        CU(cudaMemsetAsync(s.derr, 0, sizeof(int), s.stream));
        set_error("a bounded device wait timed out in the step kernel");
        return LBM_ETIMEOUT;
    }
    return LBM_OK;
}

int sum_rho(SolverImpl &s, double *out) {
    const int nb = reduction_blocks((long long)s.p.Nx * s.p.Ny);
    CU(dispatch_prec(s.p.precision, [&](auto P) { return Launch<decltype(P)::value>::mass_partials(s, s.red, nb); }));
    CU(launch_final_sum(s.stream, s.red, nb, 1, s.red + 8 * 1024));
    CU(cudaMemcpyAsync(s.pinned, s.red + 8 * 1024, sizeof(double), cudaMemcpyDeviceToHost, s.stream));
    CU(cudaStreamSynchronize(s.stream));
    *out = s.pinned[0];
    return LBM_OK;
}

// The rounding counter of the current buffer holds the step count.
int set_round_counter(SolverImpl &s) {
    s.pinned[63] = 0.0;
    unsigned v = (unsigned)s.steps;
    std::memcpy(&s.pinned[63], &v, sizeof v);
    CU(cudaMemcpyAsync(s.sr + s.cur, &s.pinned[63], sizeof(unsigned), cudaMemcpyHostToDevice, s.stream));
    CU(cudaStreamSynchronize(s.stream));
    return LBM_OK;
}

int after_init(SolverImpl &s) {
    s.steps = 0;
    if (int rc = set_round_counter(s)) return rc;
    s.last_res = -1;
    int rc = sum_rho(s, &s.mass0);
    if (rc) return rc;
    // previous-check planes of the residual start from the initial fields
    const long long n = (long long)s.p.Nx * s.p.Ny;
    CU(dispatch_prec(s.p.precision, [&](auto P) {
        return Launch<decltype(P)::value>::macros(s, nullptr, s.prev, nullptr, s.prev + n);
    }));
    return LBM_OK;
}

}  // namespace

template <class C>
void fill_consts(KConsts<C> &k, const LatticeHost &L, const lbm_params &p, int pitch) {
    std::memset(&k, 0, sizeof(k));
    k.Nx = p.Nx;
    k.Ny = p.Ny;
    k.Q = L.Q;
    const TileLayout tl = tile_layout(p.Nx, p.precision);
    k.pitch = pitch;
    k.nt = tl.nt;
    k.tw = tl.tw;
    k.tile_elems = (long long)p.Ny * L.Q * pitch;
    k.tile_rho = (long long)p.Ny * pitch;
    k.wait_ns = kDefaultWaitNs;
    k.thermal = p.thermal;
    k.eq_order = p.eq_order;
    k.const_tau = p.tau > 0;
    k.mu_is_one = p.mu_exp == 1.0;
    k.r = (C)L.r;
    k.r2 = (C)(L.r * L.r);
    k.K = (C)(std::sqrt(2.0 / M_PI) * p.Kn * L.r * p.Ny);
    k.tau_lat = (C)(p.tau * L.r * p.Ny);
    k.mu_m1 = (C)(p.mu_exp - 1.0);
    for (int a = 0; a < L.Q; ++a) {
        k.w[a] = (C)L.w[a];
        k.wsh[L.shell[a]] = (C)L.w[a];
        k.c2sh[L.shell[a]] = (C)(L.r * L.r * (L.ex[a] * L.ex[a] + L.ey[a] * L.ey[a]));
        const long long es = (long long)storage_elem_bytes(p.precision);
        k.b_src[a] = es * ((long long)(a - L.ey[a] * L.Q) * pitch - L.ex[a]);
        k.b_dst[a] = es * ((long long)a * pitch);
        k.b_rho[a] = 4LL * (-(long long)L.ey[a] * pitch - L.ex[a]);
    }
    double e2w = 0;
    for (int a = 0; a < L.Q; ++a) e2w += (double)(C)L.w[a] * (L.ex[a] * L.ex[a] + L.ey[a] * L.ey[a]);
    k.e2w = (C)e2w;
    k.th0 = (C)((double)k.r2 * e2w - 2.0);
    for (int a = 0; a < L.Q; ++a) {
        k.mirror[a] = a;
        for (int b = 0; b < L.Q; ++b)
            if (L.ex[b] == L.ex[a] && L.ey[b] == -L.ey[a]) k.mirror[a] = b;
    }
    k.accom[0] = p.accom[0];
    k.accom[1] = p.accom[1];
    // Eq. (11)-(12): g^w_a / sum_{l<N} sum_{e.n>l} g^w = g^w_a / sum_{e.n>0} |e.n| g^w
    for (int wall = 0; wall < 2; ++wall) {
        double g[kMaxQ];
        const double Tw = p.thermal ? p.T_wall[wall] : 1.0;
        wall_equilibrium(L, p.eq_order, p.u_wall[wall], Tw, g);
        const int nsgn = wall == 0 ? 1 : -1;
        double den = 0;
        for (int a = 0; a < L.Q; ++a)
            if (nsgn * L.ey[a] > 0) den += nsgn * L.ey[a] * g[a];
        for (int a = 0; a < L.Q; ++a) k.wcoef[wall][a] = nsgn * L.ey[a] > 0 ? g[a] / den : 0.0;
    }
}

template void fill_consts<float>(KConsts<float> &, const LatticeHost &, const lbm_params &, int);
template void fill_consts<double>(KConsts<double> &, const LatticeHost &, const lbm_params &, int);

int staged_variant_count(int precision) {
    return dispatch_prec(precision, [&](auto P) { return Launch<decltype(P)::value>::staged_variants(); });
}

int direct_variant_count(int precision) {
    return dispatch_prec(precision, [&](auto P) { return Launch<decltype(P)::value>::direct_variants(); });
}

int dispatch_init_rest(SolverImpl &s) {
    CU(dispatch_prec(s.p.precision, [&](auto P) { return Launch<decltype(P)::value>::init_rest(s); }));
    return after_init(s);
}

int launch_step_variant(SolverImpl &s, int src, int dst, int kernel, int variant) {
    return dispatch_prec(s.p.precision, [&](auto P) {
        constexpr int PP = decltype(P)::value;
        return kernel == LBM_KERNEL_STAGED     ? Launch<PP>::step_staged(s, src, dst, variant)
               : kernel == LBM_KERNEL_CELLWARP ? Launch<PP>::step_cellwarp(s, src, dst)
                                               : Launch<PP>::step(s, src, dst, variant);
    });
}

}  // namespace lbm

using namespace lbm;

#define API_BEGIN try {
#define API_END                                                                    \
    }                                                                              \
    catch (const std::bad_alloc &) { set_error("host allocation failed"); return LBM_ENOMEM; } \
    catch (...) { set_error("unexpected exception"); return LBM_EINVAL; }

extern "C" {

const char *lbm_status_string(int st) {
    switch (st) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_EBUDGET: return "exceeds memory budget";
    case LBM_ENOTCONVERGED: return "not converged";
    case LBM_ENONFINITE: return "non-finite value";
    case LBM_ETIMEOUT: return "timeout";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EBUSY: return "busy";
    case LBM_ECANCELLED: return "cancelled";
    default: return "unknown status";
    }
}

int lbm_last_error(char *buf, size_t n) {
    if (buf && n) {
        std::strncpy(buf, g_err.c_str(), n - 1);
        buf[n - 1] = 0;
    }
    return LBM_OK;
}

int lbm_version(int *major, int *minor) {
    if (major) *major = 0;
    if (minor) *minor = 1;
    return LBM_OK;
}

int lbm_lattice_create(int kind, lbm_lattice **out) {
    API_BEGIN
    if (!out) { set_error("out is NULL"); return LBM_EINVAL; }
    *out = nullptr;
    if (kind != LBM_LATTICE_D2Q17 && kind != LBM_LATTICE_D2Q25 && kind != LBM_LATTICE_D2Q25B &&
        kind != LBM_LATTICE_D2Q37) {
        set_error("unknown lattice kind");
        return LBM_EINVAL;
    }
    lbm_lattice *l = new lbm_lattice;
    if (lattice_build(kind, l->L) != 0) {
        delete l;
        set_error("lattice moment system has no positive root");
        return LBM_EINVAL;
    }
    *out = l;
    return LBM_OK;
    API_END
}

int lbm_lattice_create_custom(int Q, const int8_t *e, const double *w, double r,
                              lbm_lattice **out) {
    API_BEGIN
    if (!out) { set_error("out is NULL"); return LBM_EINVAL; }
    *out = nullptr;
    lbm_lattice *l = new lbm_lattice;
    const char *why = "";
    if (lattice_build_custom(Q, e, w, r, l->L, &why) != 0) {
        delete l;
        set_error(why);
        return LBM_EINVAL;
    }
    *out = l;
    return LBM_OK;
    API_END
}

int lbm_lattice_destroy(lbm_lattice *lat) {
    delete lat;
    return LBM_OK;
}

int lbm_lattice_info(const lbm_lattice *lat, int *Q, double *r, int *ghost_depth, int *degree) {
    if (!lat) { set_error("lattice is NULL"); return LBM_EINVAL; }
    if (Q) *Q = lat->L.Q;
    if (r) *r = lat->L.r;
    if (ghost_depth) *ghost_depth = lat->L.ghost_depth;
    if (degree) *degree = lat->L.degree;
    return LBM_OK;
}

int lbm_lattice_tables(const lbm_lattice *lat, int8_t *e, double *w) {
    if (!lat) { set_error("lattice is NULL"); return LBM_EINVAL; }
    for (int a = 0; a < lat->L.Q; ++a) {
        if (e) { e[2 * a] = (int8_t)lat->L.ex[a]; e[2 * a + 1] = (int8_t)lat->L.ey[a]; }
        if (w) w[a] = lat->L.w[a];
    }
    return LBM_OK;
}

int lbm_lattice_verify(const lbm_lattice *lat, int degree, double *max_err) {
    if (!lat || !max_err || degree < 0 || degree > 16) { set_error("bad argument"); return LBM_EINVAL; }
    *max_err = lattice_isotropy_error(lat->L, degree);
    return LBM_OK;
}

void lbm_params_default(lbm_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->Nx = 1;
    p->Ny = 64;
    p->eq_order = 2;
    p->thermal = 0;
    p->Kn = 0.1;
    p->tau = 0;
    p->mu_exp = 1.0;
    p->u_wall[0] = -0.1;
    p->u_wall[1] = 0.1;
    p->T_wall[0] = p->T_wall[1] = 1.0;
    p->precision = LBM_FP64;
    p->kernel = LBM_KERNEL_AUTO;
    p->rho0 = 1.0;
    p->noise_amp = 0.0;
    p->seed = 7;
    p->accom[0] = p->accom[1] = 1.0;
}

int lbm_solver_required_bytes(const lbm_lattice *lat, const lbm_params *p, size_t *bytes) {
    if (!lat || !p || !bytes) { set_error("NULL argument"); return LBM_EINVAL; }
    int rc = check_params(lat->L, *p);
    if (rc) return rc;
    *bytes = layout_of(lat->L, *p).total;
    return LBM_OK;
}

int lbm_solver_create(const lbm_lattice *lat, const lbm_params *p, void *stream, void *device_mem,
                      size_t device_bytes, lbm_solver **out) {
    API_BEGIN
    if (!lat || !p || !out) { set_error("NULL argument"); return LBM_EINVAL; }
    *out = nullptr;
    int rc = check_params(lat->L, *p);
    if (rc) return rc;
    const Layout lo = layout_of(lat->L, *p);
    if (device_mem && (device_bytes < lo.total || ((uintptr_t)device_mem % kAlign))) {
        set_error("device_mem too small or not 256-byte aligned");
        return LBM_EINVAL;
    }
    lbm_solver *h = new lbm_solver();   // value-initialised: plain fields zero
    SolverImpl &s = h->s;
    s.L = lat->L;
    s.p = *p;
    s.stream = (cudaStream_t)stream;
    s.pitch = padded_pitch(p->Nx, p->precision);
    s.nt = tile_layout(p->Nx, p->precision).nt;
    s.elem = storage_elem_bytes(p->precision);
    s.owns_mem = device_mem == nullptr;
    s.dbytes = lo.total;
    if (s.owns_mem) {
        cudaError_t e = cudaMallocAsync((void **)&s.dmem, lo.total, s.stream);
        if (e != cudaSuccess) {
            delete h;
            set_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
        }
    } else {
        s.dmem = (char *)device_mem;
    }
    if (cudaMallocHost((void **)&s.pinned, 64 * sizeof(double)) != cudaSuccess) {
        if (s.owns_mem) cudaFreeAsync(s.dmem, s.stream);
        delete h;
        set_error("cudaMallocHost failed");
        return LBM_ENOMEM;
    }
    char *q = s.dmem;
    s.f[0] = q; q += lo.f_bytes;
    s.f[1] = q; q += lo.f_bytes;
    s.rho[0] = lo.rho_bytes ? (float *)q : nullptr; q += lo.rho_bytes;
    s.rho[1] = lo.rho_bytes ? (float *)q : nullptr; q += lo.rho_bytes;
    s.stage = (double *)q; q += lo.stage_bytes;
    s.prev = (double *)q; q += lo.prev_bytes;
    s.red = (double *)q;
    s.red_elems = lo.red_bytes / 8;
    s.derr = (int *)(s.red + 8 * 1024 + 48);
    s.sr = (unsigned *)(s.red + 8 * 1024 + 56);
    s.cur = 0;
    s.tm_key = -1;
    s.variant = 0;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (s.sm_count < 1) s.sm_count = 1;
        cudaError_t e = cudaMemsetAsync(s.derr, 0, sizeof(int), s.stream);
        if (e != cudaSuccess) {
            if (s.owns_mem) cudaFreeAsync(s.dmem, s.stream);
            cudaFreeHost(s.pinned);
            delete h;
            set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
            return LBM_ECUDA;
        }
    }
    fill_consts(s.kd, s.L, s.p, s.pitch);
    fill_consts(s.kf, s.L, s.p, s.pitch);
    s.kd.f0 = s.kf.f0 = s.f[0];
    s.kd.sr = s.kf.sr = s.sr;
    s.last_res = -1;
    *out = h;
    return LBM_OK;
    API_END
}

int lbm_solver_destroy(lbm_solver *h) {
    if (!h) return LBM_OK;
    SolverImpl &s = h->s;
    if (s.step_graph) cudaGraphExecDestroy(s.step_graph);
    if (s.owns_mem && s.dmem) cudaFreeAsync(s.dmem, s.stream);
    cudaStreamSynchronize(s.stream);
    if (s.pinned) cudaFreeHost(s.pinned);
    delete h;
    return LBM_OK;
}

int lbm_solver_init(lbm_solver *h) {
    API_BEGIN
    if (!h) { set_error("NULL solver"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    CU(dispatch_prec(s.p.precision, [&](auto P) { return Launch<decltype(P)::value>::init_rest(s); }));
    return after_init(s);
    API_END
}

int lbm_solver_init_fields(lbm_solver *h, const double *rho, const double *ux, const double *uy,
                           const double *T) {
    API_BEGIN
    if (!h || !rho) { set_error("NULL solver or rho"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    const size_t n = (size_t)s.p.Nx * s.p.Ny;
    const double *src[4] = {rho, ux, uy, T};
    double *dst[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 4; ++i)
        if (src[i]) {
            dst[i] = s.stage + i * n;
            CU(cudaMemcpyAsync(dst[i], src[i], n * sizeof(double), cudaMemcpyHostToDevice, s.stream));
        }
    CU(dispatch_prec(s.p.precision, [&](auto P) {
        return Launch<decltype(P)::value>::init_fields(s, dst[0], dst[1], dst[2], dst[3]);
    }));
    return after_init(s);
    API_END
}

namespace lbm {
namespace {
// A CUDA graph of kGraphSteps step launches starting from buffer 0, captured
// once per kernel choice on a private stream and replayed on the solver's.
int ensure_step_graph(SolverImpl &s, int kern) {
    if (s.step_graph && s.graph_kernel == kern && s.graph_variant == s.variant) return LBM_OK;
    if (s.step_graph) {
        cudaGraphExecDestroy(s.step_graph);
        s.step_graph = nullptr;
    }
    cudaStream_t cs;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t keep = s.stream;
    s.stream = cs;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i)
        e = (cudaError_t)launch_step_variant(s, i & 1, (i & 1) ^ 1, kern, s.variant);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    s.stream = keep;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s.step_graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        s.step_graph = nullptr;
        set_error(std::string("step graph: ") + cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    s.graph_kernel = kern;
    s.graph_variant = s.variant;
    return LBM_OK;
}
}  // namespace
}  // namespace lbm

// NVTX range for the duration of a scope (visible in profilers' timelines)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

int lbm_solver_step(lbm_solver *h, int64_t n) {
    API_BEGIN
    NvtxRange nvtx("lbm_solver_step");
    if (!h || n < 0) { set_error("NULL solver or negative step count"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    const int kern = effective_kernel(s);
    auto one = [&]() -> int {
        CU(launch_step_variant(s, s.cur, s.cur ^ 1, kern, s.variant));
        s.cur ^= 1;
        ++s.steps;
        return LBM_OK;
    };
    int rc;
    if (n >= 2 * kGraphSteps) {
        if ((rc = ensure_step_graph(s, kern))) return rc;
        if (s.cur == 1) { if ((rc = one())) return rc; --n; }
        while (n >= kGraphSteps) {
            CU(cudaGraphLaunch(s.step_graph, s.stream));
            s.steps += kGraphSteps;
            n -= kGraphSteps;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        if ((rc = one())) return rc;
    return LBM_OK;
    API_END
}

int lbm_solver_sync(lbm_solver *h) {
    if (!h) { set_error("NULL solver"); return LBM_EINVAL; }
    CU(cudaStreamSynchronize(h->s.stream));
    return check_device_error(h->s);
}

int lbm_solver_get_f(lbm_solver *h, double *f) {
    API_BEGIN
    if (!h || !f) { set_error("NULL argument"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    const size_t n = (size_t)s.p.Nx * s.p.Ny;
    for (int a = 0; a < s.L.Q; ++a) {
        CU(dispatch_prec(s.p.precision, [&](auto P) { return Launch<decltype(P)::value>::plane_to_f64(s, a, s.stage); }));
        CU(cudaMemcpyAsync(f + a * n, s.stage, n * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
        CU(cudaStreamSynchronize(s.stream));
    }
    return LBM_OK;
    API_END
}

int lbm_solver_set_f(lbm_solver *h, const double *f) {
    API_BEGIN
    if (!h || !f) { set_error("NULL argument"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    const size_t n = (size_t)s.p.Nx * s.p.Ny;
    if (s.p.precision == LBM_BF16DEV) {
        // density of each cell first: d_a = f_a - w_a rho needs it
        double *acc = s.stage + n;
        for (int a = 0; a < s.L.Q; ++a) {
            CU(cudaMemcpyAsync(s.stage, f + a * n, n * sizeof(double), cudaMemcpyHostToDevice, s.stream));
            CU(launch_accumulate(s.stream, acc, s.stage, (long long)n, a == 0));
        }
        CU(launch_rho_plane(s.stream, s.rho[s.cur], acc, s.kf));
    }
    for (int a = 0; a < s.L.Q; ++a) {
        CU(cudaMemcpyAsync(s.stage, f + a * n, n * sizeof(double), cudaMemcpyHostToDevice, s.stream));
        CU(dispatch_prec(s.p.precision, [&](auto P) { return Launch<decltype(P)::value>::plane_from_f64(s, a, s.stage); }));
    }
    CU(cudaStreamSynchronize(s.stream));
    return after_init(s);
    API_END
}

int lbm_solver_macros(lbm_solver *h, double *rho, double *ux, double *uy, double *T) {
    API_BEGIN
    if (!h) { set_error("NULL solver"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    const size_t n = (size_t)s.p.Nx * s.p.Ny;
    double *d[4] = {s.stage, s.stage + n, s.stage + 2 * n, s.stage + 3 * n};
    double *hst[4] = {rho, ux, uy, T};
    CU(dispatch_prec(s.p.precision, [&](auto P) {
        return Launch<decltype(P)::value>::macros(s, hst[0] ? d[0] : nullptr, hst[1] ? d[1] : nullptr,
                                                  hst[2] ? d[2] : nullptr, hst[3] ? d[3] : nullptr);
    }));
    for (int i = 0; i < 4; ++i)
        if (hst[i]) CU(cudaMemcpyAsync(hst[i], d[i], n * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
    CU(cudaStreamSynchronize(s.stream));
    return LBM_OK;
    API_END
}

int lbm_solver_macros_mean(lbm_solver *h, int64_t nsteps, double *rho, double *ux, double *uy,
                           double *T) {
    API_BEGIN
    NvtxRange nvtx("lbm_solver_macros_mean");
    if (!h || nsteps < 1) { set_error("NULL solver or nsteps < 1"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    const size_t n = (size_t)s.p.Nx * s.p.Ny;
    double *d[4] = {s.stage, s.stage + n, s.stage + 2 * n, s.stage + 3 * n};
    const int kern = effective_kernel(s);
    for (int64_t i = 0; i < nsteps; ++i) {
        CU(launch_step_variant(s, s.cur, s.cur ^ 1, kern, s.variant));
        s.cur ^= 1;
        ++s.steps;
        CU(dispatch_prec(s.p.precision, [&](auto P) {
            return Launch<decltype(P)::value>::macros(s, d[0], d[1], d[2], d[3], i > 0 ? 1 : 0);
        }));
    }
    double *hst[4] = {rho, ux, uy, T};
    for (int i = 0; i < 4; ++i)
        if (hst[i]) CU(cudaMemcpyAsync(hst[i], d[i], n * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
    CU(cudaStreamSynchronize(s.stream));
    if (int rc = check_device_error(s)) return rc;
    for (int i = 0; i < 4; ++i)
        if (hst[i])
            for (size_t c = 0; c < n; ++c) hst[i][c] /= (double)nsteps;
    return LBM_OK;
    API_END
}

int lbm_solver_fluxes(lbm_solver *h, double *sxx, double *sxy, double *syy, double *qx,
                      double *qy) {
    API_BEGIN
    if (!h) { set_error("NULL solver"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    const size_t n = (size_t)s.p.Nx * s.p.Ny;
    double *hst[5] = {sxx, sxy, syy, qx, qy};
    double *d[5];
    for (int i = 0; i < 5; ++i) d[i] = hst[i] ? s.stage + i * n : nullptr;
    CU(dispatch_prec(s.p.precision, [&](auto P) {
        return Launch<decltype(P)::value>::fluxes(s, d[0], d[1], d[2], d[3], d[4]);
    }));
    for (int i = 0; i < 5; ++i)
        if (hst[i]) CU(cudaMemcpyAsync(hst[i], d[i], n * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
    CU(cudaStreamSynchronize(s.stream));
    return LBM_OK;
    API_END
}

int lbm_solver_state_bytes(lbm_solver *h, size_t *bytes) {
    if (!h || !bytes) { set_error("NULL argument"); return LBM_EINVAL; }
    const SolverImpl &s = h->s;
    const size_t fb = (size_t)s.L.Q * s.p.Ny * s.nt * s.pitch * s.elem;
    const size_t rb = s.rho[0] ? (size_t)s.p.Ny * s.nt * s.pitch * 4 : 0;
    *bytes = 64 + fb + rb;
    return LBM_OK;
}

namespace {
struct CkptHeader {
    char magic[8];
    int32_t Q, Nx, Ny, pitch, precision, pad;
    int64_t steps;
    double mass0;
};
}  // namespace

int lbm_solver_get_state(lbm_solver *h, void *buf, size_t bytes) {
    API_BEGIN
    size_t need = 0;
    if (!buf || lbm_solver_state_bytes(h, &need) || bytes < need) { set_error("buffer too small"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    CkptHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "LBMGB300", 8);
    hd.Q = s.L.Q; hd.Nx = s.p.Nx; hd.Ny = s.p.Ny; hd.pitch = s.pitch; hd.precision = s.p.precision;
    hd.steps = s.steps; hd.mass0 = s.mass0;
    char *b = (char *)buf;
    std::memset(b, 0, 64);
    std::memcpy(b, &hd, sizeof(hd));
    const size_t fb = (size_t)s.L.Q * s.p.Ny * s.nt * s.pitch * s.elem;
    CU(cudaMemcpyAsync(b + 64, s.f[s.cur], fb, cudaMemcpyDeviceToHost, s.stream));
    if (s.rho[0]) CU(cudaMemcpyAsync(b + 64 + fb, s.rho[s.cur], (size_t)s.p.Ny * s.nt * s.pitch * 4, cudaMemcpyDeviceToHost, s.stream));
    CU(cudaStreamSynchronize(s.stream));
    return LBM_OK;
    API_END
}

int lbm_solver_set_state(lbm_solver *h, const void *buf, size_t bytes) {
    API_BEGIN
    size_t need = 0;
    if (!buf || lbm_solver_state_bytes(h, &need) || bytes != need) { set_error("state size mismatch"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, "LBMGB300", 8) || hd.Q != s.L.Q || hd.Nx != s.p.Nx || hd.Ny != s.p.Ny ||
        hd.pitch != s.pitch || hd.precision != s.p.precision) {
        set_error("checkpoint does not match this solver");
        return LBM_EINVAL;
    }
    const char *b = (const char *)buf;
    const size_t fb = (size_t)s.L.Q * s.p.Ny * s.nt * s.pitch * s.elem;
    CU(cudaMemcpyAsync(s.f[s.cur], b + 64, fb, cudaMemcpyHostToDevice, s.stream));
    if (s.rho[0]) CU(cudaMemcpyAsync(s.rho[s.cur], b + 64 + fb, (size_t)s.p.Ny * s.nt * s.pitch * 4, cudaMemcpyHostToDevice, s.stream));
    CU(cudaStreamSynchronize(s.stream));
    s.steps = hd.steps;
    s.mass0 = hd.mass0;
    if (int rc = set_round_counter(s)) return rc;
    const long long n = (long long)s.p.Nx * s.p.Ny;
    CU(dispatch_prec(s.p.precision, [&](auto P) {
        return Launch<decltype(P)::value>::macros(s, nullptr, s.prev, nullptr, s.prev + n);
    }));
    CU(cudaStreamSynchronize(s.stream));
    return LBM_OK;
    API_END
}

int lbm_solver_run_to_residual(lbm_solver *h, double tol, int64_t max_steps, int32_t check_every,
                               int64_t *steps, double *res) {
    API_BEGIN
    NvtxRange nvtx("lbm_solver_run_to_residual");
    if (!h || check_every < 1 || max_steps < 0 || !(tol >= 0)) { set_error("bad argument"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    const long long n = (long long)s.p.Nx * s.p.Ny;
    const double Tref = 0.5 * (s.p.T_wall[0] + s.p.T_wall[1]);
    const int nb = reduction_blocks(n);
    int64_t done = 0;
    double best = INFINITY, r = INFINITY;
    int since_best = 0;
    int status = LBM_ENOTCONVERGED;
    int rc = LBM_OK;
    s.res_history.clear();
    while (done < max_steps) {
        int64_t k = check_every;
        if (done + k > max_steps) k = max_steps - done;
        rc = lbm_solver_step(h, k);
        if (rc) return rc;
        done += k;
        CU(dispatch_prec(s.p.precision, [&](auto P) {
            return Launch<decltype(P)::value>::macros(s, nullptr, s.stage + n, nullptr, s.stage + 3 * n);
        }));
        CU(launch_residual_partials(s.stream, s.stage + n, s.stage + 3 * n, s.prev, s.prev + n, n, Tref, s.red, nb));
        CU(launch_final_sum(s.stream, s.red, nb, 5, s.red + 8 * 1024));
        CU(cudaMemcpyAsync(s.pinned, s.red + 8 * 1024, 5 * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
        CU(cudaStreamSynchronize(s.stream));
        if ((rc = check_device_error(s))) return rc;
        const double *v = s.pinned;
        if (v[4] > 0) { status = LBM_ENONFINITE; r = NAN; break; }
        r = std::sqrt(v[0]) / std::fmax(std::sqrt(v[1]), 1e-30);
        if (s.p.thermal) r = std::fmax(r, std::sqrt(v[2]) / std::fmax(std::sqrt(v[3]), 1e-30));
        s.res_history.emplace_back(s.steps, r);
        if (!std::isfinite(r)) { status = LBM_ENONFINITE; break; }
        if (r <= tol) { status = LBM_OK; break; }
        if (r < best) { best = r; since_best = 0; }
        else if (++since_best >= 50) { status = LBM_ENOTCONVERGED; set_error("residual stagnated"); break; }
    }
    s.last_res = r;
    if (steps) *steps = done;
    if (res) *res = r;
    if (status == LBM_ENOTCONVERGED && since_best < 50) set_error("max_steps reached");
    if (status == LBM_ENONFINITE) set_error("non-finite residual");
    return status;
    API_END
}

int lbm_solver_residual_history(lbm_solver *h, int64_t *steps, double *res, int32_t max,
                                int32_t *n) {
    if (!h || !n || max < 0 || (max > 0 && (!steps || !res))) { set_error("bad argument"); return LBM_EINVAL; }
    const auto &hist = h->s.res_history;
    const int k = (int)std::min<size_t>(hist.size(), (size_t)max);
    for (int i = 0; i < k; ++i) {
        steps[i] = hist[i].first;
        res[i] = hist[i].second;
    }
    *n = (int32_t)hist.size();
    return LBM_OK;
}

int lbm_solver_stats(lbm_solver *h, lbm_stats *st) {
    API_BEGIN
    if (!h || !st) { set_error("NULL argument"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    double m = 0;
    int rc = sum_rho(s, &m);
    if (rc) return rc;
    std::vector<double> w(2 * (size_t)s.p.Nx);
    rc = lbm_solver_wall_mass(h, w.data());
    if (rc) return rc;
    st->steps = s.steps;
    st->mass0 = s.mass0;
    st->mass = m;
    st->mass_drift = std::fabs(m - s.mass0) / s.mass0;
    st->residual = s.last_res;
    st->wall_in[0] = st->wall_in[1] = 0;
    for (int wall = 0; wall < 2; ++wall)
        for (int x = 0; x < s.p.Nx; ++x) st->wall_in[wall] += w[(size_t)wall * s.p.Nx + x];
    return LBM_OK;
    API_END
}

int lbm_solver_wall_mass(lbm_solver *h, double *m_in) {
    API_BEGIN
    if (!h || !m_in) { set_error("NULL argument"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    CU(dispatch_prec(s.p.precision, [&](auto P) { return Launch<decltype(P)::value>::wall_mass(s, s.stage); }));
    CU(cudaMemcpyAsync(m_in, s.stage, 2 * (size_t)s.p.Nx * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
    CU(cudaStreamSynchronize(s.stream));
    return LBM_OK;
    API_END
}

int lbm_solver_set_kernel(lbm_solver *h, int32_t kernel, int32_t variant) {
    if (!h) { set_error("NULL solver"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    if (kernel < LBM_KERNEL_AUTO || kernel > LBM_KERNEL_CELLWARP) { set_error("bad kernel"); return LBM_EINVAL; }
    const int nv = kernel == LBM_KERNEL_STAGED     ? staged_variant_count(s.p.precision)
                   : kernel == LBM_KERNEL_CELLWARP ? 1
                                                   : direct_variant_count(s.p.precision);
    if (kernel == LBM_KERNEL_STAGED && nv == 0) {
        set_error("the staged kernel is not built for this precision");
        return LBM_EINVAL;
    }
    if (variant < 0 || variant >= nv) { set_error("bad variant"); return LBM_EINVAL; }
    if (kernel == LBM_KERNEL_STAGED && s.nt != 1) {
        set_error("the staged kernel runs grids stored as one x-tile only (Nx + 8 <= tile pitch)");
        return LBM_EINVAL;
    }
    s.p.kernel = kernel;
    s.variant = variant;
    return LBM_OK;
}

int lbm_solver_set_wait_limit(lbm_solver *h, uint64_t ns) {
    if (!h) { set_error("NULL solver"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    s.kf.wait_ns = s.kd.wait_ns = (unsigned long long)ns;
    // the replayed step graph holds the kernel constants of its capture
    if (s.step_graph) {
        CU(cudaStreamSynchronize(s.stream));
        cudaGraphExecDestroy(s.step_graph);
        s.step_graph = nullptr;
    }
    return LBM_OK;
}

int lbm_solver_kernel_info(lbm_solver *h, int32_t *kernel, int32_t *variant, int32_t *nvariants) {
    if (!h) { set_error("NULL solver"); return LBM_EINVAL; }
    if (kernel) *kernel = effective_kernel(h->s);
    if (variant) *variant = h->s.variant;
    if (nvariants) *nvariants = staged_variant_count(h->s.p.precision);
    return LBM_OK;
}

int lbm_solver_variant_count(lbm_solver *h, int32_t kernel, int32_t *n) {
    if (!h || !n || (kernel != LBM_KERNEL_DIRECT && kernel != LBM_KERNEL_STAGED &&
                     kernel != LBM_KERNEL_CELLWARP)) {
        set_error("bad argument");
        return LBM_EINVAL;
    }
    *n = kernel == LBM_KERNEL_STAGED     ? staged_variant_count(h->s.p.precision)
         : kernel == LBM_KERNEL_CELLWARP ? 1
                                         : direct_variant_count(h->s.p.precision);
    return LBM_OK;
}

int lbm_solver_autotune(lbm_solver *h, int32_t trial_steps, int32_t *best_kernel,
                        int32_t *best_variant, double *best_ms) {
    API_BEGIN
    if (!h || trial_steps < 1) { set_error("bad argument"); return LBM_EINVAL; }
    SolverImpl &s = h->s;
    int rc = autotune_solver(s, trial_steps);
    if (rc) return rc;
    if (best_kernel) *best_kernel = s.p.kernel;
    if (best_variant) *best_variant = s.variant;
    if (best_ms) *best_ms = s.tuned_ms;
    return LBM_OK;
    API_END
}

}  // extern "C"
