// Internal declarations shared by the host C-ABI layer and the kernel
// launchers of the library.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda.h>
#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

constexpr int kMaxQ = 37;
constexpr int kMaxShells = 8;
constexpr int kPadL = 4;          // periodic image columns kept left of x = 0
constexpr long long kCellwarpAutoCells = 4096;   // LBM_KERNEL_AUTO: one warp per cell up to here
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;   // bounded device waits: 2 s
// Segment pitches (elements, 128-byte multiples) for which the step kernel
// has instantiations with the pitch a compile-time constant: a grid of Nx +
// 2 kPadL > kPitchClass[p][0] / 2 columns is stored with the smallest class
// that holds its row (one x-tile; at most half of the segment is padding,
// which no kernel touches), or, past the widest class, as x-tiles of it; a
// narrower grid keeps a compact pitch.  Wider tiles measured faster (D2Q37 at
// 4096 x 2048: FP32 one tile of 4224 0.378 ms per step against four of 1056
// 0.406 ms; BF16DEV one tile 0.325 ms against two of 2112 0.337 ms): fewer
// separate row segments are streamed at once.
constexpr int kPitchClasses = 3;
inline constexpr int pitch_class(int precision, int c) {
    return precision == LBM_BF16DEV || precision == LBM_BF16SHIFT
               ? (c == 0 ? 1088 : c == 1 ? 2112 : 4224)
               : (c == 0 ? 1056 : c == 1 ? 2112 : 4224);
}
inline constexpr int widest_pitch_class(int) { return kPitchClasses - 1; }
// Columns of tile t (all tiles hold tw but the last, which holds the rest).
template <class K>
__host__ __device__ __forceinline__ int tile_width(const K &k, int t) {
    return t < k.nt - 1 ? k.tw : k.Nx - (k.nt - 1) * k.tw;
}

struct LatticeHost {
    int kind;
    int Q;
    int ex[kMaxQ], ey[kMaxQ], shell[kMaxQ];
    double w[kMaxQ];
    double r;
    int ghost_depth;
    int degree;
};

int lattice_build(int kind, LatticeHost &L);
// A built-in velocity set (Q = 17, 25 or 37) with the caller's weights and
// scale; 0 or -1 with *why set.
int lattice_build_custom(int Q, const int8_t *e, const double *w, double r, LatticeHost &L,
                         const char **why);
double lattice_isotropy_error(const LatticeHost &L, int degree);

// Per-solve constants handed to every kernel by value.  C is the compute type
// (float or double); wall coefficients stay FP64 (the wall mass flux is
// normalised in FP64).
// Single-domain storage: the columns are split into nt x-tiles; tile t holds
// columns [t tw, min((t + 1) tw, Nx)) and stores, row by row and within a row
// velocity by velocity, a segment of `pitch` elements: kPadL halo columns (the
// previous tile's last kPadL columns, periodic in x), the tile's columns,
// kPadL halo columns (the next tile's first ones), padding to 128 bytes.
// Element (a, j, x) of a state buffer sits at t * tile_elems + (j Q + a) pitch
// + x - t tw + kPadL; the BF16DEV density of (j, x) at t * tile_rho + j pitch +
// x - t tw + kPadL.  One tile (nt = 1) holds every column, its halos being the
// periodic images; wide grids use tiles of a fixed pitch (pitch_class), so the
// step kernel's Q shifted accesses are compile-time offsets from one base.
template <class C>
struct KConsts {
    int Nx, Ny, Q;
    int pitch;                // elements per (tile, row, velocity) segment
    int nt, tw;               // number of x-tiles, columns per tile (the last: the rest)
    long long tile_elems;     // Ny * Q * pitch: one tile of a state buffer
    long long tile_rho;       // Ny * pitch: one tile of the density plane
    int thermal, eq_order;
    int const_tau;            // 1: tau_lat is used as is
    int mu_is_one;            // mu = T: tau independent of T
    C r, r2;                  // lattice scale and its square
    C K;                      // sqrt(2/pi) Kn r Ny : tau/dt = K T^(mu_exp-1) / rho
    C tau_lat;                // constant tau / dt
    C mu_m1;                  // mu_exp - 1
    C wsh[kMaxShells];        // shell weights
    C c2sh[kMaxShells];       // |c|^2 = r^2 |e|^2 of each shell
    C w[kMaxQ];               // per-velocity weights
    C e2w;                    // sum_a |e_a|^2 w_a (= D / r^2 up to rounding)
    C th0;                    // r^2 e2w - D, formed in FP64: theta = T - 1 of the
                              // shifted storage without cancellation against D
    // byte offsets of the step kernel's accesses from the cell's own element
    // (a = 0) in its tile
    long long b_src[kMaxQ];   // ((a - e_ay Q) pitch - e_ax) elements: pull source
    long long b_dst[kMaxQ];   // a pitch elements: store
    long long b_rho[kMaxQ];   // (-e_ay pitch - e_ax) FP32 elements: source density (BF16DEV)
    int mirror[kMaxQ];        // velocity with (e_x, -e_y): specular partner
    double accom[2];          // wall accommodation (1: diffuse)
    double wcoef[2][kMaxQ];   // g^w_a / D_w (0 unless a leaves the wall)
    // step counter of the stochastic BF16 rounding: sr[b] is the number of
    // steps done when state buffer b (base f0 for b = 0) is the source
    const void *f0;
    unsigned *sr;
    // limit of each bounded mbarrier wait of the staged kernel (ns); the
    // wait for copies in flight before a CTA exits keeps its own fixed limit
    unsigned long long wait_ns;
};

// Kernel constants of one solve (Eq. (4)-(5) factors, Eq. (11)-(12) wall
// coefficients); defined in api.cpp.
template <class C>
void fill_consts(KConsts<C> &k, const LatticeHost &L, const lbm_params &p, int pitch);

struct SolverImpl {
    LatticeHost L;
    lbm_params p;
    cudaStream_t stream;
    char *dmem;
    size_t dbytes;
    bool owns_mem;
    void *f[2];               // storage buffers, [Q][Ny][pitch]
    float *rho[2];            // BF16DEV only: density planes [Ny][pitch]
    double *stage;            // 4 FP64 planes [Ny][Nx] (macros / conversions)
    double *prev;             // 2 FP64 planes: u_x, T at the previous check
    double *red;              // reduction partials
    size_t red_elems;
    double *pinned;           // host pinned results of reductions (16 doubles)
    int cur;                  // buffer holding the current state
    int pitch;                // segment pitch of the x-tiles (KConsts::pitch)
    int nt;                   // number of x-tiles
    size_t elem;              // storage bytes per population
    int64_t steps;
    double mass0;
    double last_res;
    std::vector<std::pair<int64_t, double>> res_history;   // (steps, residual) of the last steady-state run
    double wall_in[2];
    KConsts<float> kf;
    KConsts<double> kd;
    int sm_count;
    int *derr;                // device error flags of the staged kernel
    unsigned *sr;             // step counters of the stochastic BF16 rounding (2)
    int variant;              // staged-kernel variant in use (see launchers)
    long long tm_key;         // (TX, TY) the tensor maps were encoded for; -1 none
    CUtensorMap tm_f[2];      // 3-D maps (x, y, a) of the two state buffers
    CUtensorMap tm_r[2];      // 2-D maps of the BF16DEV density planes
    double tuned_ms;          // step time of the autotuned choice
    cudaGraphExec_t step_graph;   // kGraphSteps launches from buffer 0, replayed
    int graph_kernel, graph_variant;
};

constexpr int kGraphSteps = 64;   // steps per replayed graph (even: parity kept)

// Encode tm_f / tm_r for boxes of (TX + 2 kPadL) x TY (density: TY + 6 rows).
int encode_tensor_maps(SolverImpl &s, int TX, int TY);
// The x-tiling of a grid: pitch, number of tiles, columns per tile.
struct TileLayout {
    int pitch, nt, tw;
};
TileLayout tile_layout(int Nx, int precision);
int staged_variant_count(int precision);
int direct_variant_count(int precision);
int launch_step_variant(SolverImpl &s, int src, int dst, int kernel, int variant);
// Re-initialise the state as lbm_solver_init does (rest equilibrium + noise).
int dispatch_init_rest(SolverImpl &s);
// Pick the fastest step kernel / variant for this solver (autotune.cpp).
int autotune_solver(SolverImpl &s, int trial_steps);

size_t storage_elem_bytes(int precision);
int padded_pitch(int Nx, int precision);

void set_error(const std::string &msg);

}  // namespace lbm

struct lbm_lattice {
    lbm::LatticeHost L;
};
struct lbm_solver {
    lbm::SolverImpl s;
};
