// Internal declarations shared by the host C-ABI layer and the kernel
// launchers of the library.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace lbm {

constexpr int kMaxQ = 37;
constexpr int kMaxShells = 8;
constexpr int kPadL = 4;          // periodic image columns kept left of x = 0

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
double lattice_isotropy_error(const LatticeHost &L, int degree);

// Per-solve constants handed to every kernel by value.  C is the compute type
// (float or double); wall coefficients stay FP64 (the wall mass flux is
// normalised in FP64).
template <class C>
struct KConsts {
    int Nx, Ny, pitch;
    long long plane;          // elements per velocity plane = Ny * pitch
    int thermal, eq_order;
    int const_tau;            // 1: tau_lat is used as is
    int mu_is_one;            // mu = T: tau independent of T
    C r, r2;                  // lattice scale and its square
    C K;                      // sqrt(2/pi) Kn r Ny : tau/dt = K T^(mu_exp-1) / rho
    C tau_lat;                // constant tau / dt
    C mu_m1;                  // mu_exp - 1
    C wsh[kMaxShells];        // shell weights
    C w[kMaxQ];               // per-velocity weights
    double wcoef[2][kMaxQ];   // g^w_a / D_w (0 unless a leaves the wall)
};

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
    int pitch;
    size_t elem;              // storage bytes per population
    int64_t steps;
    double mass0;
    double last_res;
    double wall_in[2];
    KConsts<float> kf;
    KConsts<double> kd;
};

size_t storage_elem_bytes(int precision);
int padded_pitch(int Nx, int precision);

// ---- kernel launchers (return cudaError_t as int) --------------------------
int launch_step(SolverImpl &s, int src, int dst);
int launch_init_rest(SolverImpl &s);
int launch_init_fields(SolverImpl &s, const double *rho, const double *ux,
                       const double *uy, const double *T);   // device planes
int launch_plane_to_f64(SolverImpl &s, int a, double *out);   // logical plane
int launch_plane_from_f64(SolverImpl &s, int a, const double *in);
int launch_fill_pads(SolverImpl &s);                           // after set_f
int launch_macros(SolverImpl &s, double *rho, double *ux, double *uy, double *T);
int launch_wall_mass(SolverImpl &s, double *m_in);             // [2][Nx]
// Reductions: out[0..] written to s.pinned after the stream reaches them.
int launch_residual(SolverImpl &s, int thermal, double Tref);  // uses stage + prev
int launch_mass(SolverImpl &s);                                // sum rho

void set_error(const std::string &msg);

}  // namespace lbm

struct lbm_lattice {
    lbm::LatticeHost L;
};
struct lbm_solver {
    lbm::SolverImpl s;
};
