// Slot table of the batched / serving path, shared by the chunk kernel and
// the host runtime.
#pragma once

#include "lbm_internal.h"

namespace lbm {

// States of a slot (SlotStatus::state).
constexpr int kSlotIdle = 0;
constexpr int kSlotRunning = 1;
constexpr int kSlotConverged = 2;
constexpr int kSlotNonFinite = 3;
constexpr int kSlotMaxSteps = 4;
constexpr int kSlotStagnated = 5;
constexpr int kSlotCancelled = 6;         // set by the host; the kernel skips the slot

// Most velocities leaving one wall (e.n > 0): 15 for D2Q37.
constexpr int kMaxOut = 16;
// Most chunks one launch runs for one slot.
constexpr int kMaxSub = 16;
// Chunks per launch of a slot on a cluster of cl CTAs: about the factor by
// which the cluster shortens a step of a tall column, conservatively, so that
// a cluster slot is rarely the one a launch waits for.
inline int batch_sub_chunks(int cl) { return cl <= 2 ? 1 : cl / 2; }

struct SlotDesc {
    int Q;                    // 17, 25 or 37 (0: idle slot)
    int Ny;
    int cur;                  // buffer holding the current state (0 / 1)
    int check_every;          // residual every check_every chunks
    int chunk_steps;          // steps this slot runs per chunk launch
    int cl;                   // CTAs of the slot's cluster: 1, 2, 4, 8 or 16
    int sub;                  // chunks per launch (a cluster runs several, so
                              // that it keeps pace with one-CTA slots' launches)
    long long f_off;          // element offset of buffer 0 in the pool
    long long prev_off;       // element offset of the previous-check u_x, T
    double tol;               // target of the extrapolated distance to steady state
    long long max_steps;
    double u_ref;             // velocity scale of the change measure: max |u_wall|
    double mass0;             // the column's mass at admission (sum of rho)
    double precise_from;      // change per check below which the slot switches
                              // to stochastic rounding and conserving increments
    // initial state: u_x(y) = u0 + u1 (y - 1/2), T(y) = T0 + T1 y + T2 y (1 - y)
    // at rho = 1 (y = (j + 1/2) / Ny); rest: u0 = u1 = T1 = T2 = 0, T0 = 1
    double init_u0, init_u1, init_T0, init_T1, init_T2;
    // incoming terms of Eq. (12)'s numerator, built on the host: wall w (0
    // bottom, 1 top), term l < nterm is velocity term_a[w][l] at distance
    // term_row[w][l] from the wall
    int nterm;                // < 32: lane nterm of the wall warp carries wterm
    int nout;                 // outgoing velocities per wall (e.n > 0), <= kMaxOut
    signed char term_a[2][32];
    signed char term_row[2][32];
    signed char out_a[2][kMaxOut];
    double wterm[2];          // sum over the incoming terms of their weights w_a
    double out_c[2][kMaxOut]; // g^w_a / D_w of outgoing velocity out_a[w][l]
    double out_w[2][kMaxOut]; // its weight w_a as the FP32 storage holds it
    KConsts<float> k;         // per-instance constants (Nx = 1, pitch = 1)
};

struct SlotStatus {
    long long steps;          // steps run since admission
    double res;               // last change over one check: max(L-inf |du_x| / u_ref,
                              // thermal: L-inf |dT|)
    double res_prev;          // change over the check before
    double err_est;           // extrapolated distance to the steady state (same units)
    double best_res;          // smallest change so far
    double mass;              // sum of rho (FP64) at the last check
    int state;                // kSlot*
    int checks;
    int since_best;           // checks without a new smallest residual
    int chunks;               // chunks run since admission
    int precise;              // 0: round-to-nearest collision; 1: conserving
                              // increments with stochastic rounding (2: switching)
};

// Cluster sizes of the slot classes.
constexpr int kBatchClasses = 5;
constexpr int kBatchClassCL[kBatchClasses] = {1, 2, 4, 8, 16};
// Tallest column a request may have.
constexpr int kMaxNy = 8192;
// Rows of the residual's partial sums (one warp each) and their most per slot.
constexpr int kResidualChunk = 32;
constexpr int kMaxResidualChunks = kMaxNy / kResidualChunk;

// Rows per CTA of a column of Ny rows on a cluster of CL CTAs: all of them on
// one CTA, else ceil(Ny / CL) rounded up to whole residual chunks, so that no
// chunk straddles two CTAs.
__host__ __device__ inline int batch_rows_per_cta(int Ny, int CL) {
    if (CL <= 1) return Ny;
    const int r = (Ny + CL - 1) / CL;
    return (r + kResidualChunk - 1) / kResidualChunk * kResidualChunk;
}
// A split is usable when every CTA, the last included, gets >= 32 rows.
__host__ __device__ inline bool batch_split_ok(int Ny, int CL) {
    if (CL == 1) return Ny >= 6;
    const int R = batch_rows_per_cta(Ny, CL);
    return (CL == 2 || CL == 4 || CL == 8 || CL == 16) && (CL - 1) * R + 32 <= Ny;
}
// The largest cluster a column of Ny rows may use: the smallest CL whose CTAs
// get at most `rows` rows each (max_cl if none does), reduced until the split
// is usable and fits the CTA budget.
inline int batch_cluster_size(int Ny, int rows, int max_ctas, int max_cl) {
    int cl = 1;
    while (cl < max_cl && batch_rows_per_cta(Ny, cl) > rows) cl *= 2;
    while (cl > 1 && (cl > max_ctas || !batch_split_ok(Ny, cl))) cl /= 2;
    return cl;
}

int preload_batch_kernels();
// 16 when the device can schedule a 16-CTA cluster of the chunk kernel (a
// non-portable size), else 8.
int batch_max_cluster();
// dbg: 8 device ints; dbg[0] != 0 records the first invalid descriptor or
// read-out offset a kernel met (and skipped).
// One chunk of the slots [slot0, slot0 + nlanes), each on a cluster of CL
// CTAs; part: kMaxResidualChunks x 6 FP64 residual partials per slot of the
// whole table.
int launch_batch_chunk(cudaStream_t st, SlotDesc *desc, SlotStatus *status, float *pool,
                       double *part, int slot0, int nlanes, int CL, long long pool_elems,
                       int *dbg);
int launch_batch_init(cudaStream_t st, SlotDesc *desc, float *pool, const int *slots, int n,
                      float rho0, int nslots, long long pool_elems, int *dbg);
int launch_batch_macros(cudaStream_t st, const SlotDesc *desc, const float *pool,
                        const int *slots, const long long *out_off, double *out, int n,
                        int nslots, long long pool_elems, long long out_elems, int *dbg);

}  // namespace lbm
