// Continuous-batching server of steady-state Couette solves (and the batched
// solve built on it).
//
// Requests (one single-column Couette instance each: lattice, height, Kn,
// wall speeds and temperatures, tolerance) queue on the host.  A worker
// thread owns the GPU side: a device memory pool of the configured budget,
// a slot table (SlotDesc / SlotStatus) in five classes by cluster size (a
// column runs on 1, 2, 4, 8 or 16 CTAs, by height) and the chunk kernel.  Every
// loop it
//   1. admits queued requests into idle slots of their class while the CTA
//      budget (max_slots) and the pool (first-fit allocator) have room for
//      them, initialises them;
//   2. moves running requests between cluster sizes when CTAs are spare or
//      queued requests lack them (the state stays in place);
//   3. runs one launch per class, the five concurrently (a CUDA graph: fork,
//      kernels, join, status read-back), so admitted work overlaps with
//      slots already running;
//   4. retires slots whose status left "running": reads their Eq. (3)
//      profiles back, frees their memory, records the latency.
// The f-arrays of a request stay resident on the device from admission to
// retirement.  A request too large for the whole budget is refused with
// LBM_EBUDGET at submission.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "batch_internal.h"
#include "lbm_internal.h"

namespace lbm {
namespace {

// work above which a request counts as long for the cluster choice: row-steps
// per thread on one CTA (~1 s at ~4 us per step and 256 rows)
constexpr double kLongRowSteps = 2.5e5;
constexpr long long kAlignElems = 64;        // 256-byte granularity (floats)
// A request's collision rounds to nearest while its change per check is above
// kPreciseFrom x tol (far from the steady state the state changes every step,
// so round-off does not freeze into a bias), then conserving increments with
// stochastic rounding until the steady state: the convergence test restarts at
// the switch and waits until the changes (the relaxation of whatever bias the
// first phase left included) are below tol.
constexpr double kPreciseFrom = 5.0;

struct Pending {
    uint64_t id;
    lbm_request req;
    double t_submit;
};

struct SlotInfo {
    bool busy = false;
    uint64_t id = 0;
    lbm_request req{};
    double t_submit = 0, t_admit = 0;
    long long off = 0, elems = 0;
};

struct Done {
    lbm_result meta;
    std::vector<double> fields;              // [4][Ny]: rho, u_x, u_y, T
};

long long request_elems(const lbm_request &r, int Q) {
    long long e = 2LL * Q * r.Ny + 2LL * r.Ny;
    return (e + kAlignElems - 1) / kAlignElems * kAlignElems;
}

int lattice_q(int kind) {
    return kind == LBM_LATTICE_D2Q17 ? 17 : kind == LBM_LATTICE_D2Q37 ? 37 : 25;
}

}  // namespace

struct ServerImpl {
    lbm_server_cfg cfg;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::chrono::steady_clock::time_point t0;
    // device side
    float *pool = nullptr;
    long long pool_elems = 0;
    SlotDesc *d_desc = nullptr;
    SlotStatus *d_status = nullptr;
    double *d_part = nullptr;                // residual partials per 32-row chunk
    // slot classes: slots [cls_base[c], cls_base[c] + cls_cap[c]) run on
    // clusters of kBatchClassCL[c] CTAs, each class launched on its own stream
    int cls_base[kBatchClasses] = {}, cls_cap[kBatchClasses] = {};
    int max_cl = 8;            // largest cluster the device schedules (8 or 16)
    cudaStream_t side[kBatchClasses] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kBatchClasses] = {};
    int *d_idx = nullptr;                    // slot lists for init / read-out
    long long *d_off = nullptr;
    int *d_dbg = nullptr;                    // kernels' record of a rejected descriptor
    int *h_dbg = nullptr;
    double *d_out = nullptr;                 // read-out staging
    long long out_elems = 0;
    // host mirrors (pinned)
    SlotDesc *h_desc = nullptr;
    SlotStatus *h_status = nullptr;
    int *h_idx = nullptr;
    long long *h_off = nullptr;
    double *h_out = nullptr;
    cudaGraphExec_t graph = nullptr;
    // host state
    std::map<long long, long long> free_list;        // offset -> length
    long long used_elems = 0;
    std::vector<SlotInfo> slots;
    LatticeHost lat[4];                      // D2Q17, D2Q25, D2Q25B, D2Q37
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::map<uint64_t, Done> done;
    std::deque<uint64_t> unpolled;
    std::vector<uint64_t> cancels;           // running requests to stop (worker applies)
    std::vector<double> latencies;
    uint64_t next_id = 1;
    int64_t submitted = 0, completed = 0;
    int running = 0;
    int used_ctas = 0;                       // CTAs of the running slots (<= max_slots)
    int64_t promoted = 0, demoted = 0;       // running requests moved to a larger / smaller cluster
    int64_t chunks = 0;
    double occupancy_sum = 0;
    double t_first_submit = -1, t_last_done = 0;
    std::atomic<bool> stop{false};
    std::atomic<int> worker_error{0};
    std::string worker_msg;
    std::thread worker;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    const LatticeHost &lattice(int kind) const {
        return lat[kind == 17 ? 0 : kind == 25 ? 1 : kind == 26 ? 2 : 3];
    }
    // chunks per launch of a slot on a cluster of cl CTAs: the configured
    // (autotuned) value of its class, else the built-in rule
    int sub_for(int cl) const {
        for (int c = 0; c < kBatchClasses; ++c)
            if (kBatchClassCL[c] == cl && cfg.class_sub[c] > 0) return cfg.class_sub[c];
        return batch_sub_chunks(cl);
    }

    // ---- pool allocator (first fit, coalescing) ---------------------------------
    long long alloc(long long n) {
        for (auto it = free_list.begin(); it != free_list.end(); ++it) {
            if (it->second >= n) {
                long long off = it->first, len = it->second;
                free_list.erase(it);
                if (len > n) free_list[off + n] = len - n;
                used_elems += n;
                return off;
            }
        }
        return -1;
    }
    void release(long long off, long long n) {
        used_elems -= n;
        auto it = free_list.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_list.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_list.erase(nx);
        }
        if (it != free_list.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_list.erase(it);
            }
        }
    }

    void fill_slot(int s, const Pending &pd, long long off, int cl) {
        const lbm_request &r = pd.req;
        const LatticeHost &L = lattice(r.lattice);
        lbm_params p;
        lbm_params_default(&p);
        p.Nx = 1;
        p.Ny = r.Ny;
        p.eq_order = r.eq_order;
        p.thermal = r.thermal;
        p.Kn = r.Kn;
        p.tau = r.tau;
        p.mu_exp = r.mu_exp;
        p.u_wall[0] = r.u_wall[0];
        p.u_wall[1] = r.u_wall[1];
        p.T_wall[0] = r.T_wall[0];
        p.T_wall[1] = r.T_wall[1];
        p.accom[0] = r.accom[0];
        p.accom[1] = r.accom[1];
        p.precision = LBM_FP32;
        SlotDesc &d = h_desc[s];
        std::memset(&d, 0, sizeof(d));
        d.Q = L.Q;
        d.Ny = r.Ny;
        d.cur = 0;
        d.cl = cl;
        d.sub = sub_for(cl);
        // Steps per chunk launch: cheaper slots run more steps, so that every
        // CTA of a launch takes about as long (cfg.chunk_steps x 333 cost
        // units); the cost model is the velocity count times the rows per
        // thread of one 256-thread CTA plus a latency floor.  It ignores the
        // cluster on purpose: chunk lengths and residual checks then fall on
        // the same steps however the column is split.
        const double cost = L.Q * std::ceil(r.Ny / 256.0) + 37.0;
        const double cost_ref = 37.0 * 8.0 + 37.0;
        d.chunk_steps = (int)std::min<double>(32.0 * cfg.chunk_steps,
                                              std::max<double>(cfg.chunk_steps,
                                                               std::round(cfg.chunk_steps * cost_ref / cost)));
        // residual every ~quarter of the slowest e-folding time of the start-up
        // (0.127 Ny r / Kn steps for the fundamental shear mode), in chunks
        const double efold = r.tau > 0 ? r.Ny * r.Ny / (9.8696 * r.tau * L.r * r.Ny)
                                       : 0.127 * r.Ny * L.r / r.Kn;
        d.check_every = std::max(1, (int)std::lround(efold / (4.0 * d.chunk_steps)));
        d.f_off = off;
        d.prev_off = off + 2LL * L.Q * r.Ny;
        d.tol = r.tol;
        d.max_steps = r.max_steps;
        d.u_ref = std::max(std::fabs(r.u_wall[0]), std::fabs(r.u_wall[1]));
        if (!(d.u_ref > 0)) d.u_ref = 1.0;
        d.mass0 = (double)r.Ny;                  // rho = 1 at admission
        d.init_u0 = d.init_u1 = d.init_T1 = d.init_T2 = 0.0;
        d.init_T0 = 1.0;
        if (r.init == LBM_INIT_NS) {
            // Sec. IV slip solution: slip length Kn (2 - a)/a per wall (a the
            // mean accommodation), viscous heating and jump of Eq. (14)
            const double a = 0.5 * (r.accom[0] + r.accom[1]);
            const double kn = r.tau > 0 ? r.tau * std::sqrt(M_PI / 2.0) : r.Kn;
            const double lam = a > 0 ? kn * (2.0 - a) / a : 1e30;
            const double U = 0.5 * (r.u_wall[1] - r.u_wall[0]);
            d.init_u0 = 0.5 * (r.u_wall[0] + r.u_wall[1]);
            d.init_u1 = lam < 1e29 ? 2.0 * U / (1.0 + 2.0 * lam) : 0.0;
            if (r.thermal) {
                const double Cp = 2.0, gam = 2.0, Pr = 1.0, den = std::pow(1.0 + 2.0 * lam, 2);
                const double Us = lam < 1e29 ? U * U : 0.0;
                d.init_T0 = r.T_wall[0] + 8.0 * gam / (gam + 1.0) * lam * Us / (2.0 * Cp * den);
                d.init_T1 = r.T_wall[1] - r.T_wall[0];
                d.init_T2 = 2.0 * Pr * Us / (Cp * den);
            }
        }
        d.precise_from = r.rounding == LBM_ROUND_AUTO ? kPreciseFrom * r.tol : -1.0;
        // incoming terms per wall (Sec. III: at layer l the velocities with
        // e.n < -l); the bottom list takes e_y < 0 at rows 0..|e_y|-1, the top
        // list e_y > 0 at rows Ny-1.. (distance from the wall)
        int nb = 0, nt = 0;
        for (int a = 0; a < L.Q; ++a) {
            for (int kk = 0; kk < -L.ey[a]; ++kk) { d.term_a[0][nb] = (signed char)a; d.term_row[0][nb] = (signed char)kk; ++nb; }
            for (int kk = 0; kk < L.ey[a]; ++kk) { d.term_a[1][nt] = (signed char)a; d.term_row[1][nt] = (signed char)kk; ++nt; }
        }
        if (nb != nt || nb >= 32) std::abort();  // lattices are symmetric, <= 26 terms
        d.nterm = nb;
        fill_consts(d.k, L, p, 1);
        // the wall warp sums the terms' deviations d = f - w and adds their
        // weights once (wterm); it then forms M_in g^w_a / D_w - w_a for the
        // outgoing velocities of its wall (e_y > 0 bottom, e_y < 0 top)
        int no[2] = {0, 0};
        for (int a = 0; a < L.Q; ++a) {
            for (int kk = 0; kk < -L.ey[a]; ++kk) d.wterm[0] += (double)d.k.w[a];
            for (int kk = 0; kk < L.ey[a]; ++kk) d.wterm[1] += (double)d.k.w[a];
            const int wl = L.ey[a] > 0 ? 0 : (L.ey[a] < 0 ? 1 : -1);
            if (wl < 0) continue;
            if (no[wl] >= kMaxOut || !(d.k.wcoef[wl][a] > 0.0)) std::abort();
            d.out_a[wl][no[wl]] = (signed char)a;
            d.out_c[wl][no[wl]] = d.k.wcoef[wl][a];
            d.out_w[wl][no[wl]] = (double)d.k.w[a];
            ++no[wl];
        }
        if (no[0] != no[1] || no[0] < 1) std::abort();
        d.nout = no[0];
        // the kernels reject anything else; the host must never produce it
        if (!(d.Ny >= 6 && d.Ny <= kMaxNy && d.f_off >= 0 &&
              d.f_off + 2LL * d.Q * d.Ny + 2LL * d.Ny <= pool_elems &&
              d.chunk_steps >= 1 && d.check_every >= 1))
            std::abort();
        SlotStatus &st = h_status[s];
        std::memset(&st, 0, sizeof(st));
        st.state = kSlotRunning;
        st.precise = r.rounding == LBM_ROUND_STOCHASTIC ? 1 : 0;
        st.best_res = 1e300;
        st.err_est = 1e300;
        SlotInfo &si = slots[s];
        si.busy = true;
        si.id = pd.id;
        si.req = r;
        si.t_submit = pd.t_submit;
        si.t_admit = now();
        si.off = off;
        si.elems = request_elems(r, L.Q);
    }

    cudaError_t upload_slot(int s) {
        cudaError_t e = cudaMemcpyAsync(d_desc + s, h_desc + s, sizeof(SlotDesc),
                                        cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_status + s, h_status + s, sizeof(SlotStatus),
                                cudaMemcpyHostToDevice, stream);
        return e;
    }

    int reject_desc() {
        char buf[256];
        std::snprintf(buf, sizeof buf,
                      "batch kernel rejected a slot descriptor: code %d slot %d Q %d Ny %d "
                      "f_off %d prev_off %d chunk %d check %d",
                      h_dbg[0], h_dbg[1], h_dbg[2], h_dbg[3], h_dbg[4], h_dbg[5], h_dbg[6], h_dbg[7]);
        worker_msg = buf;
        worker_error = LBM_EINVAL;
        return LBM_EINVAL;
    }

    int fail(const char *what, cudaError_t e) {
        worker_msg = std::string(what) + ": " + cudaGetErrorString(e);
        worker_error = LBM_ECUDA;
        return LBM_ECUDA;
    }

    // Whether a request may be split over a cluster, with its cluster size and
    // estimated work.  A split column moves fewer lattice updates per SM than
    // one CTA (a barrier per step across the cluster), so it is only worth its
    // latency gain for long requests: estimated row-steps per thread on one
    // CTA (14 e-folding times of the slowest shear mode, Ny / 256 rows per
    // thread) above kLongRowSteps.  Results do not depend on the split: every
    // cell update is the same arithmetic on the same values, chunk lengths and
    // checks ignore the cluster, and the residual is summed over 32-row chunks
    // in a fixed order.
    // Steps to steady state: 14 e-folding times of the slowest mode, the
    // viscous decay of the shear profile (0.127 Ny r / Kn steps) plus, at
    // large Kn, about one crossing of the channel at the thermal speed
    // (r Ny steps; measured: 1.1e5 steps for 4019 rows at Kn 0.98).
    double est_steps(const lbm_request &r) const {
        const LatticeHost &L = lattice(r.lattice);
        const double efold = r.tau > 0 ? r.Ny / (9.8696 * r.tau * L.r)
                                       : 0.127 * r.Ny * L.r / r.Kn + 1.2 * r.Ny * L.r;
        return 14.0 * efold;
    }
    bool long_split(const lbm_request &r, int &cl, double &work) const {
        cl = batch_cluster_size(r.Ny, cfg.cluster_rows, cfg.max_slots, max_cl);
        if (cl == 1) return false;
        work = est_steps(r) * std::ceil(r.Ny / 256.0);
        return work >= kLongRowSteps;
    }

    // a free slot of the class of clusters of cl CTAs, or -1
    int free_slot(int cl) const {
        int c = 0;
        while (c + 1 < kBatchClasses && kBatchClassCL[c] != cl) ++c;
        for (int s = cls_base[c]; s < cls_base[c] + cls_cap[c]; ++s)
            if (!slots[s].busy) return s;
        return -1;
    }

    // Chunk launches of every class, each on its own stream between a fork
    // and a join on `st`, so that the classes run concurrently (also inside
    // the captured graph).
    cudaError_t launch_chunks(cudaStream_t st) {
        cudaError_t e = cudaEventRecord(ev_fork, st);
        for (int c = 0; c < kBatchClasses && e == cudaSuccess; ++c) {
            e = cudaStreamWaitEvent(side[c], ev_fork, 0);
            if (e == cudaSuccess)
                e = (cudaError_t)launch_batch_chunk(side[c], d_desc, d_status, pool, d_part,
                                                    cls_base[c], cls_cap[c], kBatchClassCL[c],
                                                    pool_elems, d_dbg);
            if (e == cudaSuccess) e = cudaEventRecord(ev_join[c], side[c]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_join[c], 0);
        }
        return e;
    }

    // Elastic clusters.  A running request's slot can move to a class of
    // another cluster size between chunks: its state stays where it is in the
    // pool (a slot of any cluster size reads the same [Q][Ny] buffers), only
    // the descriptor and the status move, so the results are those of an
    // unmoved run, bit for bit.  When queued requests wait for CTAs
    // (short_ctas > 0), clusters shrink, least remaining work first, until
    // they fit; otherwise CTAs beyond one per queued request and a small
    // reserve for arrivals go to the long requests with the most remaining
    // work, which would otherwise keep the size they were admitted with (one
    // CTA on a full GPU) and set the latency tail.
    double remaining(int s) const {
        // remaining row-steps on one CTA; a request past its estimate keeps a
        // quarter of it
        const double est = est_steps(slots[s].req);
        return std::max(est - (double)h_status[s].steps, 0.25 * est) *
               std::ceil(slots[s].req.Ny / 256.0);
    }
    cudaError_t rebalance(long long spare, int short_ctas, const std::vector<int> &fresh) {
        struct Cand { double rem; int s; };
        struct Move { int from, to, cl; };
        std::vector<Cand> cand;
        std::vector<Move> moves;
        auto movable = [&](int s) {
            return slots[s].busy && h_status[s].state == kSlotRunning &&
                   std::find(fresh.begin(), fresh.end(), s) == fresh.end();
        };
        if (short_ctas > 0) {
            for (int s = 0; s < (int)slots.size(); ++s)
                if (movable(s) && h_desc[s].cl > 1) cand.push_back({remaining(s), s});
            std::sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) { return x.rem < y.rem; });
            int freed = 0;
            for (const Cand &c : cand) {
                if (freed >= short_ctas) break;
                const int cur = h_desc[c.s].cl, Ny = slots[c.s].req.Ny;
                int cl = cur / 2;
                while (cl > 1 && (freed + cur - cl < short_ctas || !batch_split_ok(Ny, cl))) cl /= 2;
                const int to = free_slot(cl);
                if (to < 0) continue;
                slots[to].busy = true;               // taken for this move
                freed += cur - cl;
                moves.push_back({c.s, to, cl});
            }
        } else {
            spare -= cfg.max_slots / 64;
            if (spare <= 0) return cudaSuccess;
            for (int s = 0; s < (int)slots.size(); ++s) {
                if (!movable(s)) continue;
                int cl;
                double work;
                if (!long_split(slots[s].req, cl, work) || cl <= h_desc[s].cl) continue;
                const double rem = remaining(s);
                if (rem >= kLongRowSteps) cand.push_back({rem, s});
            }
            std::sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) { return x.rem > y.rem; });
            for (const Cand &c : cand) {
                const int cur = h_desc[c.s].cl, Ny = slots[c.s].req.Ny;
                int cl = batch_cluster_size(Ny, cfg.cluster_rows, cfg.max_slots, max_cl);
                int to = -1;
                for (; cl > cur; cl /= 2) {
                    if (cl - cur > spare || !batch_split_ok(Ny, cl)) continue;
                    if ((to = free_slot(cl)) >= 0) break;
                }
                if (to < 0) continue;
                slots[to].busy = true;               // taken for this move
                spare -= cl - cur;
                moves.push_back({c.s, to, cl});
                if (spare <= 0) break;
            }
        }
        if (moves.empty()) return cudaSuccess;
        // the buffer index of a slot on the global-memory path lives on the device
        cudaError_t e = cudaSuccess;
        for (const Move &m : moves)
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&h_desc[m.from].cur, &d_desc[m.from].cur, sizeof(int),
                                    cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        std::unique_lock<std::mutex> lk(mu);         // the counters are read by stats
        for (const Move &m : moves) {
            const int from_cl = h_desc[m.from].cl;
            h_desc[m.to] = h_desc[m.from];
            h_desc[m.to].cl = m.cl;
            h_desc[m.to].sub = sub_for(m.cl);
            h_status[m.to] = h_status[m.from];
            slots[m.to] = slots[m.from];
            used_ctas += m.cl - from_cl;
            slots[m.from].busy = false;
            h_desc[m.from].Q = 0;
            h_status[m.from].state = kSlotIdle;
            if (m.cl > from_cl) ++promoted;
            else ++demoted;
            if (e == cudaSuccess) e = upload_slot(m.to);
            if (e == cudaSuccess) e = upload_slot(m.from);
        }
        return e;
    }

    // one loop of the worker; returns false when there is nothing to do
    int loop_once(bool &idle) {
        std::vector<int> admitted, stopped;
        long long spare = 0;
        int short_ctas = 0;                          // CTAs the budget lacked for queued requests
        {
            std::unique_lock<std::mutex> lk(mu);
            // running requests cancelled since the last chunk: marked stopped
            // on the host and, below, on the device, then retired as finished
            for (uint64_t id : cancels)
                for (int s = 0; s < (int)slots.size(); ++s)
                    if (slots[s].busy && slots[s].id == id && h_status[s].state == kSlotRunning) {
                        h_status[s].state = kSlotCancelled;
                        stopped.push_back(s);
                    }
            cancels.clear();
            // CTAs beyond one for every queued request go to the longest queued
            // requests (among the first 512), longest first, as clusters: the
            // GPU's idle CTAs shorten the requests that set the latency tail,
            // and none is taken from a request still waiting.
            std::map<uint64_t, int> split;
            long long extra = (long long)cfg.max_slots - used_ctas - (long long)queue.size();
            if (extra > 0) {
                std::vector<std::pair<double, std::pair<uint64_t, int>>> cand;
                int n = 0;
                for (auto q = queue.begin(); q != queue.end() && n < 512; ++q, ++n) {
                    int cl;
                    double work;
                    if (long_split(q->req, cl, work)) cand.push_back({work, {q->id, cl}});
                }
                std::sort(cand.begin(), cand.end(),
                          [](const auto &x, const auto &y) { return x.first > y.first; });
                for (const auto &c : cand)
                    if (extra >= c.second.second - 1) {
                        split[c.second.first] = c.second.second;
                        extra -= c.second.second - 1;
                    }
            }
            // Scan the queue in arrival order (at most 64 entries).  A request
            // is admitted when its class has a free slot and its cluster fits
            // the CTA budget (max_slots) minus what the oldest request that did
            // not fit needs (so that later requests cannot starve it); the
            // first request that finds no memory stops the scan.
            int reserve = 0, scanned = 0;
            for (auto it = queue.begin(); it != queue.end() && scanned < 64; ++scanned) {
                const auto sp = split.find(it->id);
                const int cl = sp == split.end() ? 1 : sp->second;
                const bool fits = used_ctas + cl + reserve <= cfg.max_slots;
                const int s = fits ? free_slot(cl) : -1;
                if (s < 0) {
                    if (!fits) short_ctas += 1;      // one CTA is all it needs
                    if (reserve == 0) reserve = cl;
                    ++it;
                    continue;
                }
                const long long n = request_elems(it->req, lattice_q(it->req.lattice));
                const long long off = alloc(n);
                if (off < 0) break;                  // wait for memory to free up
                fill_slot(s, *it, off, cl);
                admitted.push_back(s);
                it = queue.erase(it);
                ++running;
                used_ctas += cl;
            }
            idle = running == 0;
            spare = (long long)cfg.max_slots - used_ctas - (long long)queue.size();
        }
        cudaError_t e;
        for (int s : stopped)
            if ((e = cudaMemcpyAsync(d_status + s, h_status + s, sizeof(SlotStatus),
                                     cudaMemcpyHostToDevice, stream)))
                return fail("upload cancelled status", e);
        if (idle) return LBM_OK;
        if ((e = rebalance(spare, short_ctas, admitted))) return fail("rebalance", e);
        if (!admitted.empty()) {
            // only the admitted entries: running slots' buffer index lives on the device
            for (int s : admitted)
                if ((e = upload_slot(s))) return fail("upload slot", e);
            for (size_t i = 0; i < admitted.size(); ++i) h_idx[i] = admitted[i];
            if ((e = cudaMemcpyAsync(d_idx, h_idx, sizeof(int) * admitted.size(), cudaMemcpyHostToDevice, stream)))
                return fail("upload slot list", e);
            if ((e = (cudaError_t)launch_batch_init(stream, d_desc, pool, d_idx, (int)admitted.size(), 1.0f,
                                                     (int)slots.size(), pool_elems, d_dbg)))
                return fail("init kernel", e);
        }
        // chunk launch + status read-back
        nvtxRangePushA("lbm_server_chunk");
        if (graph) {
            if ((e = cudaGraphLaunch(graph, stream))) return fail("graph launch", e);
        } else {
            if ((e = launch_chunks(stream))) return fail("chunk kernel", e);
            if ((e = cudaMemcpyAsync(h_status, d_status, sizeof(SlotStatus) * slots.size(), cudaMemcpyDeviceToHost, stream)))
                return fail("status read-back", e);
            if ((e = cudaMemcpyAsync(h_dbg, d_dbg, sizeof(int) * 8, cudaMemcpyDeviceToHost, stream)))
                return fail("check read-back", e);
        }
        e = cudaStreamSynchronize(stream);
        nvtxRangePop();
        if (e) return fail("chunk", e);
        if (h_dbg[0]) return reject_desc();
        ++chunks;
        occupancy_sum += used_ctas;
        // retire finished slots
        std::vector<int> fin;
        for (int s = 0; s < (int)slots.size(); ++s)
            if (slots[s].busy && h_status[s].state != kSlotRunning) fin.push_back(s);
        size_t pos = 0;
        while (pos < fin.size()) {
            // read-out in batches that fit the staging buffer
            long long o = 0;
            size_t n = 0;
            while (pos + n < fin.size() && o + 4LL * slots[fin[pos + n]].req.Ny <= out_elems) {
                h_idx[n] = fin[pos + n];
                h_off[n] = o;
                o += 4LL * slots[fin[pos + n]].req.Ny;
                ++n;
            }
            if ((e = cudaMemcpyAsync(d_idx, h_idx, sizeof(int) * n, cudaMemcpyHostToDevice, stream)))
                return fail("upload read-out list", e);
            if ((e = cudaMemcpyAsync(d_off, h_off, sizeof(long long) * n, cudaMemcpyHostToDevice, stream)))
                return fail("upload read-out offsets", e);
            if ((e = (cudaError_t)launch_batch_macros(stream, d_desc, pool, d_idx, d_off, d_out, (int)n,
                                                       (int)slots.size(), pool_elems, out_elems, d_dbg)))
                return fail("read-out kernel", e);
            if ((e = cudaMemcpyAsync(h_out, d_out, sizeof(double) * o, cudaMemcpyDeviceToHost, stream)))
                return fail("read-out copy", e);
            if ((e = cudaMemcpyAsync(h_dbg, d_dbg, sizeof(int) * 8, cudaMemcpyDeviceToHost, stream)))
                return fail("check read-back", e);
            if ((e = cudaStreamSynchronize(stream))) return fail("read-out", e);
            if (h_dbg[0]) return reject_desc();
            const double t = now();
            std::unique_lock<std::mutex> lk(mu);
            for (size_t i = 0; i < n; ++i) {
                const int s = fin[pos + i];
                SlotInfo &si = slots[s];
                const SlotStatus &st = h_status[s];
                Done d;
                std::memset(&d.meta, 0, sizeof(d.meta));
                d.meta.id = si.id;
                d.meta.tag = si.req.tag;
                d.meta.status = st.state == kSlotConverged   ? LBM_OK
                                : st.state == kSlotNonFinite ? LBM_ENONFINITE
                                : st.state == kSlotCancelled ? LBM_ECANCELLED
                                                             : LBM_ENOTCONVERGED;
                d.meta.Ny = si.req.Ny;
                d.meta.steps = st.steps;
                d.meta.residual = st.res;
                d.meta.err_est = st.err_est;
                d.meta.mass = st.mass;
                d.meta.t_submit = si.t_submit;
                d.meta.t_admit = si.t_admit;
                d.meta.t_done = t;
                d.fields.assign(h_out + h_off[i], h_out + h_off[i] + 4LL * si.req.Ny);
                if (d.meta.status != LBM_ECANCELLED) latencies.push_back(t - si.t_submit);
                t_last_done = t;
                done.emplace(si.id, std::move(d));
                unpolled.push_back(si.id);
                release(si.off, si.elems);
                si.busy = false;
                used_ctas -= h_desc[s].cl;
                h_desc[s].Q = 0;
                h_status[s].state = kSlotIdle;
                --running;
                ++completed;
            }
            pos += n;
        }
        if (!fin.empty()) {
            // idle the retired slots on the device too
            for (int s : fin)
                if ((e = upload_slot(s))) return fail("upload slot", e);
            cv_done.notify_all();
        }
        return LBM_OK;
    }

    void run() {
        cudaSetDevice(device);
        while (!stop) {
            bool idle = false;
            if (loop_once(idle)) {
                std::unique_lock<std::mutex> lk(mu);
                cv_done.notify_all();
                return;
            }
            if (idle) {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait_for(lk, std::chrono::milliseconds(2),
                                 [&] { return stop || !queue.empty(); });
            }
        }
    }
};

}  // namespace lbm

struct lbm_server {
    lbm::ServerImpl s;
};

using namespace lbm;

extern "C" {

void lbm_server_cfg_default(lbm_server_cfg *c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->mem_budget_bytes = (size_t)40 << 30;
    c->max_slots = 256;
    c->chunk_steps = 100;
    c->precision = LBM_FP32;
    c->use_graph = 1;
    c->cluster_rows = 256;
}

static int check_request(const lbm_request *r) {
    if (!r) { set_error("NULL request"); return LBM_EINVAL; }
    if (r->lattice != LBM_LATTICE_D2Q17 && r->lattice != LBM_LATTICE_D2Q25 &&
        r->lattice != LBM_LATTICE_D2Q25B && r->lattice != LBM_LATTICE_D2Q37) {
        set_error("unknown lattice");
        return LBM_EINVAL;
    }
    if (r->Ny < 6 || r->Ny > kMaxNy) { set_error("Ny must be in [6, 8192]"); return LBM_EINVAL; }
    if (r->eq_order < 2 || r->eq_order > 4) { set_error("eq_order must be 2..4"); return LBM_EINVAL; }
    if (!(r->Kn > 0) && !(r->tau > 0)) { set_error("need Kn > 0 or tau > 0"); return LBM_EINVAL; }
    if (!std::isfinite(r->Kn) || !std::isfinite(r->tau) || !std::isfinite(r->mu_exp) ||
        !std::isfinite(r->u_wall[0]) || !std::isfinite(r->u_wall[1]) ||
        !std::isfinite(r->T_wall[0]) || !std::isfinite(r->T_wall[1]) || !(r->tol > 0) ||
        !std::isfinite(r->tol)) {
        set_error("non-finite or non-positive request parameter");
        return LBM_EINVAL;
    }
    if (r->thermal && (r->T_wall[0] <= 0 || r->T_wall[1] <= 0)) { set_error("T_wall <= 0"); return LBM_EINVAL; }
    if (r->max_steps < 1) { set_error("max_steps < 1"); return LBM_EINVAL; }
    if (!(r->accom[0] >= 0 && r->accom[0] <= 1 && r->accom[1] >= 0 && r->accom[1] <= 1)) {
        set_error("accom must lie in [0, 1]");
        return LBM_EINVAL;
    }
    if (r->rounding != LBM_ROUND_AUTO && r->rounding != LBM_ROUND_STOCHASTIC &&
        r->rounding != LBM_ROUND_NEAREST) {
        set_error("rounding must be LBM_ROUND_AUTO, _STOCHASTIC or _NEAREST");
        return LBM_EINVAL;
    }
    if (r->init != LBM_INIT_REST && r->init != LBM_INIT_NS) {
        set_error("init must be LBM_INIT_REST or LBM_INIT_NS");
        return LBM_EINVAL;
    }
    return LBM_OK;
}

int lbm_request_bytes(const lbm_request *r, size_t *bytes) {
    int rc = check_request(r);
    if (rc) return rc;
    if (!bytes) { set_error("NULL bytes"); return LBM_EINVAL; }
    *bytes = (size_t)request_elems(*r, lattice_q(r->lattice)) * sizeof(float);
    return LBM_OK;
}

int lbm_server_create(const lbm_server_cfg *cfg, void *stream, lbm_server **out) {
    try {
        if (!cfg || !out) { set_error("NULL argument"); return LBM_EINVAL; }
        *out = nullptr;
        bool subs_ok = true;
        for (int c = 0; c < kBatchClasses; ++c)
            subs_ok = subs_ok && cfg->class_sub[c] >= 0 && cfg->class_sub[c] <= kMaxSub;
        if (cfg->max_slots < 1 || cfg->max_slots > 4096 || cfg->chunk_steps < 1 ||
            cfg->mem_budget_bytes < 4096 || cfg->precision != LBM_FP32 || cfg->cluster_rows < 32 ||
            !subs_ok) {
            set_error("bad server configuration (slots 1..4096, chunk >= 1, FP32, cluster_rows >= 32, "
                      "class_sub 0..16)");
            return LBM_EINVAL;
        }
        lbm_server *h = new lbm_server;
        ServerImpl &S = h->s;
        S.cfg = *cfg;
        S.stream = (cudaStream_t)stream;
        S.t0 = std::chrono::steady_clock::now();
        cudaGetDevice(&S.device);
        const int kinds[4] = {17, 25, 26, 37};
        for (int i = 0; i < 4; ++i)
            if (lattice_build(kinds[i], S.lat[i])) { delete h; set_error("lattice build"); return LBM_EINVAL; }
        // slot classes: max_slots / CL slots of each cluster size, so that any
        // class alone can fill the CTA budget; none for clusters larger than
        // the budget or than the device schedules
        if (int rc = preload_batch_kernels()) {
            delete h;
            set_error(std::string("batch kernels: ") + cudaGetErrorString((cudaError_t)rc));
            return LBM_ECUDA;
        }
        S.max_cl = batch_max_cluster();
        int ns = 0;
        for (int c = 0; c < kBatchClasses; ++c) {
            const int cl = kBatchClassCL[c];
            S.cls_cap[c] = cl > S.max_cl || cl > cfg->max_slots ? 0 : cfg->max_slots / cl;
            S.cls_base[c] = ns;
            ns += S.cls_cap[c];
        }
        S.slots.resize(ns);
        S.pool_elems = (long long)(cfg->mem_budget_bytes / sizeof(float)) / kAlignElems * kAlignElems;
        S.out_elems = 4LL * kMaxNy * std::min(ns, 64);
        cudaError_t e = cudaSuccess;
        auto ck = [&](cudaError_t r) { if (r != cudaSuccess && e == cudaSuccess) e = r; };
        ck(cudaMallocAsync((void **)&S.pool, (size_t)S.pool_elems * sizeof(float), S.stream));
        ck(cudaMallocAsync((void **)&S.d_desc, sizeof(SlotDesc) * ns, S.stream));
        ck(cudaMallocAsync((void **)&S.d_status, sizeof(SlotStatus) * ns, S.stream));
        ck(cudaMallocAsync((void **)&S.d_part, sizeof(double) * 6 * kMaxResidualChunks * ns, S.stream));
        ck(cudaEventCreateWithFlags(&S.ev_fork, cudaEventDisableTiming));
        for (int c = 0; c < kBatchClasses; ++c) {
            ck(cudaStreamCreateWithFlags(&S.side[c], cudaStreamNonBlocking));
            ck(cudaEventCreateWithFlags(&S.ev_join[c], cudaEventDisableTiming));
        }
        ck(cudaMallocAsync((void **)&S.d_idx, sizeof(int) * ns, S.stream));
        ck(cudaMallocAsync((void **)&S.d_off, sizeof(long long) * ns, S.stream));
        ck(cudaMallocAsync((void **)&S.d_out, sizeof(double) * S.out_elems, S.stream));
        ck(cudaMallocAsync((void **)&S.d_dbg, sizeof(int) * 8, S.stream));
        ck(cudaMallocHost((void **)&S.h_dbg, sizeof(int) * 8));
        ck(cudaMallocHost((void **)&S.h_desc, sizeof(SlotDesc) * ns));
        ck(cudaMallocHost((void **)&S.h_status, sizeof(SlotStatus) * ns));
        ck(cudaMallocHost((void **)&S.h_idx, sizeof(int) * ns));
        ck(cudaMallocHost((void **)&S.h_off, sizeof(long long) * ns));
        ck(cudaMallocHost((void **)&S.h_out, sizeof(double) * S.out_elems));
        if (e == cudaSuccess) {
            std::memset(S.h_desc, 0, sizeof(SlotDesc) * ns);
            std::memset(S.h_status, 0, sizeof(SlotStatus) * ns);
            ck(cudaMemcpyAsync(S.d_desc, S.h_desc, sizeof(SlotDesc) * ns, cudaMemcpyHostToDevice, S.stream));
            ck(cudaMemcpyAsync(S.d_status, S.h_status, sizeof(SlotStatus) * ns, cudaMemcpyHostToDevice, S.stream));
            ck(cudaMemsetAsync(S.d_dbg, 0, sizeof(int) * 8, S.stream));
            std::memset(S.h_dbg, 0, sizeof(int) * 8);
            ck(cudaStreamSynchronize(S.stream));
        }
        if (e == cudaSuccess && cfg->use_graph) {
            // capture: chunk kernels of every class, then the status read-back
            cudaStream_t cs;
            ck(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g;
            ck(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            ck(S.launch_chunks(cs));
            ck(cudaMemcpyAsync(S.h_status, S.d_status, sizeof(SlotStatus) * ns, cudaMemcpyDeviceToHost, cs));
            ck(cudaMemcpyAsync(S.h_dbg, S.d_dbg, sizeof(int) * 8, cudaMemcpyDeviceToHost, cs));
            ck(cudaStreamEndCapture(cs, &g));
            if (e == cudaSuccess) ck(cudaGraphInstantiate(&S.graph, g, 0));
            cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
        }
        if (e != cudaSuccess) {
            const bool oom = e == cudaErrorMemoryAllocation;
            set_error(std::string("server set-up: ") + cudaGetErrorString(e));
            lbm_server_destroy(h);
            return oom ? LBM_ENOMEM : LBM_ECUDA;
        }
        S.free_list[0] = S.pool_elems;
        S.worker = std::thread([&S] { S.run(); });
        *out = h;
        return LBM_OK;
    } catch (...) {
        set_error("server creation failed");
        return LBM_ENOMEM;
    }
}

int lbm_server_submit(lbm_server *h, const lbm_request *r, uint64_t *id) {
    if (!h) { set_error("NULL server"); return LBM_EINVAL; }
    int rc = check_request(r);
    if (rc) return rc;
    ServerImpl &S = h->s;
    if (S.worker_error) { set_error(S.worker_msg); return S.worker_error; }
    const long long n = request_elems(*r, lattice_q(r->lattice));
    if (n > S.pool_elems) { set_error("request exceeds the whole memory budget"); return LBM_EBUDGET; }
    {
        std::unique_lock<std::mutex> lk(S.mu);
        Pending p{S.next_id++, *r, S.now()};
        if (S.t_first_submit < 0) S.t_first_submit = p.t_submit;
        if (id) *id = p.id;
        S.queue.push_back(p);
        ++S.submitted;
    }
    S.cv_work.notify_one();
    return LBM_OK;
}

int lbm_server_poll(lbm_server *h, lbm_result *out, int32_t max, int32_t *n) {
    if (!h || !n || (max > 0 && !out)) { set_error("bad argument"); return LBM_EINVAL; }
    ServerImpl &S = h->s;
    std::unique_lock<std::mutex> lk(S.mu);
    int k = 0;
    while (k < max && !S.unpolled.empty()) {
        out[k++] = S.done.at(S.unpolled.front()).meta;
        S.unpolled.pop_front();
    }
    *n = k;
    if (S.worker_error) { set_error(S.worker_msg); return S.worker_error; }
    return LBM_OK;
}

int lbm_server_cancel(lbm_server *h, uint64_t id) {
    if (!h) { set_error("NULL server"); return LBM_EINVAL; }
    ServerImpl &S = h->s;
    {
        std::unique_lock<std::mutex> lk(S.mu);
        for (auto it = S.queue.begin(); it != S.queue.end(); ++it)
            if (it->id == id) {
                // never admitted: completes at once, with zero fields
                Done d;
                std::memset(&d.meta, 0, sizeof(d.meta));
                d.meta.id = id;
                d.meta.tag = it->req.tag;
                d.meta.status = LBM_ECANCELLED;
                d.meta.Ny = it->req.Ny;
                d.meta.t_submit = it->t_submit;
                d.meta.t_admit = d.meta.t_done = S.now();
                d.fields.assign(4 * (size_t)it->req.Ny, 0.0);
                S.done.emplace(id, std::move(d));
                S.unpolled.push_back(id);
                S.queue.erase(it);
                ++S.completed;
                S.cv_done.notify_all();
                return LBM_OK;
            }
        bool running = false;
        for (const SlotInfo &si : S.slots) running = running || (si.busy && si.id == id);
        if (!running) { set_error("no queued or running request with this id"); return LBM_EINVAL; }
        S.cancels.push_back(id);
    }
    S.cv_work.notify_one();
    return LBM_OK;
}

int lbm_server_fetch(lbm_server *h, uint64_t id, double *rho, double *ux, double *uy, double *T) {
    if (!h) { set_error("NULL server"); return LBM_EINVAL; }
    ServerImpl &S = h->s;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.done.find(id);
    if (it == S.done.end()) { set_error("no finished result with this id"); return LBM_EINVAL; }
    const int Ny = it->second.meta.Ny;
    double *dst[4] = {rho, ux, uy, T};
    for (int i = 0; i < 4; ++i)
        if (dst[i]) std::memcpy(dst[i], it->second.fields.data() + (size_t)i * Ny, sizeof(double) * Ny);
    S.done.erase(it);
    return LBM_OK;
}

int lbm_server_drain(lbm_server *h, double timeout_s) {
    if (!h) { set_error("NULL server"); return LBM_EINVAL; }
    ServerImpl &S = h->s;
    std::unique_lock<std::mutex> lk(S.mu);
    const bool ok = S.cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
        return S.completed == S.submitted || S.worker_error != 0;
    });
    if (S.worker_error) { set_error(S.worker_msg); return S.worker_error; }
    if (!ok) { set_error("drain timed out"); return LBM_ETIMEOUT; }
    return LBM_OK;
}

int lbm_server_stats(lbm_server *h, lbm_server_metrics *st) {
    if (!h || !st) { set_error("NULL argument"); return LBM_EINVAL; }
    ServerImpl &S = h->s;
    std::unique_lock<std::mutex> lk(S.mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = S.submitted;
    st->completed = S.completed;
    st->running = S.running;
    st->queued = (int64_t)S.queue.size();
    st->chunks = S.chunks;
    st->pool_bytes = (size_t)S.pool_elems * sizeof(float);
    st->pool_used_bytes = (size_t)S.used_elems * sizeof(float);
    st->mean_occupancy = S.chunks ? S.occupancy_sum / (S.chunks * (double)S.cfg.max_slots) : 0.0;
    st->promoted = S.promoted;
    st->demoted = S.demoted;
    if (!S.latencies.empty()) {
        std::vector<double> l = S.latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            const double pos = q * (l.size() - 1);
            const size_t i = (size_t)pos;
            const double fr = pos - i;
            return i + 1 < l.size() ? l[i] * (1 - fr) + l[i + 1] * fr : l[i];
        };
        st->p50_latency_s = pct(0.50);
        st->p99_latency_s = pct(0.99);
        double sum = 0;
        for (double v : l) sum += v;
        st->mean_latency_s = sum / l.size();
        const double span = S.t_last_done - S.t_first_submit;
        st->solves_per_s = span > 0 ? S.completed / span : 0.0;
    }
    return LBM_OK;
}

int lbm_server_destroy(lbm_server *h) {
    if (!h) return LBM_OK;
    ServerImpl &S = h->s;
    S.stop = true;
    S.cv_work.notify_all();
    if (S.worker.joinable()) S.worker.join();
    if (S.graph) cudaGraphExecDestroy(S.graph);
    cudaStreamSynchronize(S.stream);
    if (S.pool) cudaFreeAsync(S.pool, S.stream);
    if (S.d_desc) cudaFreeAsync(S.d_desc, S.stream);
    if (S.d_status) cudaFreeAsync(S.d_status, S.stream);
    if (S.d_idx) cudaFreeAsync(S.d_idx, S.stream);
    if (S.d_off) cudaFreeAsync(S.d_off, S.stream);
    if (S.d_out) cudaFreeAsync(S.d_out, S.stream);
    if (S.d_dbg) cudaFreeAsync(S.d_dbg, S.stream);
    if (S.d_part) cudaFreeAsync(S.d_part, S.stream);
    cudaStreamSynchronize(S.stream);
    for (int c = 0; c < kBatchClasses; ++c) {
        if (S.side[c]) cudaStreamDestroy(S.side[c]);
        if (S.ev_join[c]) cudaEventDestroy(S.ev_join[c]);
    }
    if (S.ev_fork) cudaEventDestroy(S.ev_fork);
    if (S.h_desc) cudaFreeHost(S.h_desc);
    if (S.h_status) cudaFreeHost(S.h_status);
    if (S.h_idx) cudaFreeHost(S.h_idx);
    if (S.h_off) cudaFreeHost(S.h_off);
    if (S.h_out) cudaFreeHost(S.h_out);
    if (S.h_dbg) cudaFreeHost(S.h_dbg);
    delete h;
    return LBM_OK;
}

int lbm_batch_solve(const lbm_server_cfg *cfg, void *stream, const lbm_request *reqs, int32_t n,
                    lbm_result *out, double timeout_s) {
    if (!cfg || (n > 0 && (!reqs || !out)) || n < 0) { set_error("bad argument"); return LBM_EINVAL; }
    lbm_server *h = nullptr;
    int rc = lbm_server_create(cfg, stream, &h);
    if (rc) return rc;
    std::vector<uint64_t> ids(n);
    for (int i = 0; i < n && !rc; ++i) rc = lbm_server_submit(h, &reqs[i], &ids[i]);
    if (!rc) rc = lbm_server_drain(h, timeout_s);
    if (!rc) {
        std::map<uint64_t, int> pos;
        for (int i = 0; i < n; ++i) pos[ids[i]] = i;
        std::vector<lbm_result> tmp(n > 0 ? n : 1);
        int32_t got = 0;
        rc = lbm_server_poll(h, tmp.data(), n, &got);
        for (int i = 0; i < got; ++i) out[pos[tmp[i].id]] = tmp[i];
    }
    lbm_server_destroy(h);
    return rc;
}

}  // extern "C"

namespace {

// Wall seconds from the first submit to the drain of n identical fixed-step
// requests (lattice kind, Ny rows, Kn, walls -+0.1, tol 0: never converged)
// on a server with cfg; *cell_steps gets the lattice updates they ran.
int time_fixed_steps(const lbm_server_cfg &cfg, void *stream, int kind, int Ny, double Kn, int n,
                     int64_t steps, double *seconds, double *cell_steps) {
    lbm_server *h = nullptr;
    if (int rc = lbm_server_create(&cfg, stream, &h)) return rc;
    lbm_request r;
    std::memset(&r, 0, sizeof(r));
    r.lattice = kind;
    r.Ny = Ny;
    r.thermal = kind == LBM_LATTICE_D2Q37 ? 1 : 0;
    r.eq_order = r.thermal ? 4 : 2;
    r.Kn = Kn;
    r.mu_exp = 1.0;
    r.u_wall[0] = -0.1;
    r.u_wall[1] = 0.1;
    r.T_wall[0] = r.T_wall[1] = 1.0;
    r.tol = 1e-300;
    r.max_steps = steps;
    r.accom[0] = r.accom[1] = 1.0;
    const auto t0 = std::chrono::steady_clock::now();
    int rc = LBM_OK;
    for (int i = 0; i < n && !rc; ++i) rc = lbm_server_submit(h, &r, nullptr);
    if (!rc) rc = lbm_server_drain(h, 600.0);
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    std::vector<lbm_result> res(n > 0 ? n : 1);
    int32_t got = 0;
    if (!rc) rc = lbm_server_poll(h, res.data(), n, &got);
    double cs = 0;
    for (int i = 0; i < got; ++i) cs += (double)res[i].steps * Ny;
    *cell_steps = cs;
    lbm_server_destroy(h);
    return rc;
}

double median(std::vector<double> v) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const size_t m = v.size() / 2;
    return v.size() % 2 ? v[m] : 0.5 * (v[m - 1] + v[m]);
}

}  // namespace

extern "C" int lbm_server_autotune(lbm_server_cfg *cfg, void *stream, lbm_server_tuning *report) {
    if (!cfg) { set_error("NULL configuration"); return LBM_EINVAL; }
    const auto t_start = std::chrono::steady_clock::now();
    lbm_server_tuning rep;
    std::memset(&rep, 0, sizeof(rep));
    const int kinds[3] = {LBM_LATTICE_D2Q17, LBM_LATTICE_D2Q25, LBM_LATTICE_D2Q37};
    const int heights[3] = {256, 1024, 4096};
    if (int rc = preload_batch_kernels()) {
        set_error(std::string("batch kernels: ") + cudaGetErrorString((cudaError_t)rc));
        return LBM_ECUDA;
    }
    const int max_cl = batch_max_cluster();
    // ---- lone columns on every usable cluster size --------------------------
    // a lone long request (small Kn) gets the largest usable cluster within the
    // CTA budget: the budget picks the cluster size; long chunks keep the
    // host's per-launch work out of the step time
    auto lone_us = [&](int kind, int Ny, int cl, double *us) -> int {
        *us = 0.0;
        if (cl > max_cl || batch_cluster_size(Ny, 32, cl, max_cl) != cl) return LBM_OK;
        lbm_server_cfg lc = *cfg;
        lc.max_slots = cl;
        lc.cluster_rows = 32;
        lc.chunk_steps = 1000;
        lc.mem_budget_bytes = (size_t)64 << 20;
        for (int k = 0; k < kBatchClasses; ++k) lc.class_sub[k] = 0;
        double sec = 0, cells = 0;
        if (int rc = time_fixed_steps(lc, stream, kind, Ny, 1e-3, 1, 4000, &sec, &cells)) return rc;
        *us = cells > 0 ? sec / (cells / Ny) * 1e6 : 0.0;
        return LBM_OK;
    };
    std::vector<double> rows_best;
    for (int li = 0; li < 3; ++li) {
        for (int hi = 0; hi < 3; ++hi) {
            const int Ny = heights[hi];
            rep.ny[hi] = Ny;
            double tbest = 1e300;
            for (int c = 0; c < kBatchClasses; ++c) {
                if (int rc = lone_us(kinds[li], Ny, kBatchClassCL[c], &rep.lone_us[li][hi][c])) return rc;
                const double us = rep.lone_us[li][hi][c];
                if (us > 0 && us < tbest) tbest = us;
            }
            // the smallest cluster within 15 % of the fastest: its rows per CTA
            for (int c = 0; c < kBatchClasses; ++c) {
                const double us = rep.lone_us[li][hi][c];
                if (us > 0 && us <= 1.15 * tbest) {
                    rows_best.push_back((double)batch_rows_per_cta(Ny, kBatchClassCL[c]));
                    break;
                }
            }
        }
    }
    // chunks per launch of class c: the factor by which its cluster shortens
    // a step, at the height the class serves (CL x 256 rows, the tallest a
    // CL-CTA cluster takes at 256 rows per CTA): D2Q37 there on one CTA over
    // on the cluster
    double ratio[kBatchClasses] = {1, 0, 0, 0, 0};
    for (int c = 1; c < kBatchClasses; ++c) {
        const int cl = kBatchClassCL[c], Ny = std::min(kMaxNy, 256 * cl);
        double t1 = 0, tc = 0;
        if (int rc = lone_us(LBM_LATTICE_D2Q37, Ny, 1, &t1)) return rc;
        if (int rc = lone_us(LBM_LATTICE_D2Q37, Ny, cl, &tc)) return rc;
        ratio[c] = (t1 > 0 && tc > 0) ? t1 / tc : 0.0;
    }
    // ---- chunk length on a full GPU of one-CTA columns ------------------------
    // (D2Q37, 256 rows: the heaviest one-CTA column; best of two runs each)
    const int chunks[5] = {25, 50, 100, 200, 400};
    double best = 0;
    for (int i = 0; i < 5; ++i) {
        lbm_server_cfg lc = *cfg;
        lc.cluster_rows = kMaxNy;
        lc.chunk_steps = chunks[i];
        lc.mem_budget_bytes = std::min<size_t>(cfg->mem_budget_bytes, (size_t)1 << 30);
        rep.chunk_try[i] = chunks[i];
        for (int rep_i = 0; rep_i < 2; ++rep_i) {
            double sec = 0, cells = 0;
            if (int rc = time_fixed_steps(lc, stream, LBM_LATTICE_D2Q37, 256, 0.1, cfg->max_slots,
                                          4000, &sec, &cells))
                return rc;
            rep.chunk_glups[i] = std::max(rep.chunk_glups[i], sec > 0 ? cells / sec / 1e9 : 0.0);
        }
        best = std::max(best, rep.chunk_glups[i]);
    }
    // the longest chunk within 5 % of the best rate: fewer launches (each
    // costs the host a round trip) at about the same rate
    int chunk = chunks[0];
    for (int i = 0; i < 5; ++i)
        if (rep.chunk_glups[i] >= 0.95 * best) chunk = chunks[i];
    // ---- the choices ------------------------------------------------------------
    cfg->chunk_steps = chunk;
    cfg->class_sub[0] = 1;
    for (int c = 1; c < kBatchClasses; ++c)
        cfg->class_sub[c] = ratio[c] > 0 ? std::max(1, std::min(kMaxSub, (int)std::lround(ratio[c]))) : 0;
    if (!rows_best.empty()) {
        int rows = (int)median(rows_best);
        rows = std::max(32, std::min(1024, (rows + kResidualChunk - 1) / kResidualChunk * kResidualChunk));
        cfg->cluster_rows = rows;
    }
    rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (report) *report = rep;
    return LBM_OK;
}
