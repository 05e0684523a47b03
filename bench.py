"""Benchmark of the fused pull-stream + BGK + diffuse-wall step on one GB300.

Workload: thermal Couette, D2Q37 lattice, 4th-order Hermite equilibrium,
Nx = 4096 periodic columns x Ny = 2048 rows, walls -+0.3, T_w = 1, Kn = 0.05,
rho = 1 + uniform noise +-1e-3 (SplitMix64 seed 7), FP32 storage and
arithmetic.  A step is one full lattice update of all cells (one launch of the
step kernel); the 2.5 GB state is far larger than L2, so no flush is needed.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(the reference arm of this project) on a bounded sample of the same workload.
Under torchrun every rank runs its own independent replica of the workload
(the path has no data exchange between domains); the slowest rank's time
counts and `value` sums the cells of all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(lattice="D2Q37", Nx=4096, Ny=2048, eq_order=4, thermal=True, Kn=0.05,
                u_wall=(-0.3, 0.3), T_wall=(1.0, 1.0), noise_amp=1e-3, seed=7)
BYTES_PER_LU = {"fp32": 8 * 37, "fp64": 16 * 37, "bf16dev": 4 * 37 + 8, "bf16shift": 4 * 37}
DTYPE = {"fp32": "f32", "fp64": "f64", "bf16dev": "bf16-storage/f32", "bf16shift": "bf16-storage/f32"}


def reduce_max(value: float, dist=None, device="cpu") -> float:
    """Largest value over the ranks (the slowest rank's time); identity alone."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, cells_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job MLUPS: every rank advances its own replica by `steps`."""
    return world * cells_per_rank * steps / seconds / 1e6


def workload_name(prec: str, Nx: int, Ny: int) -> str:
    return f"D2Q37 4th-order thermal Couette {Nx}x{Ny} {prec.upper()}"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """SM clocks and throttle reasons sampled DURING the timed region.

    A thread polls NVML (libnvidia-ml, read-only queries) about every
    millisecond, so that a timed region of a few milliseconds still gets
    samples; only samples taken between mark_start() and mark_stop() count.
    Without NVML it falls back to nvidia-smi every 100 ms."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []           # (t, sm_mhz, reasons bitmask, power_w)
        self.t0 = self.t1 = None
        self.source = None
        self._stop = False
        self._thread = None
        self._smi = None

    def _nvml(self):
        import ctypes as C
        import torch
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit")
        pr = torch.cuda.get_device_properties(self.gpu)
        bus = f"{pr.pci_domain_id:x}:{pr.pci_bus_id:x}:{pr.pci_device_id:x}.0".encode()
        h = C.c_void_p()
        if lib.nvmlDeviceGetHandleByPciBusId_v2(C.c_char_p(bus), C.byref(h)) != 0:
            raise RuntimeError("nvml handle")
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        clk, mx, rs, pw = C.c_uint(), C.c_uint(), C.c_ulonglong(), C.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx)) != 0:
            raise RuntimeError("nvml max clock")
        self.max_mhz = float(mx.value)

        def sample():
            ok = lib.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0      # NVML_CLOCK_SM
            ok = ok and get_reasons(h, C.byref(rs)) == 0
            p = pw.value / 1000.0 if lib.nvmlDeviceGetPowerUsage(h, C.byref(pw)) == 0 else None
            return (float(clk.value), int(rs.value), p) if ok else None
        return sample

    def start(self):
        import threading
        try:
            sample = self._nvml()
            self.source = "nvml"
        except Exception:
            sample = None
        if sample is None:
            return self._start_smi()

        def loop():
            while not self._stop:
                r = sample()
                if r is not None:
                    self.samples.append((time.perf_counter(), *r))
                time.sleep(0.001)
        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()
        time.sleep(0.01)

    def _start_smi(self):
        self.source = "nvidia-smi"
        fields = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                  "clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self._smi = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={fields}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._smi = None
            return
        import threading

        def reader():
            bits = (0x8, 0x40, 0x20, 0x4)
            for line in self._smi.stdout:
                parts = [x.strip() for x in line.split(",")]
                try:
                    r = sum(b for b, v in zip(bits, parts[3:7]) if v.lower() == "active")
                    self.max_mhz = float(parts[1])
                    self.samples.append((time.perf_counter(), float(parts[0]), r,
                                         float(parts[2])))
                except (ValueError, IndexError):
                    continue
        self._thread = threading.Thread(target=reader, daemon=True)
        self._thread.start()

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_stop(self):
        self.t1 = time.perf_counter()

    def stop(self):
        self._stop = True
        if self._smi is not None:
            self._smi.terminate()
        if self._thread is not None:
            self._thread.join(timeout=5)
        if self.source is None or (self._smi is None and self.source != "nvml"):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"],
                    "samples": 0}
        inside = [x for x in self.samples
                  if self.t0 is not None and self.t1 is not None and self.t0 <= x[0] <= self.t1]
        bits = 0
        for x in inside:
            bits |= x[2]
        pw = [x[3] for x in inside if x[3] is not None]
        return {"sm_mhz": statistics.median(x[1] for x in inside) if inside else None,
                "sm_max_mhz": getattr(self, "max_mhz", None),
                "reasons": sorted(n for b, n in self.REASONS.items() if bits & b),
                "samples": len(inside), "source": self.source,
                "power_w_max": max(pw) if pw else None}


def cpu_baseline(prec: str, budget_s: float = 12.0):
    """The FP64 oracle (as it stands) on this host's cores, on a bounded sample
    of the workload: the full 4096-column width with 128 rows (both walls),
    for as many steps as fit in about budget_s seconds (at least one)."""
    import numpy as np

    import inputs
    from oracle import oracle as orc
    Nx, Ny = WORKLOAD["Nx"], 128
    p = orc.Problem(lattice="D2Q37", Nx=Nx, Ny=Ny, eq_order=4, thermal=True, Kn=0.05,
                    u_wall=(-0.3, 0.3), T_wall=(1.0, 1.0))
    f = orc.init_fields(p, inputs.rho_field(Nx, Ny, 1e-3, seed=7))
    t0 = time.perf_counter()
    orc.run(p, f, 1)
    t1 = time.perf_counter() - t0
    steps = max(1, min(50, int(budget_s / max(t1, 1e-6)) - 1))
    t0 = time.perf_counter()
    orc.run(p, f, steps)
    dt = time.perf_counter() - t0
    return {"value": Nx * Ny * steps / dt / 1e6, "unit": "MLUPS", "cores": orc.num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle, {Nx}x{Ny} rows of the same Couette setup, {steps} steps "
                      f"after 1 untimed step ({dt:.1f} s)"}


def _request(lbm, inst, tol):
    """A steady-state solve of the instance, started from the Navier-Stokes
    slip solution of the Couette problem (the same steady state as from rest,
    in fewer steps)."""
    return lbm.make_request(inst.lattice, inst.Ny, inst.Kn, inst.U_w, inst.T_w, tol=tol,
                            max_steps=20_000_000, init=lbm.LBM_INIT_NS)


Q_OF = {"D2Q17": 17, "D2Q25": 25, "D2Q25b": 25, "D2Q37": 37}
# Stopping target of the batched and serving solves: the extrapolated L-inf
# distance of u_x / U_w (and T) to the steady state; chosen below the 1e-5
# accuracy the workloads ask for, which the oracle legs measure.
SOLVE_TOL = 5e-6


def resident_ctas() -> int:
    """CTA budget of the server: every batch CTA resident at once (two 256-thread
    CTAs per SM)."""
    import torch
    return 2 * torch.cuda.get_device_properties(0).multi_processor_count


_TUNED = {}


def tuned_server_cfg(lbm):
    """Server configuration of the batched and serving legs: 40 GB budget,
    every CTA resident, chunk length, cluster rows and chunks per launch from
    the library's batched-path autotuner (run once per process, before any
    timed region)."""
    if "cfg" not in _TUNED:
        cfg = lbm.lbm_server_cfg_default()
        cfg.mem_budget_bytes = 40 << 30
        cfg.max_slots = resident_ctas()
        rep = lbm.lbm_server_autotune(cfg)
        _TUNED["cfg"] = cfg
        _TUNED["report"] = {"chunk_steps": cfg.chunk_steps, "cluster_rows": cfg.cluster_rows,
                            "class_sub": list(cfg.class_sub), "seconds": rep["seconds"],
                            "chunk_glups": dict(zip(rep["chunk_try"], rep["chunk_glups"])),
                            "lone_us_per_step": {
                                lat: {ny: [round(v, 3) for v in rep["lone_us"][li][hi]]
                                      for hi, ny in enumerate(rep["ny"])}
                                for li, lat in enumerate(("D2Q17", "D2Q25", "D2Q37"))}}
    return type(_TUNED["cfg"]).from_buffer_copy(_TUNED["cfg"]), _TUNED["report"]


def _oracle_problem(orc, it):
    return orc.Problem(lattice=it.lattice, Nx=1, Ny=it.Ny, eq_order=it.eq_order,
                       thermal=it.thermal, Kn=it.Kn, u_wall=(-it.U_w, it.U_w),
                       T_wall=(it.T_w, it.T_w))


def oracle_leg(insts, results, fields, budget_s=10.0, limit=40, max_cell_steps=3e7):
    """CPU baseline and accuracy of a batched / serving run: the FP64 oracle (as
    it stands) on the host's cores, on the cheapest instances of `insts` (at
    most `limit`, est. <= max_cell_steps each), in order of cost until about
    budget_s seconds of timed work: timed over the GPU's step count (the
    baseline rate), then run on, untimed, to its own steady state (residual
    1e-12), against which the GPU's steady profile is measured (L-inf of
    u_x / U_w, and of T when thermal)."""
    import numpy as np

    from oracle import lattice as olat
    from oracle import oracle as orc

    def est(it):
        return 14 * (0.127 * it.Ny * olat.get(it.lattice).r / it.Kn) * it.Ny
    cand = sorted((k for k in range(len(insts)) if est(insts[k]) <= max_cell_steps),
                  key=lambda k: est(insts[k]))[:limit]
    t_sum, cells, done, err_u, err_T = 0.0, 0, [], [], []
    for k in cand:
        if t_sum > budget_s:
            break
        it, r = insts[k], results[k]
        p = _oracle_problem(orc, it)
        f = orc.init_fields(p, np.ones((it.Ny, 1)))
        t1 = time.perf_counter()
        orc.run(p, f, r.steps)
        t_sum += time.perf_counter() - t1
        cells += r.steps * it.Ny
        done.append(k)
        ok, _, _ = orc.run_to_residual(p, f, 1e-12, 20_000_000, 200)
        _, ux, _, T = orc.macros(p, f)
        _, gux, _, gT = fields[k]
        err_u.append(float(np.max(np.abs(gux - ux[:, 0])) / it.U_w))
        err_T.append(float(np.max(np.abs(gT - T[:, 0]))) if it.thermal else 0.0)
    return {"value": len(done) / t_sum if t_sum > 0 else None, "unit": "solves/s",
            "MLUPS": cells / t_sum / 1e6 if t_sum > 0 else None, "cores": orc.num_threads(),
            "kind": "oracle",
            "sample": f"{len(done)} cheapest instances ({cells:.3g} lattice updates, the GPU's "
                      f"step counts); then each run on to its steady state (residual 1e-12)",
            "max_err_vs_oracle": {"u_x_over_U_w": max(err_u, default=None),
                                  "T": max(err_T, default=None), "instances": len(done),
                                  "max_Ny": max((insts[k].Ny for k in done), default=None)}}


def run_batched(lbm, n=256, seed=7, tol=SOLVE_TOL, baseline_every=16):
    """Batched workload: n single-column instances in one slot table, all
    submitted at t=0, solved to the extrapolated distance tol.  Baselines on the
    same GPU, every baseline_every-th instance timed to completion: (a) alone,
    one request at a time through the same server (the same kernel, stopping
    rule and step counts); (b) the single-domain solver with its AUTO kernel
    (one warp per cell for a column), run for the same step count."""
    import numpy as np

    import inputs
    insts = inputs.batched_instances(n, seed=seed)
    ctas = resident_ctas()
    tuned = tuned_server_cfg(lbm)

    def server():
        return lbm.Server(cfg=tuned_server_cfg(lbm)[0])
    srv = server()
    t0 = time.perf_counter()
    ids = [srv.submit(_request(lbm, it, tol)) for it in insts]
    srv.drain(3600)
    makespan = time.perf_counter() - t0
    res = {r.id: r for r in srv.poll(n)}
    st = srv.stats()
    results = [res[i] for i in ids]
    fields = {k: srv.fetch(ids[k], insts[k].Ny) for k in range(n)}
    srv.close()
    ok = sum(r.status == 0 for r in results)
    sample = list(range(0, n, baseline_every))
    # (a) alone through the server, one request at a time
    srv = server()
    t_alone = 0.0
    for k in sample:
        t1 = time.perf_counter()
        srv.submit(_request(lbm, insts[k], tol))
        srv.drain(3600)
        t_alone += time.perf_counter() - t1
        srv.poll(4)
    srv.close()
    # (b) single-domain solver, AUTO kernel, the same step counts
    t_solver = 0.0
    for k in sample:
        it = insts[k]
        cfg = lbm.Config(lattice=it.lattice, Nx=1, Ny=it.Ny, eq_order=it.eq_order,
                         thermal=it.thermal, Kn=it.Kn, u_wall=(-it.U_w, it.U_w),
                         T_wall=(it.T_w, it.T_w), precision="fp32")
        sv = lbm.Solver(cfg)
        sv.init()
        sv.sync()
        t1 = time.perf_counter()
        sv.step(results[k].steps)
        sv.sync()
        t_solver += time.perf_counter() - t1
        sv.close()
    rate = n / makespan
    rate_alone = len(sample) / t_alone
    rate_solver = len(sample) / t_solver
    cpu = oracle_leg(insts, results, fields)
    return {"instances": n, "seed": seed, "tol": tol, "converged": ok,
            "makespan_s": makespan, "solves_per_s": rate,
            "one_request_at_a_time_solves_per_s": rate_alone,
            "speedup_vs_one_request_at_a_time": rate / rate_alone,
            "single_domain_solver_solves_per_s": rate_solver,
            "speedup_vs_single_domain_solver": rate / rate_solver,
            "baseline_sample": f"every {baseline_every}th instance ({len(sample)}), each timed "
                               "to completion: alone through the same server, and on the "
                               "single-domain FP32 solver (AUTO kernel) for the same steps",
            **err_est_summary(results, tol),
            "cta_budget": ctas, "autotune": tuned[1],
            "accuracy": "solves stop at an extrapolated L-inf distance tol of u_x/U_w (and T) "
                        "to the steady state; cpu_baseline.max_err_vs_oracle is the measured "
                        "error on the instances the oracle solved",
            "cpu_baseline": cpu,
            "p50_latency_s": st.p50_latency_s,
            "p99_latency_s": st.p99_latency_s, "mean_occupancy": st.mean_occupancy,
            "total_steps": int(sum(r.steps for r in results)),
            "cell_steps": int(sum(r.steps * it.Ny for r, it in zip(results, insts))),
            # one read and one write of every population per lattice update,
            # over the makespan (the pool is L2-resident: an L2 rate)
            "achieved_GBps": sum(r.steps * it.Ny * 8 * Q_OF[it.lattice]
                                 for r, it in zip(results, insts)) / makespan / 1e9}


def err_est_summary(results, tol):
    """How the converged requests stopped: by the extrapolation rule (the
    extrapolated distance to the steady state, err_est, at most tol at two
    checks in a row; its largest value is reported) or at the round-off floor
    (the change per check stopped shrinking below tol / 4; err_est is then no
    distance: 1e30 where the change no longer contracts).  Their measured
    error against the oracle is the cpu_baseline leg's max_err_vs_oracle."""
    est = [r.err_est for r in results if r.status == 0]
    extrap = [e for e in est if e <= tol]
    return {"stopped_by_extrapolation": len(extrap), "max_err_est": max(extrap, default=None),
            "stopped_at_noise_floor": len(est) - len(extrap)}


def run_serving(lbm, n=10000, seed=11, rate=200.0, tol=SOLVE_TOL):
    """Serving workload: Poisson arrivals at `rate`/s submitted in real time
    to a continuous-batching server (40 GB budget, every CTA resident)."""
    import inputs
    reqs = inputs.serving_requests(n, seed=seed, rate=rate)
    ctas = resident_ctas()
    cfg, tuning = tuned_server_cfg(lbm)
    srv = lbm.Server(cfg=cfg)
    t0 = time.perf_counter()
    ids = []
    for q in reqs:
        dt = q.arrival - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(_request(lbm, q, tol)))
    srv.drain(3600)
    wall = time.perf_counter() - t0
    res = {r.id: r for r in srv.poll(n)}
    st = srv.stats()
    results = [res[i] for i in ids]
    # the oracle leg's candidates: the cheapest of the first 2000 requests
    head = min(n, 2000)
    fields = {k: srv.fetch(ids[k], reqs[k].Ny) for k in range(head)}
    srv.close()
    cell_steps = sum(r.steps * q.Ny for r, q in zip(results, reqs))
    return {"requests": n, "seed": seed, "rate_per_s": rate, "tol": tol,
            "converged": sum(r.status == 0 for r in results),
            "p50_latency_s": st.p50_latency_s, "p99_latency_s": st.p99_latency_s,
            "mean_latency_s": st.mean_latency_s, "solves_per_s": st.solves_per_s,
            "wall_s": wall, "mean_occupancy": st.mean_occupancy, "cta_budget": ctas,
            "server_cfg": {"chunk_steps": cfg.chunk_steps, "cluster_rows": cfg.cluster_rows,
                           "class_sub": list(cfg.class_sub)},
            "cell_steps": int(cell_steps), "GLUPS": cell_steps / wall / 1e9,
            **err_est_summary(results, tol),
            "cpu_baseline": oracle_leg(reqs[:head], results[:head], fields, limit=50)}


def run_slots(lbm, n, lattice, Ny, Kn, steps, cluster_rows=256, rounding=0):
    """Rate of the batched path at a fixed step count: n identical
    single-column requests (walls -+0.1) that never meet their tolerance,
    each run for `steps` steps (rounded up to whole chunks); wall time from
    the first submit to the drain.  rounding: 0 (auto, round-to-nearest for a
    fixed step count), 1 (stochastic with conserving increments), 2 (nearest)."""
    srv = lbm.Server(mem_budget_bytes=8 << 30, max_slots=resident_ctas(), chunk_steps=100,
                     cluster_rows=cluster_rows)
    t0 = time.perf_counter()
    for _ in range(n):
        srv.submit(lbm.make_request(lattice, Ny, Kn, 0.1, tol=1e-30, max_steps=steps,
                                    rounding=rounding))
    srv.drain(600)
    wall = time.perf_counter() - t0
    res = srv.poll(n)
    srv.close()
    mean_steps = sum(r.steps for r in res) / len(res)
    return {"slots": n, "lattice": lattice, "Ny": Ny, "Kn": Kn, "cluster_rows": cluster_rows,
            "rounding": rounding,
            "mean_steps": mean_steps, "wall_s": wall,
            "us_per_step_per_slot": wall / mean_steps * 1e6,
            "GLUPS": n * mean_steps * Ny / wall / 1e9}


def run_precision(lbm, prec: str, steps: int, warmup: int):
    """The grid workload (D2Q37 4096 x 2048) with another storage format: the
    autotuned kernel's step time by CUDA events on the solver's stream over
    `steps` steps after `warmup`, and its roofline at that format's
    algorithmic bytes per lattice update."""
    import torch

    cfg = lbm.Config(lattice="D2Q37", Nx=WORKLOAD["Nx"], Ny=WORKLOAD["Ny"], eq_order=4,
                     thermal=True, Kn=WORKLOAD["Kn"], u_wall=WORKLOAD["u_wall"],
                     T_wall=WORKLOAD["T_wall"], precision=prec,
                     noise_amp=WORKLOAD["noise_amp"], seed=WORKLOAD["seed"])
    stream = torch.cuda.Stream()
    s = lbm.Solver(cfg, stream=stream)
    kern, var, _ = s.autotune(10)
    s.init()
    s.step(warmup)
    s.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    e1.synchronize()
    s.close()
    cells = cfg.Nx * cfg.Ny
    ms_step = e0.elapsed_time(e1) / steps
    peak, peak_kind = measured_peaks()
    bpl = BYTES_PER_LU[prec]
    achieved = bpl * cells / (ms_step * 1e-3) / 1e9
    return {"workload": workload_name(prec, cfg.Nx, cfg.Ny), "dtype": DTYPE[prec],
            "value": job_rate(1, cells, steps, ms_step * steps * 1e-3), "unit": "MLUPS",
            "ms_per_step": ms_step, "steps": steps, "warmup": warmup,
            "kernel": kernel_name(kern, var, prec),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": step_traffic(f"{prec}:{kern}:{var}:{cfg.Nx}x{cfg.Ny}"),
                         "peak_kind": f"{peak_kind} (copy burst)", "bytes_per_lu": bpl}}


def run_column_fp64(lbm, steps=20000):
    """Single-column FP64 run (D2Q25, 1 x 64, Kn 0.1, walls -+0.1): 20000 steps,
    GPU microseconds per step and MLUPS, against the oracle on the host."""
    import numpy as np
    import torch
    from oracle import oracle as orc
    cfg = lbm.Config(lattice="D2Q25", Nx=1, Ny=64, Kn=0.1, u_wall=(-0.1, 0.1), precision="fp64")
    s = lbm.Solver(cfg)
    s.init()
    s.step(100)
    s.sync()
    s_kernel = {1: "direct", 2: "staged", 3: "cellwarp"}.get(s.kernel_info()[0], "?")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(steps)
    e1.record(s.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    s.close()
    # CPU baseline: the oracle (as it stands) on the same 20000 steps, on all
    # host cores and on one
    p = orc.Problem(lattice="D2Q25", Nx=1, Ny=64, Kn=0.1, u_wall=(-0.1, 0.1))
    cores = orc.num_threads()
    ot = {}
    for n in (cores, 1):
        orc.set_num_threads(n)
        f = orc.init_fields(p, np.ones((64, 1)))
        t0 = time.perf_counter()
        orc.run(p, f, steps)
        ot[n] = time.perf_counter() - t0
    orc.set_num_threads(cores)
    return {"workload": "D2Q25 2nd-order isothermal Couette 1x64 FP64, 20000 steps",
            "us_per_step": ms * 1e3 / steps, "MLUPS": 64 * steps / (ms * 1e-3) / 1e6,
            "kernel": s_kernel, "gpu_launches": steps,
            "cpu_baseline": {"value": 64 * steps / ot[cores] / 1e6, "unit": "MLUPS",
                             "us_per_step": ot[cores] * 1e6 / steps, "cores": cores,
                             "kind": "oracle", "sample": "the same 20000 steps",
                             "one_core": {"value": 64 * steps / ot[1] / 1e6,
                                          "us_per_step": ot[1] * 1e6 / steps}}}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, one bounded sample step per timed step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import inputs
    from oracle import oracle as orc
    orc.build()
    Nx, Ny = WORKLOAD["Nx"], 32
    p = orc.Problem(lattice="D2Q37", Nx=Nx, Ny=Ny, eq_order=4, thermal=True, Kn=0.05,
                    u_wall=(-0.3, 0.3), T_wall=(1.0, 1.0))
    f = orc.init_fields(p, inputs.rho_field(Nx, Ny, 1e-3, seed=7))
    orc.run(p, f, args.warmup)
    t0 = time.perf_counter()
    orc.run(p, f, args.steps)
    dt = time.perf_counter() - t0
    v = Nx * Ny * args.steps / dt / 1e6
    sample = f"FP64 oracle, {Nx}x{Ny} rows of the same Couette setup per step"
    print(json.dumps({
        "impl": "reference", "metric": "D2Q37 MLUPS", "value": v, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.precision, WORKLOAD["Nx"], WORKLOAD["Ny"]),
                   "sample_rows": Ny},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": orc.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


# kernel sources whose change invalidates recorded DRAM counters
TRAFFIC_SOURCES = ["k_step_direct.cuh", "k_step_staged.cuh", "lbm_device.cuh", "lbm_internal.h",
                   "launchers_impl.cuh"]


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1209_5201_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def step_traffic(key: str):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch recorded by an ncu
    capture (profiles/step_traffic.json), or None when there is no capture of
    this configuration or the kernel sources changed since it was taken."""
    tf = os.path.join(ROOT, "profiles", "step_traffic.json")
    try:
        with open(tf) as fh:
            d = json.load(fh)
        e = d["entries"].get(key)
        if e is None or d.get("kernel_sources_sha256") != kernel_sources_sha256():
            return None
        return e["dram_bytes_per_launch"]
    except (OSError, KeyError, ValueError):
        return None


def kernel_name(kern: int, var: int, prec: str) -> str:
    """Readable name of a (kernel, variant) choice."""
    if kern == 2:
        return f"staged{var}"
    if kern == 3:
        return "cellwarp"
    return f"direct{var}"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16dev", "bf16shift"])
    ap.add_argument("--kernel", type=int, default=-1,
                    help="-1: autotune; 1: direct; 2: staged (with --variant)")
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--Nx", type=int, default=WORKLOAD["Nx"])
    ap.add_argument("--Ny", type=int, default=WORKLOAD["Ny"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the per-variant timing diagnostic")
    ap.add_argument("--workload", default="grid", choices=["grid", "batched", "serving", "slots"],
                    help="grid: the D2Q37 4096x2048 line (default, also runs the batched "
                         "workload and a shortened serving run); batched / serving: only that; "
                         "slots: batched-path rate of --slots identical columns")
    ap.add_argument("--slots", type=int, default=1)
    ap.add_argument("--lattice", default="D2Q37", choices=["D2Q17", "D2Q25", "D2Q37"])
    ap.add_argument("--Kn", type=float, default=0.005)
    ap.add_argument("--slot-steps", type=int, default=20000)
    ap.add_argument("--cluster-rows", type=int, default=256)
    ap.add_argument("--rounding", type=int, default=0, choices=[0, 1, 2],
                    help="slots workload: 0 auto, 1 stochastic, 2 nearest")
    ap.add_argument("--serving-requests", type=int, default=10000)
    ap.add_argument("--no-extras", action="store_true",
                    help="grid line only (skip the batched and serving runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import inputs
    from paper_1209_5201_gb300 import lbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    lbm.load()
    if args.workload in ("batched", "serving", "slots"):
        if rank == 0:
            if args.workload == "batched":
                r = run_batched(lbm)
            elif args.workload == "serving":
                r = run_serving(lbm, n=args.serving_requests)
            else:
                r = run_slots(lbm, args.slots, args.lattice, args.Ny, args.Kn, args.slot_steps,
                              args.cluster_rows, args.rounding)
            print(json.dumps({"workload": args.workload, **r}))
        return 0
    cfg = lbm.Config(lattice="D2Q37", Nx=args.Nx, Ny=args.Ny, eq_order=4, thermal=True,
                     Kn=WORKLOAD["Kn"], u_wall=WORKLOAD["u_wall"], T_wall=WORKLOAD["T_wall"],
                     precision=args.precision, kernel=max(args.kernel, 0),
                     noise_amp=WORKLOAD["noise_amp"], seed=WORKLOAD["seed"])
    stream = torch.cuda.Stream()
    s = lbm.Solver(cfg, stream=stream)
    cells = cfg.Nx * cfg.Ny

    # step time of every compiled kernel variant (diagnostic), then the choice
    variants_ms = {}
    s.init()
    nd, ns = s.variant_count(1), s.variant_count(2)
    for kv in ([] if args.no_variants else [(1, v) for v in range(nd)] + [(2, v) for v in range(ns)]):
        try:
            s.set_kernel(*kv)
        except lbm.LBMError:
            continue               # the staged kernel on a grid of several x-tiles
        s.step(3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(20)
        e1.record(stream)
        e1.synchronize()
        variants_ms[kernel_name(kv[0], kv[1], args.precision)] = e0.elapsed_time(e1) / 20
    if args.kernel < 0:
        kern, var, _ = s.autotune(10)
    else:
        s.set_kernel(args.kernel, args.variant)
        kern, var = args.kernel, args.variant

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    # ---- device-resident throughput -------------------------------------------
    s.init()
    s.step(args.warmup)
    s.sync()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark_start()
    ev0.record(stream)
    s.step(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    clocks.mark_stop()
    barrier()
    clk = clocks.stop()
    ms = reduce_max(ev0.elapsed_time(ev1), dist, "cuda")
    ms_step = ms / args.steps
    value = job_rate(world, cells, args.steps, ms * 1e-3)

    # ---- end to end through the public API with host buffers --------------------
    # per job: init from a pinned host density field, the K steps, then the four
    # macroscopic fields back into pinned host memory
    # (one untimed pass first, then the median of three timed passes: the
    # first host-buffer round trip of a process pays one-off host costs)
    rho_h = torch.from_numpy(inputs.rho_field(cfg.Nx, cfg.Ny, 1e-3, seed=7)).pin_memory()
    outs = [torch.empty((cfg.Ny, cfg.Nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    passes = []
    for rep in range(4):
        barrier()
        t0 = time.perf_counter()
        lbm.lbm_solver_init_fields(s.h, rho_h.numpy())
        s.step(args.steps)
        lbm.lbm_solver_macros(s.h, *[o.numpy() for o in outs])
        dt = reduce_max(time.perf_counter() - t0, dist, "cuda")
        if rep > 0:
            passes.append(dt)
    e2e_s = statistics.median(passes)
    e2e = {"value": job_rate(world, cells, args.steps, e2e_s), "unit": "MLUPS",
           "h2d_bytes_per_step": cells * 8 / args.steps,
           "d2h_bytes_per_step": 4 * cells * 8 / args.steps,
           "passes": "median of 3 timed passes after 1 untimed",
           "pass_ms": [round(1e3 * p, 3) for p in passes]}
    s.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = measured_peaks()
    bpl = BYTES_PER_LU[args.precision]
    achieved = bpl * cells / (ms_step * 1e-3) / 1e9
    traffic = step_traffic(f"{args.precision}:{kern}:{var}:{cfg.Nx}x{cfg.Ny}")
    out = {
        "metric": "D2Q37 MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": workload_name(args.precision, cfg.Nx, cfg.Ny), "lattice": "D2Q37",
                   "Nx": cfg.Nx, "Ny": cfg.Ny, "eq_order": 4, "Kn": WORKLOAD["Kn"],
                   "U_w": 0.3, "kernel": kernel_name(kern, var, args.precision),
                   "l2": "inputs larger than L2 (state %.2f GB)" % (2 * cells * bpl / 2 / 1e9),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} (copy burst)",
                     "bytes_per_lu": bpl},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk,
        "variants_ms": variants_ms,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.precision)
    if not args.no_extras and world == 1:
        if args.precision == "fp32":
            # the two BF16 storage formats on the same grid
            out["precisions"] = {p: run_precision(lbm, p, max(args.steps, 500), args.warmup)
                                 for p in ("bf16shift", "bf16dev")}
        out["column_fp64"] = run_column_fp64(lbm)
        out["batched"] = run_batched(lbm)
        out["serving"] = run_serving(lbm, n=args.serving_requests)
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
