"""Thin ctypes binding of include/lbm.h (argument marshalling only).

Every function named lbm_* here calls the C function of the same name in the
in-tree CUDA library (paper_1209_5201_gb300/_build/liblbm_gb300.so) and raises
LBMError on a non-zero status.  There is no fallback: if the library is
missing, load() raises.  Host arrays are numpy float64; device memory and the
CUDA stream come from PyTorch when a Solver is built through the helper class.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm_gb300.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_EBUDGET, LBM_ENOTCONVERGED = 0, 1, 2, 3, 4
LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ECUDA, LBM_EBUSY, LBM_ECANCELLED = 5, 6, 7, 8, 9
LBM_LATTICE_D2Q17, LBM_LATTICE_D2Q25, LBM_LATTICE_D2Q25B, LBM_LATTICE_D2Q37 = 17, 25, 26, 37
LBM_FP64, LBM_FP32, LBM_BF16DEV, LBM_BF16SHIFT = 0, 1, 2, 3
LBM_KERNEL_AUTO, LBM_KERNEL_DIRECT, LBM_KERNEL_STAGED, LBM_KERNEL_CELLWARP = 0, 1, 2, 3
LBM_ROUND_AUTO, LBM_ROUND_STOCHASTIC, LBM_ROUND_NEAREST = 0, 1, 2
LBM_INIT_REST, LBM_INIT_NS = 0, 1

LATTICE_KIND = {"D2Q17": 17, "D2Q25": 25, "D2Q25b": 26, "D2Q37": 37}
PRECISION = {"fp64": 0, "fp32": 1, "bf16dev": 2, "bf16shift": 3}


class LBMError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class lbm_params(C.Structure):
    _fields_ = [("Nx", C.c_int32), ("Ny", C.c_int32), ("eq_order", C.c_int32),
                ("thermal", C.c_int32), ("Kn", C.c_double), ("tau", C.c_double),
                ("mu_exp", C.c_double), ("u_wall", C.c_double * 2), ("T_wall", C.c_double * 2),
                ("precision", C.c_int32), ("kernel", C.c_int32), ("rho0", C.c_double),
                ("noise_amp", C.c_double), ("seed", C.c_uint64), ("accom", C.c_double * 2)]


class lbm_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("mass0", C.c_double), ("mass", C.c_double),
                ("mass_drift", C.c_double), ("residual", C.c_double),
                ("wall_in", C.c_double * 2)]


class lbm_request(C.Structure):
    _fields_ = [("lattice", C.c_int32), ("Ny", C.c_int32), ("eq_order", C.c_int32),
                ("thermal", C.c_int32), ("Kn", C.c_double), ("tau", C.c_double),
                ("mu_exp", C.c_double), ("u_wall", C.c_double * 2), ("T_wall", C.c_double * 2),
                ("tol", C.c_double), ("max_steps", C.c_int64), ("tag", C.c_uint64),
                ("accom", C.c_double * 2), ("rounding", C.c_int32), ("init", C.c_int32)]


class lbm_result(C.Structure):
    _fields_ = [("id", C.c_uint64), ("tag", C.c_uint64), ("status", C.c_int32),
                ("Ny", C.c_int32), ("steps", C.c_int64), ("residual", C.c_double),
                ("err_est", C.c_double), ("mass", C.c_double), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double)]


class lbm_server_cfg(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_size_t), ("max_slots", C.c_int32),
                ("chunk_steps", C.c_int32), ("precision", C.c_int32), ("use_graph", C.c_int32),
                ("cluster_rows", C.c_int32), ("class_sub", C.c_int32 * 5)]


class lbm_server_tuning(C.Structure):
    _fields_ = [("ny", C.c_int32 * 3), ("lone_us", C.c_double * 5 * 3 * 3),
                ("chunk_try", C.c_int32 * 5), ("chunk_glups", C.c_double * 5),
                ("seconds", C.c_double)]


class lbm_server_metrics(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("running", C.c_int64),
                ("queued", C.c_int64), ("chunks", C.c_int64), ("p50_latency_s", C.c_double),
                ("p99_latency_s", C.c_double), ("mean_latency_s", C.c_double),
                ("solves_per_s", C.c_double), ("mean_occupancy", C.c_double),
                ("pool_bytes", C.c_size_t), ("pool_used_bytes", C.c_size_t),
                ("promoted", C.c_int64), ("demoted", C.c_int64)]


_lib = None
_VP = C.c_void_p
_DP = C.POINTER(C.c_double)

_SIGS = {
    "lbm_status_string": ([C.c_int], C.c_char_p),
    "lbm_last_error": ([C.c_char_p, C.c_size_t], C.c_int),
    "lbm_version": ([C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "lbm_lattice_create": ([C.c_int, C.POINTER(_VP)], C.c_int),
    "lbm_lattice_create_custom": ([C.c_int, C.POINTER(C.c_int8), _DP, C.c_double, C.POINTER(_VP)],
                                  C.c_int),
    "lbm_lattice_destroy": ([_VP], C.c_int),
    "lbm_lattice_info": ([_VP, C.POINTER(C.c_int), _DP, C.POINTER(C.c_int), C.POINTER(C.c_int)],
                         C.c_int),
    "lbm_lattice_tables": ([_VP, C.POINTER(C.c_int8), _DP], C.c_int),
    "lbm_lattice_verify": ([_VP, C.c_int, _DP], C.c_int),
    "lbm_params_default": ([C.POINTER(lbm_params)], None),
    "lbm_solver_required_bytes": ([_VP, C.POINTER(lbm_params), C.POINTER(C.c_size_t)], C.c_int),
    "lbm_solver_create": ([_VP, C.POINTER(lbm_params), _VP, _VP, C.c_size_t, C.POINTER(_VP)],
                          C.c_int),
    "lbm_solver_destroy": ([_VP], C.c_int),
    "lbm_solver_init": ([_VP], C.c_int),
    "lbm_solver_init_fields": ([_VP, _DP, _DP, _DP, _DP], C.c_int),
    "lbm_solver_step": ([_VP, C.c_int64], C.c_int),
    "lbm_solver_sync": ([_VP], C.c_int),
    "lbm_solver_get_f": ([_VP, _DP], C.c_int),
    "lbm_solver_set_f": ([_VP, _DP], C.c_int),
    "lbm_solver_macros": ([_VP, _DP, _DP, _DP, _DP], C.c_int),
    "lbm_solver_macros_mean": ([_VP, C.c_int64, _DP, _DP, _DP, _DP], C.c_int),
    "lbm_solver_fluxes": ([_VP, _DP, _DP, _DP, _DP, _DP], C.c_int),
    "lbm_solver_state_bytes": ([_VP, C.POINTER(C.c_size_t)], C.c_int),
    "lbm_solver_get_state": ([_VP, _VP, C.c_size_t], C.c_int),
    "lbm_solver_set_state": ([_VP, _VP, C.c_size_t], C.c_int),
    "lbm_solver_residual_history": ([_VP, C.POINTER(C.c_int64), _DP, C.c_int32,
                                     C.POINTER(C.c_int32)], C.c_int),
    "lbm_solver_run_to_residual": ([_VP, C.c_double, C.c_int64, C.c_int32,
                                    C.POINTER(C.c_int64), _DP], C.c_int),
    "lbm_solver_stats": ([_VP, C.POINTER(lbm_stats)], C.c_int),
    "lbm_solver_wall_mass": ([_VP, _DP], C.c_int),
    "lbm_solver_set_kernel": ([_VP, C.c_int32, C.c_int32], C.c_int),
    "lbm_solver_set_wait_limit": ([_VP, C.c_uint64], C.c_int),
    "lbm_solver_kernel_info": ([_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                C.POINTER(C.c_int32)], C.c_int),
    "lbm_solver_variant_count": ([_VP, C.c_int32, C.POINTER(C.c_int32)], C.c_int),
    "lbm_solver_autotune": ([_VP, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _DP],
                            C.c_int),
    "lbm_server_cfg_default": ([C.POINTER(lbm_server_cfg)], None),
    "lbm_request_bytes": ([C.POINTER(lbm_request), C.POINTER(C.c_size_t)], C.c_int),
    "lbm_server_create": ([C.POINTER(lbm_server_cfg), _VP, C.POINTER(_VP)], C.c_int),
    "lbm_server_submit": ([_VP, C.POINTER(lbm_request), C.POINTER(C.c_uint64)], C.c_int),
    "lbm_server_poll": ([_VP, C.POINTER(lbm_result), C.c_int32, C.POINTER(C.c_int32)], C.c_int),
    "lbm_server_fetch": ([_VP, C.c_uint64, _DP, _DP, _DP, _DP], C.c_int),
    "lbm_server_cancel": ([_VP, C.c_uint64], C.c_int),
    "lbm_server_drain": ([_VP, C.c_double], C.c_int),
    "lbm_server_stats": ([_VP, C.POINTER(lbm_server_metrics)], C.c_int),
    "lbm_server_destroy": ([_VP], C.c_int),
    "lbm_server_autotune": ([C.POINTER(lbm_server_cfg), _VP, C.POINTER(lbm_server_tuning)], C.c_int),
    "lbm_batch_solve": ([C.POINTER(lbm_server_cfg), _VP, C.POINTER(lbm_request), C.c_int32,
                         C.POINTER(lbm_result), C.c_double], C.c_int),
    "lbm_residual_noalloc": ([_VP, _VP, _VP, _VP, C.c_int64, C.c_double, C.c_int32, _VP, _VP],
                             C.c_int),
}


def load() -> C.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                              "(run __graft_entry__.build())")
        lib = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def lbm_last_error() -> str:
    buf = C.create_string_buffer(512)
    load().lbm_last_error(buf, 512)
    return buf.value.decode(errors="replace")


last_error = lbm_last_error


def _check(status: int, where: str, ok=(LBM_OK,)) -> int:
    if status not in ok:
        raise LBMError(status, where, last_error())
    return status


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


# ---- functions with the C names ------------------------------------------------

def lbm_status_string(st: int) -> str:
    return load().lbm_status_string(st).decode()


def lbm_version():
    a, b = C.c_int(), C.c_int()
    load().lbm_version(C.byref(a), C.byref(b))
    return a.value, b.value


def lbm_lattice_create(kind: int):
    h = _VP()
    _check(load().lbm_lattice_create(kind, C.byref(h)), "lbm_lattice_create")
    return h


def lbm_lattice_create_custom(e, w, r: float):
    """e: (Q, 2) integer velocities, w: (Q,) weights in the same order, r: scale."""
    e = np.ascontiguousarray(e, dtype=np.int8)
    w = np.ascontiguousarray(w, dtype=np.float64)
    if e.ndim != 2 or e.shape[1] != 2 or w.shape != (e.shape[0],):
        raise ValueError("e must be (Q, 2) and w (Q,)")
    h = _VP()
    _check(load().lbm_lattice_create_custom(e.shape[0], e.ctypes.data_as(C.POINTER(C.c_int8)),
                                            _dp(w), float(r), C.byref(h)),
           "lbm_lattice_create_custom")
    return h


def lbm_lattice_destroy(h) -> None:
    load().lbm_lattice_destroy(h)


def lbm_lattice_info(h):
    Q, N, deg = C.c_int(), C.c_int(), C.c_int()
    r = C.c_double()
    _check(load().lbm_lattice_info(h, C.byref(Q), C.byref(r), C.byref(N), C.byref(deg)),
           "lbm_lattice_info")
    return Q.value, r.value, N.value, deg.value


def lbm_lattice_tables(h):
    Q = lbm_lattice_info(h)[0]
    e = np.zeros((Q, 2), dtype=np.int8)
    w = np.zeros(Q, dtype=np.float64)
    _check(load().lbm_lattice_tables(h, e.ctypes.data_as(C.POINTER(C.c_int8)), _dp(w)),
           "lbm_lattice_tables")
    return e, w


def lbm_lattice_verify(h, degree: int) -> float:
    v = C.c_double()
    _check(load().lbm_lattice_verify(h, degree, C.byref(v)), "lbm_lattice_verify")
    return v.value


def lbm_params_default() -> lbm_params:
    p = lbm_params()
    load().lbm_params_default(C.byref(p))
    return p


def lbm_solver_required_bytes(lat, p: lbm_params) -> int:
    n = C.c_size_t()
    _check(load().lbm_solver_required_bytes(lat, C.byref(p), C.byref(n)),
           "lbm_solver_required_bytes")
    return n.value


def lbm_solver_create(lat, p: lbm_params, stream: int = 0, device_mem: int = 0,
                      device_bytes: int = 0):
    h = _VP()
    _check(load().lbm_solver_create(lat, C.byref(p), _VP(stream or None), _VP(device_mem or None),
                                    device_bytes, C.byref(h)), "lbm_solver_create")
    return h


def lbm_solver_destroy(h) -> None:
    load().lbm_solver_destroy(h)


def lbm_solver_init(h) -> None:
    _check(load().lbm_solver_init(h), "lbm_solver_init")


def lbm_solver_init_fields(h, rho, ux=None, uy=None, T=None) -> None:
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64)
            for a in (rho, ux, uy, T)]
    _check(load().lbm_solver_init_fields(h, *[_dp(a) for a in arrs]), "lbm_solver_init_fields")


def lbm_solver_step(h, n: int) -> None:
    _check(load().lbm_solver_step(h, int(n)), "lbm_solver_step")


def lbm_solver_sync(h) -> None:
    _check(load().lbm_solver_sync(h), "lbm_solver_sync")


def lbm_solver_get_f(h, out: np.ndarray) -> np.ndarray:
    _check(load().lbm_solver_get_f(h, _dp(out)), "lbm_solver_get_f")
    return out


def lbm_solver_set_f(h, f: np.ndarray) -> None:
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(load().lbm_solver_set_f(h, _dp(f)), "lbm_solver_set_f")


def lbm_solver_macros(h, rho=None, ux=None, uy=None, T=None) -> None:
    _check(load().lbm_solver_macros(h, _dp(rho), _dp(ux), _dp(uy), _dp(T)), "lbm_solver_macros")


def lbm_solver_macros_mean(h, nsteps: int, rho=None, ux=None, uy=None, T=None) -> None:
    _check(load().lbm_solver_macros_mean(h, int(nsteps), _dp(rho), _dp(ux), _dp(uy), _dp(T)),
           "lbm_solver_macros_mean")


def lbm_solver_fluxes(h, sxx=None, sxy=None, syy=None, qx=None, qy=None) -> None:
    _check(load().lbm_solver_fluxes(h, _dp(sxx), _dp(sxy), _dp(syy), _dp(qx), _dp(qy)),
           "lbm_solver_fluxes")


def lbm_solver_state_bytes(h) -> int:
    n = C.c_size_t()
    _check(load().lbm_solver_state_bytes(h, C.byref(n)), "lbm_solver_state_bytes")
    return n.value


def lbm_solver_get_state(h) -> bytes:
    n = lbm_solver_state_bytes(h)
    buf = C.create_string_buffer(n)
    _check(load().lbm_solver_get_state(h, buf, n), "lbm_solver_get_state")
    return buf.raw


def lbm_solver_set_state(h, data: bytes) -> None:
    buf = C.create_string_buffer(data, len(data))
    _check(load().lbm_solver_set_state(h, buf, len(data)), "lbm_solver_set_state")


def lbm_solver_run_to_residual(h, tol: float, max_steps: int, check_every: int = 100):
    steps = C.c_int64()
    res = C.c_double()
    st = _check(load().lbm_solver_run_to_residual(h, tol, int(max_steps), int(check_every),
                                                  C.byref(steps), C.byref(res)),
                "lbm_solver_run_to_residual", ok=(LBM_OK, LBM_ENOTCONVERGED))
    return st, steps.value, res.value


def lbm_solver_residual_history(h):
    n = C.c_int32()
    _check(load().lbm_solver_residual_history(h, None, None, 0, C.byref(n)),
           "lbm_solver_residual_history")
    steps = np.zeros(n.value, dtype=np.int64)
    res = np.zeros(n.value, dtype=np.float64)
    if n.value:
        _check(load().lbm_solver_residual_history(
            h, steps.ctypes.data_as(C.POINTER(C.c_int64)), _dp(res), n.value, C.byref(n)),
            "lbm_solver_residual_history")
    return steps, res


def lbm_solver_stats(h) -> lbm_stats:
    s = lbm_stats()
    _check(load().lbm_solver_stats(h, C.byref(s)), "lbm_solver_stats")
    return s


def lbm_solver_wall_mass(h, out: np.ndarray) -> np.ndarray:
    _check(load().lbm_solver_wall_mass(h, _dp(out)), "lbm_solver_wall_mass")
    return out


def lbm_solver_set_kernel(h, kernel: int, variant: int = 0) -> None:
    _check(load().lbm_solver_set_kernel(h, int(kernel), int(variant)), "lbm_solver_set_kernel")


def lbm_solver_set_wait_limit(h, ns: int) -> None:
    _check(load().lbm_solver_set_wait_limit(h, int(ns)), "lbm_solver_set_wait_limit")


def lbm_solver_kernel_info(h):
    k, v, n = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().lbm_solver_kernel_info(h, C.byref(k), C.byref(v), C.byref(n)),
           "lbm_solver_kernel_info")
    return k.value, v.value, n.value


def lbm_solver_variant_count(h, kernel: int) -> int:
    n = C.c_int32()
    _check(load().lbm_solver_variant_count(h, int(kernel), C.byref(n)), "lbm_solver_variant_count")
    return n.value


def lbm_solver_autotune(h, trial_steps: int = 10):
    k, v = C.c_int32(), C.c_int32()
    ms = C.c_double()
    _check(load().lbm_solver_autotune(h, int(trial_steps), C.byref(k), C.byref(v), C.byref(ms)),
           "lbm_solver_autotune")
    return k.value, v.value, ms.value


def lbm_server_cfg_default() -> lbm_server_cfg:
    c = lbm_server_cfg()
    load().lbm_server_cfg_default(C.byref(c))
    return c


def lbm_request_bytes(req: lbm_request) -> int:
    n = C.c_size_t()
    _check(load().lbm_request_bytes(C.byref(req), C.byref(n)), "lbm_request_bytes")
    return n.value


def lbm_server_create(cfg: lbm_server_cfg, stream: int = 0):
    h = _VP()
    _check(load().lbm_server_create(C.byref(cfg), _VP(stream or None), C.byref(h)),
           "lbm_server_create")
    return h


def lbm_server_submit(h, req: lbm_request) -> int:
    i = C.c_uint64()
    _check(load().lbm_server_submit(h, C.byref(req), C.byref(i)), "lbm_server_submit")
    return i.value


def lbm_server_poll(h, max_results: int = 1024):
    buf = (lbm_result * max(1, max_results))()
    n = C.c_int32()
    _check(load().lbm_server_poll(h, buf, int(max_results), C.byref(n)), "lbm_server_poll")
    return [buf[i] for i in range(n.value)]


def lbm_server_cancel(h, rid: int) -> None:
    _check(load().lbm_server_cancel(h, int(rid)), "lbm_server_cancel")


def lbm_server_fetch(h, rid: int, Ny: int):
    out = [np.empty(Ny) for _ in range(4)]
    _check(load().lbm_server_fetch(h, C.c_uint64(rid), *[_dp(a) for a in out]),
           "lbm_server_fetch")
    return tuple(out)


def lbm_server_drain(h, timeout_s: float = 600.0) -> None:
    _check(load().lbm_server_drain(h, float(timeout_s)), "lbm_server_drain")


def lbm_server_stats(h) -> lbm_server_metrics:
    m = lbm_server_metrics()
    _check(load().lbm_server_stats(h, C.byref(m)), "lbm_server_stats")
    return m


def lbm_server_destroy(h) -> None:
    load().lbm_server_destroy(h)


def lbm_server_autotune(cfg: lbm_server_cfg, stream: int = 0):
    """Tune cfg in place (chunk_steps, cluster_rows, class_sub); returns the
    measured times as a dict."""
    rep = lbm_server_tuning()
    _check(load().lbm_server_autotune(C.byref(cfg), _VP(stream or None), C.byref(rep)),
           "lbm_server_autotune")
    return {"ny": list(rep.ny),
            "lone_us": [[list(rep.lone_us[li][hi]) for hi in range(3)] for li in range(3)],
            "chunk_try": list(rep.chunk_try), "chunk_glups": list(rep.chunk_glups),
            "seconds": rep.seconds}


def lbm_batch_solve(cfg: lbm_server_cfg, reqs, stream: int = 0, timeout_s: float = 600.0):
    arr = (lbm_request * len(reqs))(*reqs)
    out = (lbm_result * max(1, len(reqs)))()
    _check(load().lbm_batch_solve(C.byref(cfg), _VP(stream or None), arr, len(reqs), out,
                                  float(timeout_s)), "lbm_batch_solve")
    return [out[i] for i in range(len(reqs))]


def _devptr(a) -> int:
    return a.data_ptr() if hasattr(a, "data_ptr") else int(a)


def lbm_residual_noalloc(ux, T, ux_prev, T_prev, n: int, T_ref: float, thermal: bool, res,
                         stream: int = 0) -> None:
    """Device arrays (torch tensors or raw pointers); see include/lbm.h."""
    _check(load().lbm_residual_noalloc(_VP(_devptr(ux)), _VP(_devptr(T)), _VP(_devptr(ux_prev)),
                                       _VP(_devptr(T_prev)), int(n), float(T_ref), int(thermal),
                                       _VP(_devptr(res)), _VP(stream or None)),
           "lbm_residual_noalloc")


def make_request(lattice: str, Ny: int, Kn: float, U_w: float, T_w: float = 1.0,
                 tol: float = 1e-5, max_steps: int = 10_000_000, tag: int = 0,
                 eq_order: int | None = None, thermal: bool | None = None,
                 tau: float = 0.0, accom: tuple = (1.0, 1.0),
                 rounding: int = LBM_ROUND_AUTO, init: int = LBM_INIT_REST) -> lbm_request:
    """A Couette request: walls at -U_w (bottom) and +U_w (top), both at T_w."""
    o, t = (4, True) if lattice == "D2Q37" else (2, False)
    r = lbm_request()
    r.lattice = LATTICE_KIND[lattice]
    r.Ny = Ny
    r.eq_order = o if eq_order is None else eq_order
    r.thermal = int(t if thermal is None else thermal)
    r.Kn, r.tau, r.mu_exp = Kn, tau, 1.0
    r.u_wall[0], r.u_wall[1] = -U_w, U_w
    r.T_wall[0] = r.T_wall[1] = T_w
    r.tol, r.max_steps, r.tag = tol, max_steps, tag
    r.accom[0], r.accom[1] = accom
    r.rounding = rounding
    r.init = init
    return r


# ---- convenience wrappers (still marshalling only) -----------------------------

class Lattice:
    def __init__(self, name: str, custom=None):
        """A built-in lattice by name, or custom=(e, w, r): one of the built-in
        velocity sets with the caller's weights and scale."""
        self.name = name
        self.h = lbm_lattice_create(LATTICE_KIND[name]) if custom is None else \
            lbm_lattice_create_custom(*custom)
        self.Q, self.r, self.ghost_depth, self.degree = lbm_lattice_info(self.h)
        self.e, self.w = lbm_lattice_tables(self.h)

    def verify(self, degree: int) -> float:
        return lbm_lattice_verify(self.h, degree)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            lbm_lattice_destroy(self.h)
            self.h = None


@dataclass
class Config:
    lattice: str = "D2Q25"
    Nx: int = 1
    Ny: int = 64
    eq_order: int = 2
    thermal: bool = False
    Kn: float = 0.1
    tau: float = 0.0
    mu_exp: float = 1.0
    u_wall: tuple = (-0.1, 0.1)
    T_wall: tuple = (1.0, 1.0)
    precision: str = "fp64"
    kernel: int = LBM_KERNEL_AUTO
    rho0: float = 1.0
    noise_amp: float = 0.0
    seed: int = 7
    accom: tuple = (1.0, 1.0)

    def params(self) -> lbm_params:
        p = lbm_params_default()
        p.Nx, p.Ny, p.eq_order, p.thermal = self.Nx, self.Ny, self.eq_order, int(self.thermal)
        p.Kn, p.tau, p.mu_exp = self.Kn, self.tau, self.mu_exp
        p.u_wall[0], p.u_wall[1] = self.u_wall
        p.T_wall[0], p.T_wall[1] = self.T_wall
        p.precision, p.kernel = PRECISION[self.precision], self.kernel
        p.rho0, p.noise_amp, p.seed = self.rho0, self.noise_amp, self.seed
        p.accom[0], p.accom[1] = self.accom
        return p


class Server:
    """Continuous-batching server on torch's current CUDA device; the worker
    thread owns its own CUDA stream."""

    def __init__(self, mem_budget_bytes: int = 40 << 30, max_slots: int = 256,
                 chunk_steps: int = 100, use_graph: bool = True, cluster_rows: int = 256,
                 cfg: "lbm_server_cfg | None" = None):
        """A server with the given settings, or with `cfg` as a whole (e.g. one
        lbm_server_autotune filled in)."""
        import torch
        if cfg is not None:
            self.cfg = cfg
        else:
            self.cfg = lbm_server_cfg_default()
            self.cfg.mem_budget_bytes = int(mem_budget_bytes)
            self.cfg.max_slots = int(max_slots)
            self.cfg.chunk_steps = int(chunk_steps)
            self.cfg.use_graph = int(use_graph)
            self.cfg.cluster_rows = int(cluster_rows)
        self.stream = torch.cuda.Stream()
        self.h = lbm_server_create(self.cfg, self.stream.cuda_stream)

    def submit(self, req: lbm_request) -> int:
        return lbm_server_submit(self.h, req)

    def poll(self, max_results: int = 1024):
        return lbm_server_poll(self.h, max_results)

    def cancel(self, rid: int):
        lbm_server_cancel(self.h, rid)

    def fetch(self, rid: int, Ny: int):
        return lbm_server_fetch(self.h, rid, Ny)

    def drain(self, timeout_s: float = 600.0):
        lbm_server_drain(self.h, timeout_s)

    def stats(self) -> lbm_server_metrics:
        return lbm_server_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """A solver whose device memory is a torch allocation on the current device
    and whose work runs on torch's current CUDA stream."""

    def __init__(self, cfg: Config, stream=None, lattice: "Lattice | None" = None):
        import torch
        self.cfg = cfg
        self.lat = lattice if lattice is not None else Lattice(cfg.lattice)
        self.p = cfg.params()
        nbytes = lbm_solver_required_bytes(self.lat.h, self.p)
        self.mem = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.mem.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = lbm_solver_create(self.lat.h, self.p, self.stream.cuda_stream, aligned, nbytes)
        self.Q = self.lat.Q

    def init(self):
        lbm_solver_init(self.h)

    def init_fields(self, rho, ux=None, uy=None, T=None):
        lbm_solver_init_fields(self.h, rho, ux, uy, T)

    def step(self, n: int):
        lbm_solver_step(self.h, n)

    def sync(self):
        lbm_solver_sync(self.h)

    def get_f(self) -> np.ndarray:
        out = np.empty((self.Q, self.cfg.Ny, self.cfg.Nx), dtype=np.float64)
        return lbm_solver_get_f(self.h, out)

    def set_f(self, f: np.ndarray):
        lbm_solver_set_f(self.h, f)

    def macros(self):
        shp = (self.cfg.Ny, self.cfg.Nx)
        out = [np.empty(shp) for _ in range(4)]
        lbm_solver_macros(self.h, *out)
        return tuple(out)

    def macros_mean(self, nsteps: int):
        """Time means over the next nsteps steps of (rho, u_x, u_y, T)."""
        shp = (self.cfg.Ny, self.cfg.Nx)
        out = [np.empty(shp) for _ in range(4)]
        lbm_solver_macros_mean(self.h, nsteps, *out)
        return tuple(out)

    def fluxes(self):
        """(sigma_xx, sigma_xy, sigma_yy, q_x, q_y), each FP64 [Ny][Nx]."""
        shp = (self.cfg.Ny, self.cfg.Nx)
        out = [np.empty(shp) for _ in range(5)]
        lbm_solver_fluxes(self.h, *out)
        return tuple(out)

    def set_kernel(self, kernel: int, variant: int = 0):
        lbm_solver_set_kernel(self.h, kernel, variant)

    def kernel_info(self):
        return lbm_solver_kernel_info(self.h)

    def set_wait_limit(self, ns: int):
        lbm_solver_set_wait_limit(self.h, ns)

    def variant_count(self, kernel: int) -> int:
        return lbm_solver_variant_count(self.h, kernel)

    def autotune(self, trial_steps: int = 10):
        return lbm_solver_autotune(self.h, trial_steps)

    def wall_mass(self) -> np.ndarray:
        return lbm_solver_wall_mass(self.h, np.empty((2, self.cfg.Nx)))

    def run_to_residual(self, tol, max_steps, check_every=100):
        return lbm_solver_run_to_residual(self.h, tol, max_steps, check_every)

    def stats(self) -> lbm_stats:
        return lbm_solver_stats(self.h)

    def residual_history(self):
        """(steps, residual) arrays of the checks of the last run_to_residual."""
        return lbm_solver_residual_history(self.h)

    def get_state(self) -> bytes:
        return lbm_solver_get_state(self.h)

    def set_state(self, data: bytes):
        lbm_solver_set_state(self.h, data)

    def close(self):
        if getattr(self, "h", None):
            lbm_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
