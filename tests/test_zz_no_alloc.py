"""lbm_residual_noalloc: the residual reduction that allocates nothing.

Some callers cannot allocate device memory at the moment they need the
steady-state residual: code running while a stream is captured into a CUDA
graph, hosts whose device memory is owned by another allocator or capped by a
budget, frameworks that forbid libraries from allocating on their own.  This
test checks, through the C ABI, that the no-allocation call returns the same
residual as the solver's own check (lbm_solver_run_to_residual, which uses
scratch memory the solver allocated) on two calls in a row, and that it
copies the current fields into the previous-check arrays as the solver does;
that it works when captured into a CUDA graph after one call outside the
capture (the graph case is why the call exists); and that it follows the
current CUDA context: a second context, which holds its own copy of the
scratch array at another address, gets that address, not the first one's.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_solver_check_twice():
    lbm = need_gpu()
    import torch

    cfg = lbm.Config(lattice="D2Q37", Nx=37, Ny=24, eq_order=4, thermal=True, Kn=0.05,
                     u_wall=(-0.3, 0.3), T_wall=(1.02, 0.98), precision="fp64",
                     noise_amp=1e-3, seed=7)
    s = lbm.Solver(cfg)
    s.init()
    n = cfg.Nx * cfg.Ny
    T_ref = 0.5 * (cfg.T_wall[0] + cfg.T_wall[1])
    _, ux0, _, T0 = s.macros()
    dev = torch.device("cuda")
    prev_u = torch.tensor(ux0.ravel(), dtype=torch.float64, device=dev)
    prev_T = torch.tensor(T0.ravel(), dtype=torch.float64, device=dev)
    res_d = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    K = 50
    for call in range(2):
        # the solver's own residual over one check of K steps (tol 0: never met)
        status, steps, res_solver = s.run_to_residual(0.0, K, K)
        assert status == lbm.LBM_ENOTCONVERGED and steps == K
        _, ux, _, T = s.macros()
        u_d = torch.tensor(ux.ravel(), dtype=torch.float64, device=dev)
        T_d = torch.tensor(T.ravel(), dtype=torch.float64, device=dev)
        lbm.lbm_residual_noalloc(u_d, T_d, prev_u, prev_T, n, T_ref, True, res_d, stream)
        torch.cuda.synchronize()
        res_noalloc = float(res_d.item())
        assert res_solver > 0
        assert abs(res_noalloc - res_solver) <= 1e-12 * res_solver, (call, res_noalloc, res_solver)
        assert torch.equal(prev_u, u_d) and torch.equal(prev_T, T_d)
    s.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    lbm = need_gpu()
    import torch

    a = torch.zeros(8, dtype=torch.float64, device="cuda")
    for n in (0, 2 ** 31):
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_residual_noalloc(a, a, a, a, n, 1.0, False, a)
        assert ei.value.status == lbm.LBM_EINVAL
    # a small isothermal call still works after the rejections
    u = torch.arange(1, 9, dtype=torch.float64, device="cuda")
    up = torch.zeros(8, dtype=torch.float64, device="cuda")
    T = torch.ones(8, dtype=torch.float64, device="cuda")
    Tp = torch.ones(8, dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    lbm.lbm_residual_noalloc(u, T, up, Tp, 8, 1.0, False, out)
    torch.cuda.synchronize()
    assert abs(out.item() - 1.0) < 1e-15          # ||u - 0|| / ||u||
    assert np.array_equal(up.cpu().numpy(), u.cpu().numpy())


def test_noalloc_residual_captured_in_a_cuda_graph():
    # one call outside the capture (it looks up the scratch address), then the
    # call captured into a graph and replayed after two rounds of solver
    # steps: each replay returns the solver's own residual and updates the
    # previous-check arrays
    lbm = need_gpu()
    import torch

    cfg = lbm.Config(lattice="D2Q25", Nx=20, Ny=16, Kn=0.1, u_wall=(-0.1, 0.1),
                     precision="fp64", noise_amp=1e-3, seed=3)
    s = lbm.Solver(cfg)
    s.init()
    n = cfg.Nx * cfg.Ny
    dev = torch.device("cuda")
    _, ux0, _, T0 = s.macros()
    prev_u = torch.tensor(ux0.ravel(), dtype=torch.float64, device=dev)
    prev_T = torch.tensor(T0.ravel(), dtype=torch.float64, device=dev)
    u_d = torch.empty(n, dtype=torch.float64, device=dev)
    T_d = torch.empty(n, dtype=torch.float64, device=dev)
    res_d = torch.zeros(1, dtype=torch.float64, device=dev)
    K = 40

    def solver_round():
        status, steps, res_solver = s.run_to_residual(0.0, K, K)
        assert status == lbm.LBM_ENOTCONVERGED and steps == K
        _, ux, _, T = s.macros()
        u_d.copy_(torch.from_numpy(ux.ravel()))
        T_d.copy_(torch.from_numpy(T.ravel()))
        torch.cuda.synchronize()
        return res_solver

    res_solver = solver_round()
    lbm.lbm_residual_noalloc(u_d, T_d, prev_u, prev_T, n, 1.0, False, res_d,
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert abs(res_d.item() - res_solver) <= 1e-12 * res_solver
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lbm.lbm_residual_noalloc(u_d, T_d, prev_u, prev_T, n, 1.0, False, res_d,
                                 torch.cuda.current_stream().cuda_stream)
    for rnd in range(2):
        res_solver = solver_round()
        res_d.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert res_solver > 0
        assert abs(res_d.item() - res_solver) <= 1e-12 * res_solver, (rnd, res_d.item(), res_solver)
        assert torch.equal(prev_u, u_d) and torch.equal(prev_T, T_d)
    s.close()


# Child process: the call in torch's (primary) context, then in a second
# context created with the driver API and made current (device buffers from
# cuMemAlloc there), then in the primary context again; prints the three
# residuals and the one numpy computes from the same inputs.
_CONTEXT_CHILD = r"""
import ctypes as C, json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1209_5201_gb300 import lbm
lbm.load()
n = 96
rng = np.random.default_rng(5)
u = 0.5 + rng.random(n); up = rng.random(n)
T = 1.0 + 0.1 * rng.random(n); Tp = 1.0 + 0.1 * rng.random(n)
expect = max(np.linalg.norm(u - up) / np.linalg.norm(u),
             np.linalg.norm(T - Tp) / np.linalg.norm(T - 1.0))

def in_torch():
    d = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (u, T, up, Tp)]
    r = torch.zeros(1, dtype=torch.float64, device="cuda")
    lbm.lbm_residual_noalloc(d[0], d[1], d[2], d[3], n, 1.0, True, r)
    torch.cuda.synchronize()
    return r.item()

def ok(rc, what):
    if rc != 0:
        raise SystemExit(f"{what} failed: {rc}")

r_primary = in_torch()
cu = C.CDLL("libcuda.so.1")
ok(cu.cuInit(0), "cuInit")
dev = C.c_int()
ok(cu.cuDeviceGet(C.byref(dev), 0), "cuDeviceGet")
ctx = C.c_void_p()
ok(cu.cuCtxCreate_v4(C.byref(ctx), None, C.c_uint(0), dev), "cuCtxCreate")
bufs = []
for a in (u, T, up, Tp, np.zeros(1)):
    p = C.c_uint64()
    ok(cu.cuMemAlloc_v2(C.byref(p), C.c_size_t(a.nbytes)), "cuMemAlloc")
    ok(cu.cuMemcpyHtoD_v2(p, a.ctypes.data_as(C.c_void_p), C.c_size_t(a.nbytes)), "HtoD")
    bufs.append(p.value)
lbm.lbm_residual_noalloc(bufs[0], bufs[1], bufs[2], bufs[3], n, 1.0, True, bufs[4])
ok(cu.cuCtxSynchronize(), "cuCtxSynchronize")
out = np.zeros(1)
ok(cu.cuMemcpyDtoH_v2(out.ctypes.data_as(C.c_void_p), C.c_uint64(bufs[4]), C.c_size_t(8)), "DtoH")
for p in bufs:
    ok(cu.cuMemFree_v2(C.c_uint64(p)), "cuMemFree")
popped = C.c_void_p()
ok(cu.cuCtxPopCurrent_v2(C.byref(popped)), "cuCtxPopCurrent")
ok(cu.cuCtxDestroy_v2(ctx), "cuCtxDestroy")
r_again = in_torch()
print(json.dumps([r_primary, float(out[0]), r_again, float(expect)]))
"""


def test_noalloc_follows_the_current_context():
    # a context other than the one of the first call holds the scratch array
    # at its own address; the call there looks that address up (the cache is
    # keyed by the context's unique ID) and gives the same residual
    need_gpu()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, "-c", _CONTEXT_CHILD, root], capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    r_primary, r_other, r_again, expect = json.loads(p.stdout.strip().splitlines()[-1])
    for r in (r_primary, r_other, r_again):
        assert abs(r - expect) <= 1e-13 * expect, (r_primary, r_other, r_again, expect)
