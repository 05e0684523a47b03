"""lbm_residual_noalloc: the residual reduction that allocates nothing.

Some callers cannot allocate device memory at the moment they need the
steady-state residual: code running while a stream is captured into a CUDA
graph, hosts whose device memory is owned by another allocator or capped by a
budget, frameworks that forbid libraries from allocating on their own.  This
test checks, through the C ABI, that the no-allocation call returns the same
residual as the solver's own check (lbm_solver_run_to_residual, which uses
scratch memory the solver allocated) on two calls in a row, and that it
copies the current fields into the previous-check arrays as the solver does.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
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
