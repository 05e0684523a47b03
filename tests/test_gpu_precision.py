"""Precision sweep on the single-column D2Q25 Couette (Nx = 1, Ny = 64, walls
-+0.1, Kn = 0.1): FP64, FP32 (deviations from the rest weights) and BF16
deviation storage, each run to its steady-state tolerance (1e-8 FP64, 1e-6
otherwise), against the FP64 oracle's steady state (residual 1e-10).
L-inf errors in rho, u_x / U_w and the kinetic temperature, with the
one-thread-per-cell kernel and with the one-warp-per-cell kernel (the
automatic choice on a grid this small), of the final state and of the time
mean over the next 4000 steps (lbm_solver_macros_mean)."""
import numpy as np
import pytest

from gpu_util import need_gpu, report

pytestmark = pytest.mark.gpu

# BF16 keeps 8 significant bits of d = f - w rho (|d| up to ~0.3 w here).
# With round-to-nearest the steady state carried that round-off as a bias
# amplified by the relaxation time (4.4e-2 U_w in u_x); the step kernels
# round stochastically, so the steady state carries zero-mean noise instead:
# over two random streams and both kernels, measured 3.7e-3 .. 5.3e-3 U_w in
# u_x, 2.5e-4 .. 6.6e-4 in rho, 1.3e-4 .. 2.3e-4 in T for the final state
# (bounds 1.5x the largest); the noise keeps the residual near 4e-3, so the
# 1e-6 target is not reached (ENOTCONVERGED is expected: the noise floor).
# The time mean over 4000 steps is the steady field to within the bound of
# the BF16 variant, 5e-3 in u_x / U_w and in rho.
# BF16SHIFT keeps 8 significant bits of d = f - w (the FP32 format's
# deviations; here rho stays within 1e-3 of 1, so |d| is about that of
# BF16DEV) with the same stochastic rounding and no density plane: measured
# on both kernels 2.3e-3 .. 2.5e-3 U_w in u_x, 4.4e-4 .. 4.5e-4 in rho,
# 1.4e-4 .. 1.5e-4 in T for the final state (bounds 2x the largest, one
# random stream measured), residual noise near 2.6e-3, and the time mean
# within 3.4e-4 in rho and u_x / U_w and 2.6e-6 in T (bounds 1e-3, 1e-3, 1e-5).
BOUNDS = {          # rho, u_x / U_w, T
    "fp64": (1e-9, 1e-7, 1e-9),
    "fp32": (2e-6, 5e-6, 2e-6),
    "bf16dev": (1e-3, 8e-3, 4e-4),
    "bf16shift": (9e-4, 5e-3, 3e-4),
}
MEAN_BOUNDS = {
    "fp64": (1e-9, 1e-7, 1e-9),
    "fp32": (2e-6, 5e-6, 2e-6),
    "bf16dev": (5e-3, 5e-3, 4e-4),
    "bf16shift": (1e-3, 1e-3, 1e-5),
}
KERNELS = {"thread": 1, "warp": 3}
TOL = {"fp64": 1e-8, "fp32": 1e-6, "bf16dev": 1e-6, "bf16shift": 1e-6}


def sweep(lbm, oracle, kernel):
    Uw = 0.1
    p = oracle.Problem(lattice="D2Q25", Nx=1, Ny=64, Kn=0.1, u_wall=(-Uw, Uw))
    f = oracle.init_fields(p, np.ones((64, 1)))
    ok, _, _ = oracle.run_to_residual(p, f, 1e-10, 2_000_000, 100)
    assert ok
    # the GPU stores the post-collision state; an isothermal collision does not
    # conserve energy, so the kinetic T is compared on the collided oracle state
    orho, oux, _, oT = oracle.macros_kinetic(p, oracle.collide(p, f))
    out = {}
    for prec in ("fp64", "fp32", "bf16dev", "bf16shift"):
        s = lbm.Solver(lbm.Config(lattice="D2Q25", Nx=1, Ny=64, Kn=0.1, u_wall=(-Uw, Uw),
                                  precision=prec, kernel=kernel))
        s.init()
        st, steps, res = s.run_to_residual(TOL[prec], 2_000_000, 100)
        rho, ux, uy, T = s.macros()
        mrho, mux, _, mT = s.macros_mean(4000)
        out[prec] = dict(status=st, steps=steps, res=res,
                         err_rho=float(np.max(np.abs(rho - orho))),
                         err_u=float(np.max(np.abs(ux - oux)) / Uw),
                         err_T=float(np.max(np.abs(T - oT))),
                         mean_err_rho=float(np.max(np.abs(mrho - orho))),
                         mean_err_u=float(np.max(np.abs(mux - oux)) / Uw),
                         mean_err_T=float(np.max(np.abs(mT - oT))))
        s.close()
    return out


@pytest.fixture(scope="module")
def lbm_mod():
    return need_gpu()


@pytest.mark.parametrize("kname", sorted(KERNELS))
def test_precision_sweep_against_oracle_steady_state(lbm_mod, oracle, kname):
    res = sweep(lbm_mod, oracle, KERNELS[kname])
    report("precision_sweep" + ("" if kname == "thread" else "_cellwarp"), res)
    for prec, r in res.items():
        b, m = BOUNDS[prec], MEAN_BOUNDS[prec]
        assert r["err_rho"] < b[0] and r["err_u"] < b[1] and r["err_T"] < b[2], (prec, r)
        assert r["mean_err_rho"] < m[0] and r["mean_err_u"] < m[1] and r["mean_err_T"] < m[2], \
            (prec, r)
    assert res["fp64"]["status"] == lbm_mod.LBM_OK and res["fp32"]["status"] == lbm_mod.LBM_OK
