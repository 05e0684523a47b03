"""Grid-convergence study of Sec. IV on the GPU (FP64, through the C ABI).

Thermal Couette at Kn = 0.01, walls at -+0.2 and T_w = 1, on the 2-D thermal
lattice (D2Q37, 4th-order equilibrium); the paper runs N_G = 20, 50, 100, 200,
500, 1000 with N_G = 1000 as the reference and reports E_U and E_T (the two
relative L2 errors defined after Fig. 5) falling at second order.  The coarse
grid N_G = 20 is also checked against the oracle's steady state.
"""
import math

import numpy as np
import pytest

from gpu_util import need_gpu, report

pytestmark = pytest.mark.gpu

KN, UW = 0.01, 0.2
GRIDS = (20, 50, 100, 200, 500)
REF = 1000


@pytest.fixture(scope="module")
def lbm():
    return need_gpu()


def _steady(lbm, Ny):
    s = lbm.Solver(lbm.Config(lattice="D2Q37", Nx=1, Ny=Ny, eq_order=4, thermal=True, Kn=KN,
                              u_wall=(-UW, UW), precision="fp64"))
    s.init()
    st, steps, res = s.run_to_residual(1e-12, 3_000_000, 500)
    assert st == lbm.LBM_OK, (Ny, steps, res)
    _, ux, _, T = s.macros()
    s.close()
    return steps, res, ux[:, 0], T[:, 0]


def test_second_order_convergence_and_coarse_grid_parity(lbm, oracle):
    sols = {Ny: _steady(lbm, Ny) for Ny in GRIDS + (REF,)}
    yf = (np.arange(REF) + 0.5) / REF
    _, _, uf, Tf = sols[REF]
    EU, ET = [], []
    for Ny in GRIDS:
        y = (np.arange(Ny) + 0.5) / Ny
        _, _, u, T = sols[Ny]
        ur, Tr = np.interp(y, yf, uf), np.interp(y, yf, Tf)
        EU.append(math.sqrt(np.sum((u - ur) ** 2) / np.sum(ur ** 2)))
        ET.append(math.sqrt(np.sum((T - Tr) ** 2) / np.sum((Tr - 1.0) ** 2)))
    lg = np.log(GRIDS[:4])
    sU = np.polyfit(lg, np.log(EU[:4]), 1)[0]
    sT = np.polyfit(lg, np.log(ET[:4]), 1)[0]
    report("convergence_study", {"N_G": list(GRIDS), "reference": REF, "E_U": EU, "E_T": ET,
                                 "order_U": -sU, "order_T": -sT,
                                 "steps": {Ny: sols[Ny][0] for Ny in GRIDS + (REF,)}})
    assert -2.4 < sU < -1.6, (EU, sU)
    assert -2.4 < sT < -1.6, (ET, sT)
    # the coarsest grid against the oracle's steady state of the same problem
    p = oracle.Problem(lattice="D2Q37", Nx=1, Ny=20, eq_order=4, thermal=True, Kn=KN,
                       u_wall=(-UW, UW))
    f = oracle.init_fields(p, np.ones((20, 1)))
    ok, _, _ = oracle.run_to_residual(p, f, 1e-13, 3_000_000, 500)
    assert ok
    _, ou, _, oT = oracle.macros(p, f)
    _, _, u, T = sols[20]
    assert np.max(np.abs(u - ou[:, 0])) / UW < 1e-9
    assert np.max(np.abs(T - oT[:, 0])) < 1e-10
