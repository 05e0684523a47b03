"""The one-warp-per-cell step kernel (LBM_KERNEL_CELLWARP) against the oracle:
widths below, at and above the 7 ghost columns a wall row sums, every lattice,
moving walls of different temperatures, partial and specular accommodation,
FP64 / FP32 / BF16 storage; and the automatic choice of it on small grids."""
import numpy as np
import pytest

import inputs
from gpu_util import need_gpu, order_for, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    return need_gpu()


def run(lbm, oracle, lattice, Nx, Ny, precision, nsteps, accom=(1.0, 1.0), kernel=3):
    o, t = order_for(lattice)
    kw = dict(lattice=lattice, Nx=Nx, Ny=Ny, eq_order=o, thermal=t, Kn=0.07,
              u_wall=(-0.2, 0.25), T_wall=(1.04, 0.97))
    p = oracle.Problem(**kw, accom=accom)
    rho = inputs.rho_field(Nx, Ny, 1e-2, seed=6)
    fo = oracle.init_fields(p, rho)
    oracle.run(p, fo, nsteps)
    ref = oracle.collide(p, fo)
    s = lbm.Solver(lbm.Config(**kw, precision=precision, accom=accom, kernel=kernel))
    s.init_fields(rho)
    s.step(nsteps)
    pos = {tuple(v): i for i, v in enumerate(p.lat.e.tolist())}
    perm = [pos[tuple(v)] for v in s.lat.e.tolist()]
    f = s.get_f()
    info = s.kernel_info()
    s.close()
    return rel_err(f, ref[perm]), info


@pytest.mark.parametrize("lattice", ["D2Q17", "D2Q25", "D2Q25b", "D2Q37"])
@pytest.mark.parametrize("Nx,Ny", [(1, 6), (3, 11), (9, 14), (40, 7)])
def test_fp64_matches_oracle(lbm, oracle, lattice, Nx, Ny):
    err, _ = run(lbm, oracle, lattice, Nx, Ny, "fp64", 40)
    assert err < 1e-12, (lattice, Nx, Ny, err)


@pytest.mark.parametrize("accom", [(0.0, 0.6), (0.3, 1.0)])
def test_fp64_accommodation(lbm, oracle, accom):
    err, _ = run(lbm, oracle, "D2Q37", 5, 12, "fp64", 40, accom=accom)
    assert err < 1e-12, err


# FP32 and BF16 storage against the FP64 oracle after 40 steps.  FP32: the
# bound of the one-thread kernels (1e-5).  BF16 keeps 8 significant bits of
# d = f - w rho (BF16SHIFT: d = f - w) and the step kernels round it
# stochastically: each store errs
# by up to one BF16 ulp (2^-7 of |d|, zero-mean), and over 40 steps the errors
# add like a random walk; measured 7.7e-3 relative per population, bound 1.5e-2.
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16dev", 1.5e-2),
                                           ("bf16shift", 1.5e-2)])
def test_reduced_precision(lbm, oracle, precision, tol):
    err, _ = run(lbm, oracle, "D2Q37", 9, 14, precision, 40)
    assert err < tol, (precision, err)


def test_auto_picks_it_on_small_grids_only(lbm, oracle):
    _, small = run(lbm, oracle, "D2Q25", 1, 64, "fp64", 5, kernel=0)
    assert small[0] == lbm.LBM_KERNEL_CELLWARP
    _, big = run(lbm, oracle, "D2Q25", 80, 64, "fp64", 5, kernel=0)
    assert big[0] == lbm.LBM_KERNEL_DIRECT
