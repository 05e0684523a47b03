"""Stress and heat flux read-out (Sec. II conversion of f~) on the GPU, through
the C ABI, against the oracle's orc_fluxes on the same state.

The GPU starts from a post-collision f~* = rho g^eq and the oracle from the same
values taken as pre-collision f~ (a fixed point of the collision), so the GPU
state after n steps is the oracle's state after n steps, collided.
lbm_solver_fluxes pulls it (streaming + wall fill) to the next pre-collision
f~: the oracle's state after n + 1 steps.
"""
import numpy as np
import pytest

import inputs
from gpu_util import need_gpu, order_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    return need_gpu()


def _close(g, o, rel):
    scale = max(np.max(np.abs(o)), 1e-300)
    return float(np.max(np.abs(g - o)) / scale) <= rel


@pytest.mark.parametrize("lattice,Nx,Ny,accom", [
    ("D2Q37", 300, 14, (1.0, 1.0)),      # several 128-column blocks and a ragged tail
    ("D2Q25", 1, 10, (1.0, 0.4)),        # single periodic column, partial accommodation
    ("D2Q17", 7, 12, (0.0, 1.0)),        # narrow width, specular bottom wall
])
def test_fp64_fluxes_match_oracle(lbm, oracle, lattice, Nx, Ny, accom):
    o, t = order_for(lattice)
    kw = dict(lattice=lattice, Nx=Nx, Ny=Ny, eq_order=o, thermal=t, Kn=0.07,
              u_wall=(-0.2, 0.25), T_wall=(1.04, 0.97))
    p = oracle.Problem(**kw, accom=accom)
    rho = inputs.rho_field(Nx, Ny, 1e-2, seed=4)
    fo = oracle.init_fields(p, rho)
    oracle.run(p, fo, 31)
    ref = oracle.fluxes(p, fo)
    s = lbm.Solver(lbm.Config(**kw, precision="fp64", accom=accom))
    s.init_fields(rho)
    s.step(30)
    got = s.fluxes()
    s.close()
    for name, g, r in zip(("sxx", "sxy", "syy", "qx", "qy"), got, ref):
        assert _close(g, r, 1e-10), (name, float(np.max(np.abs(g - r))), float(np.max(np.abs(r))))


@pytest.mark.parametrize("precision,rel", [("fp32", 2e-3), ("bf16dev", 0.1), ("bf16shift", 0.1)])
def test_reduced_precision_steady_shear_stress(lbm, oracle, precision, rel):
    # steady isothermal Couette: the uniform bulk shear stress against the
    # oracle's steady state (the FP32 / BF16 round-off floors of the state)
    Ny, Kn, Uw = 40, 0.05, 0.1
    p = oracle.Problem(lattice="D2Q25", Nx=1, Ny=Ny, eq_order=2, thermal=False, Kn=Kn,
                       u_wall=(-Uw, Uw))
    fo = oracle.init_fields(p, np.ones((Ny, 1)))
    ok, _, _ = oracle.run_to_residual(p, fo, 1e-12, 800000, 100)
    assert ok
    ref = oracle.fluxes(p, fo)[1][:, 0]
    s = lbm.Solver(lbm.Config(lattice="D2Q25", Nx=1, Ny=Ny, eq_order=2, thermal=False, Kn=Kn,
                              u_wall=(-Uw, Uw), precision=precision))
    s.init()
    s.step(20000)
    sxy = s.fluxes()[1][:, 0]
    s.close()
    mid = slice(Ny // 4, 3 * Ny // 4)
    assert np.max(np.abs(sxy[mid] - ref[mid])) < rel * np.max(np.abs(ref)), \
        (float(np.max(np.abs(sxy[mid] - ref[mid]))), float(np.max(np.abs(ref))))
