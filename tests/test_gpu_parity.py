"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

The GPU stores the post-collision state f~*; the oracle advances the
pre-collision state f~ in the paper's collide-then-stream order.  After n
steps from f~*(0) = C(f~(0)) the two agree as f~*_gpu(n) = C(f~_oracle(n)),
C the oracle's collision.  FP64 tolerance: 1e-12 relative per population.
"""
import numpy as np
import pytest

import inputs
from gpu_util import make_pair, need_gpu, rel_err, report

pytestmark = pytest.mark.gpu

LATTICES = ["D2Q17", "D2Q25", "D2Q25b", "D2Q37"]


@pytest.fixture(scope="module")
def lbm():
    return need_gpu()


def _nonequilibrium_state(p, orc, seed):
    rng = np.random.default_rng(seed)
    shp = (p.Ny, p.Nx)
    f = orc.init_fields(p, 1 + 0.02 * rng.random(shp), 0.1 * rng.random(shp) - 0.05,
                        0.1 * rng.random(shp) - 0.05,
                        1 + (0.04 * rng.random(shp) - 0.02 if p.thermal else 0.0))
    f *= 1 + 0.05 * rng.random(f.shape)
    return f


@pytest.mark.parametrize("lattice", LATTICES)
@pytest.mark.parametrize("nsteps", [1, 37])
def test_fp64_steps_from_nonequilibrium_state(lbm, oracle, lattice, nsteps):
    # ragged small grid: 7 columns (< one block), 9 rows (wall rows overlap)
    s, p, perm = make_pair(lbm, oracle, lattice, 7, 9, u_wall=(-0.2, 0.15),
                           T_wall=(1.03, 0.97), Kn=0.07)
    f = _nonequilibrium_state(p, oracle, 11)
    s.set_f(oracle.collide(p, f)[perm])
    s.step(nsteps)
    oracle.run(p, f, nsteps)
    err = rel_err(s.get_f(), oracle.collide(p, f)[perm])
    s.close()
    assert err < 1e-12, err


def test_fp64_couette_d2q25_1x64(lbm, oracle):
    # isothermal Couette, D2Q25 order 2, Nx=1 x Ny=64, walls -+0.1, Kn=0.1, FP64
    s, p, perm = make_pair(lbm, oracle, "D2Q25", 1, 64, Kn=0.1, u_wall=(-0.1, 0.1))
    rho = np.ones((64, 1))
    s.init_fields(rho)
    f = oracle.init_fields(p, rho)
    done = 0
    for target in (1000, 20000):
        s.step(target - done)
        oracle.run(p, f, target - done)
        done = target
        err = rel_err(s.get_f(), oracle.collide(p, f)[perm])
        assert err < 1e-12, (target, err)
    s.close()


# FP32: relative error per population on the 4th-order thermal lattice, bound
# 1e-5 after 200 and after 1000 steps (the FP32 tolerance of the config-2
# domain).  The FP32 store holds deviations d = f - w, theta = T - 1 is formed
# without cancellation against D and 1 - omega is never formed, so the
# round-off per step scales with |d|, not with f; measured 3.9e-6 at 1000
# steps.
@pytest.mark.parametrize("precision,n,tol", [("fp64", 1000, 1e-12), ("fp32", 200, 1e-5),
                                             ("fp32", 1000, 1e-5)])
def test_d2q37_thermal_grid_multi_block(lbm, oracle, precision, n, tol):
    # 300 columns = 2 full 128-column blocks + a ragged 44, 40 rows, noise on rho
    Nx, Ny = 300, 40
    s, p, perm = make_pair(lbm, oracle, "D2Q37", Nx, Ny, precision=precision, Kn=0.05,
                           u_wall=(-0.3, 0.3), T_wall=(1.02, 0.98))
    rho = inputs.rho_field(Nx, Ny, 1e-3, seed=7)
    s.init_fields(rho)
    f = oracle.init_fields(p, rho)
    s.step(n)
    oracle.run(p, f, n)
    err = rel_err(s.get_f(), oracle.collide(p, f)[perm])
    s.close()
    report(f"parity_grid_d2q37_{precision}_{n}", {"max_rel_err_per_population": err, "steps": n})
    assert err < tol, err


@pytest.mark.parametrize("lattice", ["D2Q17", "D2Q25", "D2Q37"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16dev", "bf16shift"])
def test_init_from_seed_matches_input_generator(lbm, oracle, lattice, precision):
    # the device SplitMix64 initialisation equals the input module's draw
    Nx, Ny = 33, 8
    o, t = (4, True) if lattice == "D2Q37" else (2, False)
    cfg = lbm.Config(lattice=lattice, Nx=Nx, Ny=Ny, eq_order=o, thermal=t,
                     precision=precision, noise_amp=1e-3, seed=7)
    rho = inputs.rho_field(Nx, Ny, 1e-3, seed=7)
    s1 = lbm.Solver(cfg)
    s1.init()
    s2 = lbm.Solver(cfg)
    s2.init_fields(rho)
    f1, f2 = s1.get_f(), s2.get_f()
    assert np.array_equal(f1, f2)
    # and it is the oracle's equilibrium of that density field
    p = oracle.Problem(lattice=lattice, Nx=Nx, Ny=Ny, eq_order=o, thermal=t)
    pos = {tuple(v): i for i, v in enumerate(p.lat.e.tolist())}
    perm = [pos[tuple(v)] for v in s1.lat.e.tolist()]
    fo = oracle.init_fields(p, rho)[perm]
    # BF16SHIFT holds d = f - w = w (rho - 1) at rest, rounded to nearest in
    # BF16 (half an ulp, between 2^-9 and 2^-8 of |d|): with |rho - 1| <= 1e-3,
    # at most 3.91e-6 relative to f (measured 3.4e-6); BF16DEV's d = f - w rho
    # is zero at rest
    tol = {"fp64": 1e-15, "fp32": 2e-7, "bf16dev": 2e-7, "bf16shift": 4e-6}[precision]
    assert rel_err(f1, fo) < tol
    s1.close()
    s2.close()


@pytest.mark.parametrize("lattice", ["D2Q17", "D2Q25", "D2Q37"])
def test_wall_incoming_mass(lbm, oracle, lattice):
    # numerator of Eq. (12): the GPU's per-column M_in of the current state summed
    # over columns equals the oracle's incoming mass of its next step
    s, p, perm = make_pair(lbm, oracle, lattice, 11, 10, u_wall=(-0.25, 0.2),
                           T_wall=(1.05, 0.96), Kn=0.04)
    f = _nonequilibrium_state(p, oracle, 3)
    s.set_f(oracle.collide(p, f)[perm])
    s.step(5)
    oracle.run(p, f, 5)
    m = s.wall_mass()
    st = oracle.run(p, f.copy(), 1, stats=True)
    for wall in (0, 1):
        assert abs(m[wall].sum() - st["m_in"][wall]) < 1e-13 * st["m_in"][wall]
    assert np.all(m > 0)
    s.close()


def test_mass_conservation_and_stats(lbm, oracle):
    s, p, perm = make_pair(lbm, oracle, "D2Q25", 4, 16, Kn=0.1)
    s.init_fields(inputs.rho_field(4, 16, 1e-3, seed=7))
    s.step(4000)
    st = s.stats()
    assert st.steps == 4000
    assert st.mass_drift < 1e-13
    assert st.wall_in[0] > 0 and st.wall_in[1] > 0
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16dev", "bf16shift"])
def test_checkpoint_resume_is_bitwise(lbm, oracle, precision):
    s, p, perm = make_pair(lbm, oracle, "D2Q37", 40, 12, precision=precision, Kn=0.05,
                           u_wall=(-0.3, 0.3))
    s.init_fields(inputs.rho_field(40, 12, 1e-3, seed=5))
    s.step(30)
    ck = s.get_state()
    s.step(20)
    a = s.get_f()
    s.set_state(ck)
    s.step(20)
    b = s.get_f()
    assert np.array_equal(a, b)
    t = lbm.Solver(s.cfg)
    t.set_state(ck)
    t.step(20)
    assert np.array_equal(a, t.get_f())
    assert t.stats().steps == 50
    s.close()
    t.close()


def test_macros_match_oracle(lbm, oracle):
    s, p, perm = make_pair(lbm, oracle, "D2Q37", 19, 8, u_wall=(-0.3, 0.3), T_wall=(1.1, 0.9))
    f = _nonequilibrium_state(p, oracle, 9)
    s.set_f(oracle.collide(p, f)[perm])
    rho, ux, uy, T = s.macros()
    orho, oux, ouy, oT = oracle.macros(p, f)
    assert np.max(np.abs(rho - orho)) < 1e-14
    assert np.max(np.abs(ux - oux)) < 1e-14 and np.max(np.abs(uy - ouy)) < 1e-14
    assert np.max(np.abs(T - oT)) < 1e-13
    s.close()


def test_steady_state_residual_driver(lbm, oracle):
    # the precision sweep's FP64 leg: D2Q25 Couette to res <= 1e-10, against the
    # oracle's steady state
    s, p, perm = make_pair(lbm, oracle, "D2Q25", 1, 64, Kn=0.1)
    s.init_fields(np.ones((64, 1)))
    st, steps, res = s.run_to_residual(1e-10, 400000, 100)
    assert st == lbm.LBM_OK and res <= 1e-10
    f = oracle.init_fields(p, np.ones((64, 1)))
    ok, osteps, ores = oracle.run_to_residual(p, f, 1e-10, 400000, 100)
    assert ok and abs(osteps - steps) <= 100
    _, ux, _, _ = s.macros()
    assert np.max(np.abs(ux - oracle.macros(p, f)[1])) / 0.1 < 1e-11
    s.close()


def test_residual_driver_reports_nonconvergence_and_nan(lbm, oracle):
    s, p, perm = make_pair(lbm, oracle, "D2Q17", 1, 32, Kn=0.05)
    s.init_fields(np.ones((32, 1)))
    st, steps, res = s.run_to_residual(1e-14, 300, 100)
    assert st == lbm.LBM_ENOTCONVERGED and steps == 300
    # one (steps, residual) record per check; the middle one against the
    # oracle's driver stopped at that check
    hs, hr = s.residual_history()
    assert list(hs) == [100, 200, 300] and hr[-1] == res
    f = oracle.init_fields(p, np.ones((32, 1)))
    ok, osteps, ores = oracle.run_to_residual(p, f, 0.0, 200, 100)
    assert not ok and osteps == 200 and abs(hr[1] - ores) <= 1e-8 * ores
    f = s.get_f()
    f[3, 5, 0] = np.nan                     # poisoned state, injected on the host
    s.set_f(f)
    with pytest.raises(lbm.LBMError) as ei:
        s.run_to_residual(1e-8, 1000, 100)
    assert ei.value.status == lbm.LBM_ENONFINITE
    s.close()
