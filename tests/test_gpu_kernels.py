"""Every step-kernel variant against the oracle and against each other.

The direct kernel and every TMA-staged variant evaluate the same arithmetic on
the same values, so their states must agree bit for bit; each must also match
the FP64 oracle (1e-12 relative per population in FP64, 1e-5 in FP32).
"""
import numpy as np
import pytest

import inputs
from gpu_util import make_pair, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    return need_gpu()


def kernels(lbm, precision):
    # (kernel, variant) pairs compiled for a precision
    s = lbm.Solver(lbm.Config(lattice="D2Q17", Nx=64, Ny=8, precision=precision))
    nd = s.variant_count(lbm.LBM_KERNEL_DIRECT)
    ns = s.variant_count(lbm.LBM_KERNEL_STAGED)
    s.close()
    return [(lbm.LBM_KERNEL_DIRECT, v) for v in range(nd)] + \
        [(lbm.LBM_KERNEL_STAGED, v) for v in range(ns)]


def run_variant(lbm, oracle, lattice, Nx, Ny, precision, kv, nsteps, **kw):
    s, p, perm = make_pair(lbm, oracle, lattice, Nx, Ny, precision=precision, **kw)
    s.set_kernel(*kv)
    rho = inputs.rho_field(Nx, Ny, 1e-3, seed=7)
    s.init_fields(rho)
    s.step(nsteps)
    s.sync()
    f = s.get_f()
    s.close()
    return f, p, perm, rho


# FP32: relative error per population after 120 steps of the 4th-order
# thermal lattice, bound 1e-5 (the FP32 tolerance; deviations d = f - w are
# stored, so round-off scales with |d|).
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_every_variant_matches_oracle_d2q37(lbm, oracle, precision, tol):
    # 300 columns: ragged against 64- and 128-column tiles; 42 rows: ragged
    # against 2- and 4-row tiles; walls move and differ in temperature
    Nx, Ny, n = 300, 42, 120
    kw = dict(Kn=0.05, u_wall=(-0.3, 0.3), T_wall=(1.02, 0.98))
    ref = None
    for kv in kernels(lbm, precision):
        f, p, perm, rho = run_variant(lbm, oracle, "D2Q37", Nx, Ny, precision, kv, n, **kw)
        if ref is None:
            fo = oracle.init_fields(p, rho)
            oracle.run(p, fo, n)
            ref = oracle.collide(p, fo)[perm]
            first = f
        assert rel_err(f, ref) < tol, kv
        assert np.array_equal(f, first), kv


@pytest.mark.parametrize("lattice", ["D2Q17", "D2Q25", "D2Q25b"])
def test_every_variant_matches_oracle_isothermal(lbm, oracle, lattice):
    Nx, Ny, n = 150, 20, 80
    ref = None
    for kv in kernels(lbm, "fp64"):
        f, p, perm, rho = run_variant(lbm, oracle, lattice, Nx, Ny, "fp64", kv, n, Kn=0.08,
                                      u_wall=(-0.1, 0.2))
        if ref is None:
            fo = oracle.init_fields(p, rho)
            oracle.run(p, fo, n)
            ref = oracle.collide(p, fo)[perm]
        assert rel_err(f, ref) < 1e-12, kv


@pytest.mark.parametrize("precision", ["bf16dev", "bf16shift"])
def test_bf16_variants_agree_bitwise(lbm, oracle, precision):
    outs = [run_variant(lbm, oracle, "D2Q37", 200, 18, precision, kv, 40, Kn=0.05,
                        u_wall=(-0.3, 0.3))[0] for kv in kernels(lbm, precision)]
    for f in outs[1:]:
        assert np.array_equal(f, outs[0])


@pytest.mark.parametrize("precision", ["fp32", "bf16dev", "bf16shift"])
@pytest.mark.parametrize("Nx,Ny", [(1, 6), (3, 7), (9, 6), (33, 6), (257, 13), (300, 8)])
def test_edge_sizes_fp32_bf16_variants_agree(lbm, oracle, precision, Nx, Ny):
    # FP32 and BF16 storage: every direct and staged variant gives the same
    # state bit for bit, on odd widths, widths below 8 (every column an image
    # column) and ragged blocks; FP32 also within 1e-5 of the oracle
    n = 25
    outs = []
    for kv in kernels(lbm, precision):
        f, p, perm, rho = run_variant(lbm, oracle, "D2Q37", Nx, Ny, precision, kv, n, Kn=0.1,
                                      u_wall=(-0.2, 0.3), T_wall=(1.05, 0.95))
        outs.append((kv, f))
    for kv, f in outs[1:]:
        assert np.array_equal(f, outs[0][1]), (kv, Nx, Ny)
    if precision == "fp32":
        fo = oracle.init_fields(p, rho)
        oracle.run(p, fo, n)
        assert rel_err(outs[0][1], oracle.collide(p, fo)[perm]) < 1e-5


@pytest.mark.parametrize("Nx,Ny", [(1, 6), (3, 7), (33, 6), (130, 9), (257, 13)])
def test_edge_sizes_all_variants(lbm, oracle, Nx, Ny):
    # minimum height (two ghost depths), widths below / around one tile, with
    # periodic images wrapping several times when Nx < 4
    n = 25
    ref = None
    for kv in kernels(lbm, "fp64"):
        f, p, perm, rho = run_variant(lbm, oracle, "D2Q37", Nx, Ny, "fp64", kv, n, Kn=0.1,
                                      u_wall=(-0.2, 0.3), T_wall=(1.05, 0.95))
        if ref is None:
            fo = oracle.init_fields(p, rho)
            oracle.run(p, fo, n)
            ref = oracle.collide(p, fo)[perm]
        assert rel_err(f, ref) < 1e-12, (kv, Nx, Ny)


def direct_kernels(lbm, precision):
    return [kv for kv in kernels(lbm, precision) if kv[0] == lbm.LBM_KERNEL_DIRECT]


# Rows of Nx + 8 > 528 elements are stored with a pitch class (1056 / 2112 /
# 4224 elements; BF16 1088 / 2112 / 4224), for which the 37-velocity step has
# instantiations with the pitch a compile-time constant; past the widest class
# (4224) a grid is stored as x-tiles of it, each with halos of its
# neighbours' columns.  700 columns: one tile of pitch 1056; 1101:
# one tile of pitch 2112; 4301: two tiles of 2151 and 2150 columns.
@pytest.mark.parametrize("precision,Nx,tol", [("fp64", 700, 1e-12), ("fp32", 1101, 1e-5),
                                              ("fp64", 4301, 1e-12), ("fp32", 4301, 1e-5)])
def test_pitch_class_grids_every_direct_variant_matches_oracle(lbm, oracle, precision, Nx, tol):
    Ny, n = 10, 30
    kw = dict(Kn=0.05, u_wall=(-0.3, 0.3), T_wall=(1.02, 0.98))
    ref = first = None
    for kv in direct_kernels(lbm, precision):
        f, p, perm, rho = run_variant(lbm, oracle, "D2Q37", Nx, Ny, precision, kv, n, **kw)
        if ref is None:
            fo = oracle.init_fields(p, rho)
            oracle.run(p, fo, n)
            ref = oracle.collide(p, fo)[perm]
            first = f
        assert rel_err(f, ref) < tol, kv
        assert np.array_equal(f, first), kv


@pytest.mark.parametrize("precision", ["bf16dev", "bf16shift"])
def test_tiled_grid_bf16_variants_agree_and_staged_is_refused(lbm, oracle, precision):
    # 4301 columns in BF16: two x-tiles of 2151 and 2150 columns (pitch 4224)
    outs = [run_variant(lbm, oracle, "D2Q37", 4301, 9, precision, kv, 20, Kn=0.05,
                        u_wall=(-0.3, 0.3))[0] for kv in direct_kernels(lbm, precision)]
    for f in outs[1:]:
        assert np.array_equal(f, outs[0])
    s = lbm.Solver(lbm.Config(lattice="D2Q37", Nx=4301, Ny=9, eq_order=4, thermal=True,
                              precision=precision))
    with pytest.raises(lbm.LBMError) as ei:
        s.set_kernel(lbm.LBM_KERNEL_STAGED, 0)
    assert ei.value.status == lbm.LBM_EINVAL
    s.close()


def test_three_tiles_other_lattice_and_accommodation(lbm, oracle):
    # D2Q17 on 8500 columns: three x-tiles (2834, 2834, 2832 columns), the
    # step with its pitch from the constants; partly specular walls, whose
    # mirrored source lies up to 6 columns away, across tile boundaries
    Nx, Ny, n = 8500, 8, 20
    accom = (0.6, 0.8)
    kw = dict(lattice="D2Q17", Nx=Nx, Ny=Ny, eq_order=2, thermal=False, Kn=0.07,
              u_wall=(-0.2, 0.15))
    p = oracle.Problem(**kw, accom=accom)
    rho = inputs.rho_field(Nx, Ny, 1e-2, seed=5)
    fo = oracle.init_fields(p, rho)
    oracle.run(p, fo, n)
    pos = {tuple(v): i for i, v in enumerate(p.lat.e.tolist())}
    first = None
    for kv in direct_kernels(lbm, "fp64"):
        s = lbm.Solver(lbm.Config(**kw, precision="fp64", accom=accom))
        s.set_kernel(*kv)
        s.init_fields(rho)
        s.step(n)
        s.sync()
        f = s.get_f()
        perm = np.array([pos[tuple(v)] for v in s.lat.e.tolist()])
        s.close()
        assert rel_err(f, oracle.collide(p, fo)[perm]) < 1e-12, kv
        if first is None:
            first = f
        assert np.array_equal(f, first), kv


def test_autotune_picks_a_compiled_kernel_and_reinitialises(lbm, oracle):
    cfg = lbm.Config(lattice="D2Q37", Nx=512, Ny=64, eq_order=4, thermal=True,
                     precision="fp32", noise_amp=1e-3)
    s = lbm.Solver(cfg)
    k, v, ms = s.autotune(5)
    assert k in (lbm.LBM_KERNEL_DIRECT, lbm.LBM_KERNEL_STAGED) and ms > 0
    assert s.kernel_info()[:2] == (k, v)
    after = s.get_f()
    t = lbm.Solver(cfg)
    t.init()
    assert np.array_equal(after, t.get_f())
    assert s.stats().steps == 0
    s.close()
    t.close()


def test_full_size_workload_sampled_columns(lbm, oracle):
    # The benchmark's workload (D2Q37 4th order, 4096 x 2048, FP32, walls -+0.3,
    # Kn 0.05) in the benchmark's launch configuration (the autotuned kernel), without the
    # density noise: the exact solution is then independent of x, so every
    # column must equal the oracle's single-column solve of the same height.
    Nx, Ny, n = 4096, 2048, 30
    cfg = lbm.Config(lattice="D2Q37", Nx=Nx, Ny=Ny, eq_order=4, thermal=True, Kn=0.05,
                     u_wall=(-0.3, 0.3), precision="fp32")
    s = lbm.Solver(cfg)
    s.autotune(5)                                  # the benchmark's kernel choice
    s.init()
    s.step(n)
    s.sync()
    _, ux, _, T = s.macros()
    cols = [0, 1, 2, 3, 127, 128, 1000, 2047, 2048, 4092, 4093, 4094, 4095]
    p = oracle.Problem(lattice="D2Q37", Nx=1, Ny=Ny, eq_order=4, thermal=True, Kn=0.05,
                       u_wall=(-0.3, 0.3))
    fo = oracle.init_fields(p, np.ones((Ny, 1)))
    oracle.run(p, fo, n)
    _, oux, _, oT = oracle.macros(p, fo)
    for c in cols:
        assert np.max(np.abs(ux[:, c] - oux[:, 0])) < 1e-5 * 0.3, c
        assert np.max(np.abs(T[:, c] - oT[:, 0])) < 1e-5, c
    # and x-independence across all columns, to FP32 round-off
    assert np.max(np.abs(ux - ux[:, :1])) < 1e-6
    st = s.stats()
    assert st.mass_drift < 1e-6
    s.close()


def test_largest_grid_the_offsets_address(lbm, oracle):
    # D2Q37 FP32 at 8192 x 6870 (two x-tiles of 4096 columns): a state buffer
    # just under 2^31 elements, so the tile offsets of the step kernel reach
    # their largest values; no density noise, so every column equals the
    # oracle's single-column solve of the same height
    Nx, Ny, n = 8192, 6870, 8
    cfg = lbm.Config(lattice="D2Q37", Nx=Nx, Ny=Ny, eq_order=4, thermal=True, Kn=0.05,
                     u_wall=(-0.3, 0.3), precision="fp32", kernel=lbm.LBM_KERNEL_DIRECT)
    s = lbm.Solver(cfg)
    s.init()
    s.step(n)
    s.sync()
    _, ux, _, T = s.macros()
    st = s.stats()
    s.close()
    p = oracle.Problem(lattice="D2Q37", Nx=1, Ny=Ny, eq_order=4, thermal=True, Kn=0.05,
                       u_wall=(-0.3, 0.3))
    fo = oracle.init_fields(p, np.ones((Ny, 1)))
    oracle.run(p, fo, n)
    _, oux, _, oT = oracle.macros(p, fo)
    for c in (0, 3, 4096, 8188, 8191):
        assert np.max(np.abs(ux[:, c] - oux[:, 0])) < 1e-5 * 0.3, c
        assert np.max(np.abs(T[:, c] - oT[:, 0])) < 1e-5, c
    assert np.max(np.abs(ux - ux[:, :1])) < 1e-6
    assert st.mass_drift < 1e-6
