"""Partially accommodating and specular walls (the paper's general scattering
kernel, Sec. III Eq. (9)-(10), as R = a R_D + (1 - a) R_S) on the GPU, against
the oracle: every step-kernel variant in FP64 and the batched path in FP32."""
import numpy as np
import pytest

import inputs
from gpu_util import need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    return need_gpu()


def variants(lbm):
    s = lbm.Solver(lbm.Config(lattice="D2Q17", Nx=64, Ny=8))
    nd, ns = s.variant_count(lbm.LBM_KERNEL_DIRECT), s.variant_count(lbm.LBM_KERNEL_STAGED)
    s.close()
    return [(1, v) for v in range(nd)] + [(2, v) for v in range(ns)]


@pytest.mark.parametrize("lattice,Nx,Ny,accom", [
    ("D2Q37", 150, 14, (0.0, 0.6)),     # the specular source shifts by up to 6 columns
    ("D2Q25", 5, 10, (0.3, 1.0)),       # and wraps around a narrow periodic width
    ("D2Q17", 1, 12, (0.5, 0.0)),
])
def test_variants_match_oracle(lbm, oracle, lattice, Nx, Ny, accom):
    o, t = (4, True) if lattice == "D2Q37" else (2, False)
    kw = dict(lattice=lattice, Nx=Nx, Ny=Ny, eq_order=o, thermal=t, Kn=0.06,
              u_wall=(-0.2, 0.25), T_wall=(1.04, 0.97))
    p = oracle.Problem(**kw, accom=accom)
    rho = inputs.rho_field(Nx, Ny, 1e-2, seed=3)
    fo = oracle.init_fields(p, rho)
    oracle.run(p, fo, 40)
    ref = oracle.collide(p, fo)
    for kv in variants(lbm):
        s = lbm.Solver(lbm.Config(**kw, precision="fp64", accom=accom))
        s.set_kernel(*kv)
        s.init_fields(rho)
        s.step(40)
        pos = {tuple(v): i for i, v in enumerate(p.lat.e.tolist())}
        perm = [pos[tuple(v)] for v in s.lat.e.tolist()]
        err = rel_err(s.get_f(), ref[perm])
        s.close()
        assert err < 1e-12, (kv, err)


def test_fp32_specular_walls_keep_the_gas_at_rest(lbm):
    # fully specular walls transmit no tangential momentum: u stays ~0
    s = lbm.Solver(lbm.Config(lattice="D2Q37", Nx=64, Ny=32, eq_order=4, thermal=True, Kn=0.05,
                              u_wall=(-0.3, 0.3), precision="fp32", accom=(0.0, 0.0)))
    s.init()
    s.step(500)
    _, ux, _, _ = s.macros()
    s.close()
    assert np.max(np.abs(ux)) < 1e-6


def test_batched_partial_accommodation_steady_state(lbm, oracle):
    cases = [("D2Q25", 40, 0.1, 0.1, (0.5, 0.5)), ("D2Q37", 24, 0.2, 0.2, (0.7, 0.4))]
    srv = lbm.Server(mem_budget_bytes=1 << 26, max_slots=4, chunk_steps=50)
    ids = [srv.submit(lbm.make_request(lat, Ny, Kn, Uw, tol=1e-6, accom=acc))
           for lat, Ny, Kn, Uw, acc in cases]
    srv.drain(300)
    res = {r.id: r for r in srv.poll(8)}
    for rid, (lat, Ny, Kn, Uw, acc) in zip(ids, cases):
        assert res[rid].status == lbm.LBM_OK
        _, ux, _, T = srv.fetch(rid, Ny)
        o, t = (4, True) if lat == "D2Q37" else (2, False)
        p = oracle.Problem(lattice=lat, Nx=1, Ny=Ny, eq_order=o, thermal=t, Kn=Kn,
                           u_wall=(-Uw, Uw), accom=acc)
        f = oracle.init_fields(p, np.ones((Ny, 1)))
        ok, _, _ = oracle.run_to_residual(p, f, 1e-13, 2_000_000, 100)
        assert ok
        oux = oracle.macros(p, f)[1][:, 0]
        assert np.max(np.abs(ux - oux)) / Uw < 1e-5, (lat, acc)
    srv.close()
