"""Solver options beyond the default closure, on the GPU against the oracle:
constant relaxation time, a viscosity law mu = T^mu_exp other than mu = T
(Sec. II: tau may depend on the local temperature), the third-order and the
isothermal fourth-order truncations of Eq. (4).  FP64 single-domain kernels
(every direct and staged variant) and the FP32 batched path."""
import numpy as np
import pytest

import inputs
from gpu_util import need_gpu, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "constant tau": dict(lattice="D2Q25", eq_order=2, thermal=False, Kn=0.0, tau=0.02),
    "mu = T^0.7": dict(lattice="D2Q37", eq_order=4, thermal=True, Kn=0.06, mu_exp=0.7),
    "third order": dict(lattice="D2Q37", eq_order=3, thermal=True, Kn=0.06),
    "isothermal fourth order": dict(lattice="D2Q37", eq_order=4, thermal=False, Kn=0.06),
}


@pytest.fixture(scope="module")
def lbm():
    return need_gpu()


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_kernels_match_oracle(lbm, oracle, name):
    c = CASES[name]
    Nx, Ny = 70, 13
    kw = dict(c, Nx=Nx, Ny=Ny, u_wall=(-0.2, 0.15), T_wall=(1.03, 0.98))
    p = oracle.Problem(**kw)
    rho = inputs.rho_field(Nx, Ny, 1e-2, seed=5)
    fo = oracle.init_fields(p, rho)
    oracle.run(p, fo, 30)
    ref = oracle.collide(p, fo)
    probe = lbm.Solver(lbm.Config(**kw, precision="fp64"))
    nd, ns = probe.variant_count(lbm.LBM_KERNEL_DIRECT), probe.variant_count(lbm.LBM_KERNEL_STAGED)
    probe.close()
    for kv in [(1, v) for v in range(nd)] + [(2, v) for v in range(ns)]:
        s = lbm.Solver(lbm.Config(**kw, precision="fp64"))
        s.set_kernel(*kv)
        s.init_fields(rho)
        s.step(30)
        pos = {tuple(v): i for i, v in enumerate(p.lat.e.tolist())}
        perm = [pos[tuple(v)] for v in s.lat.e.tolist()]
        err = rel_err(s.get_f(), ref[perm])
        s.close()
        assert err < 1e-12, (name, kv, err)


@pytest.mark.parametrize("name", sorted(CASES))
def test_batched_path_follows_the_oracle(lbm, oracle, name):
    c = CASES[name]
    Ny, Uw, steps = 40, 0.15, 600
    req = lbm.make_request(c["lattice"], Ny, c["Kn"] or 0.05, Uw, 1.0, tol=1e-30, max_steps=steps,
                           eq_order=c["eq_order"], thermal=c["thermal"], tau=c.get("tau", 0.0))
    req.mu_exp = c.get("mu_exp", 1.0)
    if c.get("tau", 0.0) > 0:
        req.Kn = 0.0
    s = lbm.Server(mem_budget_bytes=1 << 26, max_slots=4, chunk_steps=50)
    rid = s.submit(req)
    s.drain(120)
    r = s.poll(4)[0]
    _, ux, _, T = s.fetch(rid, Ny)
    s.close()
    p = oracle.Problem(lattice=c["lattice"], Nx=1, Ny=Ny, eq_order=c["eq_order"],
                       thermal=c["thermal"], Kn=c["Kn"], tau=c.get("tau", 0.0),
                       mu_exp=c.get("mu_exp", 1.0), u_wall=(-Uw, Uw))
    f = oracle.init_fields(p, np.ones((Ny, 1)))
    oracle.run(p, f, r.steps)
    _, oux, _, oT = oracle.macros(p, f)
    assert np.max(np.abs(ux - oux[:, 0])) / Uw < 1e-5, (name, r.steps)
    if c["thermal"]:
        assert np.max(np.abs(T - oT[:, 0])) < 1e-5, name


def test_custom_lattice_runs_like_the_built_in_one(lbm, oracle):
    # the D2Q25 velocity set with the weights and scale of the other root,
    # given as tables in a shuffled order: the same steps as the built-in D2Q25b
    ref = lbm.Lattice("D2Q25b")
    perm = np.random.default_rng(8).permutation(ref.Q)
    cus = lbm.Lattice("custom", custom=(ref.e[perm], ref.w[perm], ref.r))
    kw = dict(lattice="D2Q25b", Nx=9, Ny=16, Kn=0.08, u_wall=(-0.1, 0.1), precision="fp64")
    rho = inputs.rho_field(9, 16, 1e-2, seed=2)
    out = []
    for lat in (None, cus):
        s = lbm.Solver(lbm.Config(**kw), lattice=lat)
        s.init_fields(rho)
        s.step(50)
        out.append(s.get_f())
        s.close()
    assert np.array_equal(out[0], out[1])
    p = oracle.Problem(lattice="D2Q25b", Nx=9, Ny=16, Kn=0.08, u_wall=(-0.1, 0.1))
    f = oracle.init_fields(p, rho)
    oracle.run(p, f, 50)
    pos = {tuple(v): i for i, v in enumerate(p.lat.e.tolist())}
    perm_o = [pos[tuple(v)] for v in ref.e.tolist()]
    assert rel_err(out[1], oracle.collide(p, f)[perm_o]) < 1e-12
