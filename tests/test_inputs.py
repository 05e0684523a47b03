"""The seeded input generator against its published definition.

SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; the same generator seeds the
xoshiro family): the stream seeded with 0 starts 0xE220A8397B1DCDAF,
0x6E789E6AA1B965F4, 0x06C45D188009454F.  The counter-based draw for counter k
under seed s is the first output of the stream seeded with s XOR k, so the
stream's i-th output is the draw of seed i * 0x9E3779B97F4A7C15.  Also the
workload recipes' ranges and reproducibility."""
import math

import numpy as np

import inputs

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1
PUBLISHED_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_published_outputs():
    for i, want in enumerate(PUBLISHED_SEED0):
        got = int(inputs.splitmix64((i * GAMMA) & MASK, np.array([0], dtype=np.uint64))[0])
        assert got == want, (i, hex(got))


def test_counter_is_xored_into_the_seed():
    k = np.arange(64, dtype=np.uint64)
    a = inputs.splitmix64(0x1234, k)
    b = np.array([int(inputs.splitmix64(0x1234 ^ int(i), np.array([0], dtype=np.uint64))[0])
                  for i in range(64)], dtype=np.uint64)
    assert np.array_equal(a, b)


def test_uniform_draws_and_density_field():
    u = inputs.uniform01(7, np.arange(1 << 16, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1.0 / 12.0) < 0.005
    rho = inputs.rho_field(64, 32, 1e-3, seed=7)
    assert rho.shape == (32, 64) and np.all(np.abs(rho - 1.0) <= 1e-3)
    assert np.array_equal(rho, inputs.rho_field(64, 32, 1e-3, seed=7))
    assert not np.array_equal(rho, inputs.rho_field(64, 32, 1e-3, seed=8))
    assert np.all(inputs.rho_field(8, 8) == 1.0)


def test_serving_workload_recipe():
    reqs = inputs.serving_requests(2000, seed=11, rate=200.0)
    assert [r.arrival for r in reqs] == sorted(r.arrival for r in reqs)
    # Poisson arrivals: mean gap 1 / rate
    assert abs(reqs[-1].arrival / len(reqs) - 1.0 / 200.0) < 0.1 / 200.0
    assert all(32 <= r.Ny <= 4096 and 0.005 <= r.Kn <= 1.0 and 0.05 <= r.U_w <= 0.3 for r in reqs)
    assert {r.lattice for r in reqs} == set(inputs.LATTICES)
    # log-uniform heights: about half below the geometric mean of the range
    below = sum(r.Ny < math.sqrt(32 * 4096) for r in reqs) / len(reqs)
    assert abs(below - 0.5) < 0.05
    again = inputs.serving_requests(2000, seed=11, rate=200.0)
    assert [(r.lattice, r.Ny, r.Kn) for r in reqs] == [(r.lattice, r.Ny, r.Kn) for r in again]


def test_batched_workload_recipe():
    insts = inputs.batched_instances(256, seed=7)
    assert len(insts) == 256 and {i.lattice for i in insts} == set(inputs.LATTICES)
    assert all(32 <= i.Ny <= 2048 and 0.01 <= i.Kn <= 1.0 and 0.05 <= i.U_w <= 0.3 for i in insts)
    for i in insts:
        # the wall temperature is drawn for every instance but only the thermal
        # lattice uses it (isothermal lattices keep T_w = 1)
        if i.thermal:
            assert 0.9 <= i.T_w <= 1.1 and i.lattice == "D2Q37" and i.eq_order == 4
        else:
            assert i.T_w == 1.0 and i.eq_order == 2
    # Kn log-uniform: about half below the geometric mean of the range
    below = sum(i.Kn < 0.1 for i in insts) / len(insts)
    assert abs(below - 0.5) < 0.1
    again = inputs.batched_instances(256, seed=7)
    assert [(i.lattice, i.Ny, i.Kn, i.T_w) for i in insts] == \
        [(i.lattice, i.Ny, i.Kn, i.T_w) for i in again]
