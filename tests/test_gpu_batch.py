"""Batched chunk kernel and continuous-batching server, through the C ABI.

Accuracy: each steady profile against the FP64 oracle's steady state of the
same single-column problem (L-inf of u_x / U_w, and of T - 1 when thermal).
Independence: a request's result is the same bit for bit alone and in a mix
(each slot's arithmetic does not depend on the other slots, and checks fall on
the same step counts).
"""
import time

import numpy as np
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

MIX = [("D2Q17", 24, 0.2, 0.10, 1.0), ("D2Q25", 40, 0.1, 0.20, 1.0),
       ("D2Q37", 32, 0.3, 0.30, 1.05), ("D2Q17", 64, 0.5, 0.05, 1.0),
       ("D2Q25", 16, 1.0, 0.15, 1.0), ("D2Q37", 20, 0.08, 0.25, 0.95),
       ("D2Q25b", 30, 0.2, 0.10, 1.0), ("D2Q37", 48, 0.5, 0.12, 1.0)]


@pytest.fixture(scope="module")
def lbm():
    return need_gpu()


def oracle_steady(oracle, lat, Ny, Kn, Uw, Tw):
    o, t = (4, True) if lat == "D2Q37" else (2, False)
    p = oracle.Problem(lattice=lat, Nx=1, Ny=Ny, eq_order=o, thermal=t, Kn=Kn,
                       u_wall=(-Uw, Uw), T_wall=(Tw, Tw))
    f = oracle.init_fields(p, np.ones((Ny, 1)))
    ok, _, _ = oracle.run_to_residual(p, f, 1e-13, 2_000_000, 100)
    assert ok
    _, ux, _, T = oracle.macros(p, f)
    return ux[:, 0], T[:, 0]


def solve(lbm, items, tol=1e-6, **srv):
    s = lbm.Server(**{**dict(mem_budget_bytes=1 << 28, max_slots=16, chunk_steps=50), **srv})
    ids = [s.submit(lbm.make_request(lat, Ny, Kn, Uw, Tw, tol=tol, tag=i))
           for i, (lat, Ny, Kn, Uw, Tw) in enumerate(items)]
    s.drain(300)
    res = {r.id: r for r in s.poll(len(items))}
    out = []
    for rid, (lat, Ny, Kn, Uw, Tw) in zip(ids, items):
        r = res[rid]
        rho, ux, uy, T = s.fetch(rid, Ny)
        out.append((r, rho, ux, T))
    st = s.stats()
    s.close()
    return out, st


def test_batch_matches_oracle_steady_states(lbm, oracle):
    out, st = solve(lbm, MIX)
    assert st.completed == len(MIX)
    for (lat, Ny, Kn, Uw, Tw), (r, rho, ux, T) in zip(MIX, out):
        assert r.status == lbm.LBM_OK, (lat, Ny, r.status, r.residual)
        oux, oT = oracle_steady(oracle, lat, Ny, Kn, Uw, Tw)
        err_u = np.max(np.abs(ux - oux)) / Uw
        assert err_u < 1e-5, (lat, Ny, Kn, err_u)
        if lat == "D2Q37":
            assert np.max(np.abs(T - oT)) < 1e-5, (lat, Ny)
        assert abs(r.mass - Ny) < 1e-5 * Ny          # rho = 1 start, wall conserves mass
        assert np.max(np.abs(ux + ux[::-1])) < 1e-5 * Uw * 10


# Tall columns and rarefied or dense ones, where the slowest relaxation time
# is long: with round-to-nearest FP32 stores and a collision that did not
# conserve mass and momentum exactly in FP32, the steady state moved by up to
# 1.5e-4 U_w (the same round-off at every step, amplified by that time); the
# batched kernel's stochastic rounding and conserving increments bring every
# one within the 1e-5 bound.
TALL = [("D2Q37", 300, 0.5, 0.20, 1.0), ("D2Q25", 700, 0.8, 0.10, 1.0),
        ("D2Q17", 1500, 1.0, 0.15, 1.0), ("D2Q37", 1100, 0.6, 0.25, 1.05),
        ("D2Q25", 120, 0.01, 0.30, 1.0), ("D2Q17", 700, 0.01, 0.20, 1.0)]
# Long requests (small Kn): the server splits them over clusters of 2, 4 and
# 8 CTAs while CTAs are spare; the 2500-row one has more rows per CTA than fit
# shared memory (its state stays in global memory).
LONG = [("D2Q37", 300, 0.004, 0.20, 1.0), ("D2Q25", 700, 0.004, 0.10, 1.0),
        ("D2Q17", 1500, 0.004, 0.15, 1.0), ("D2Q37", 1100, 0.004, 0.25, 1.05),
        ("D2Q17", 2500, 0.004, 0.15, 1.0)]


def fixed_steps(lbm, items, steps, rounding=0, **srv):
    """Run every item for `steps` steps (rounded up to whole chunks)."""
    s = lbm.Server(**{**dict(mem_budget_bytes=1 << 28, max_slots=32, chunk_steps=50), **srv})
    ids = [s.submit(lbm.make_request(lat, Ny, Kn, Uw, Tw, tol=1e-30, max_steps=steps,
                                     rounding=rounding))
           for lat, Ny, Kn, Uw, Tw in items]
    s.drain(300)
    res = {r.id: r for r in s.poll(64)}
    out = [(res[i], *s.fetch(i, it[1])) for i, it in zip(ids, items)]
    s.close()
    return out


@pytest.mark.parametrize("rounding,bound_T", [(1, 1e-5), (2, 2e-5)])
def test_cluster_slots_follow_the_oracle_transient(lbm, oracle, rounding, bound_T):
    # a fixed number of steps (no convergence stop): every row of the state,
    # including the rows next to the cluster's CTA boundaries, against the
    # oracle after the same steps.  With stochastic rounding and conserving
    # increments (rounding 1) within 1e-5 in u_x / U_w and T; rounded to
    # nearest throughout (rounding 2), the FP32 transient's T drifts further
    # (measured 1.2e-5 after 1500 steps of the 300-row D2Q37 column at Kn
    # 0.004), bound 2e-5 for T
    for (lat, Ny, Kn, Uw, Tw), (r, rho, ux, uy, T) in zip(
            LONG, fixed_steps(lbm, LONG, 1500, rounding=rounding)):
        o, t = (4, True) if lat == "D2Q37" else (2, False)
        p = oracle.Problem(lattice=lat, Nx=1, Ny=Ny, eq_order=o, thermal=t, Kn=Kn,
                           u_wall=(-Uw, Uw), T_wall=(Tw, Tw))
        f = oracle.init_fields(p, np.ones((Ny, 1)))
        oracle.run(p, f, r.steps)
        _, oux, _, oT = oracle.macros(p, f)
        assert np.max(np.abs(ux - oux[:, 0])) / Uw < 1e-5, (lat, Ny, r.steps)
        if t:
            assert np.max(np.abs(T - oT[:, 0])) < bound_T, (lat, Ny)


@pytest.mark.parametrize("how", ["no clusters", "one CTA of budget"])
def test_result_does_not_depend_on_the_split(lbm, how):
    # the same long requests split over clusters (default) and on one CTA each:
    # the same steps, residual and fields, bit for bit
    kw = dict(cluster_rows=8192) if how == "no clusters" else dict(max_slots=1)
    items = LONG[1:4] + LONG[4:]
    split = fixed_steps(lbm, items, 2000)
    whole = [fixed_steps(lbm, [it], 2000, **kw)[0] for it in items] if how != "no clusters" \
        else fixed_steps(lbm, items, 2000, **kw)
    for it, a, b in zip(items, split, whole):
        assert a[0].steps == b[0].steps and a[0].residual == b[0].residual, it
        for x, y in zip(a[1:], b[1:]):
            assert np.array_equal(x, y), it


def test_tall_columns_match_oracle_steady_states(lbm, oracle):
    items = TALL + MIX[:2]
    out, st = solve(lbm, items)
    assert st.completed == len(items)
    for (lat, Ny, Kn, Uw, Tw), (r, rho, ux, T) in zip(items, out):
        assert r.status == lbm.LBM_OK, (lat, Ny, r.status, r.residual)
        oux, oT = oracle_steady(oracle, lat, Ny, Kn, Uw, Tw)
        err_u = np.max(np.abs(ux - oux)) / Uw
        assert err_u < 1e-5, (lat, Ny, Kn, err_u)
        if lat == "D2Q37":
            assert np.max(np.abs(T - oT)) < 1e-5, (lat, Ny)
        assert abs(r.mass - Ny) < 1e-5 * Ny


def test_cluster_slot_is_the_same_alone_and_in_the_mix(lbm):
    items = LONG[:4] + MIX
    mixed = fixed_steps(lbm, items, 1500)
    for k in (0, 2, 3):
        alone = fixed_steps(lbm, [items[k]], 1500)[0]
        assert alone[0].steps == mixed[k][0].steps
        assert np.array_equal(alone[2], mixed[k][2]) and np.array_equal(alone[4], mixed[k][4])


def test_cta_budget_admits_a_tall_column_behind_short_ones(lbm):
    # budget of 8 CTAs, short requests ahead of and behind a long tall one:
    # with others waiting the tall one runs on one CTA and is admitted in order
    s = lbm.Server(mem_budget_bytes=1 << 28, max_slots=8, chunk_steps=50)
    short = [s.submit(lbm.make_request("D2Q17", 24, 0.5, 0.1, tol=1e-6)) for _ in range(4)]
    tall = s.submit(lbm.make_request("D2Q17", 1500, 1.0, 0.1, tol=1e-6))
    more = [s.submit(lbm.make_request("D2Q17", 24, 0.5, 0.1, tol=1e-6)) for _ in range(12)]
    s.drain(300)
    res = {r.id: r for r in s.poll(32)}
    assert all(res[i].status == lbm.LBM_OK for i in short + [tall] + more)
    assert res[tall].t_admit < max(res[i].t_admit for i in more)
    s.close()


def test_result_is_the_same_alone_and_in_the_mix(lbm):
    mixed, _ = solve(lbm, MIX)
    for k in (0, 2, 5):
        alone, _ = solve(lbm, [MIX[k]])
        a, b = alone[0], mixed[k]
        assert a[0].steps == b[0].steps
        assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def test_admission_under_a_small_memory_budget(lbm):
    items = [("D2Q37", 64, 0.3, 0.1, 1.0)] * 5
    one = lbm.lbm_request_bytes(lbm.make_request("D2Q37", 64, 0.3, 0.1))
    s = lbm.Server(mem_budget_bytes=2 * one + 100, max_slots=8, chunk_steps=50)
    ids = [s.submit(lbm.make_request(*it, tol=1e-6)) for it in items]
    peak = 0
    t0 = time.time()
    while s.stats().completed < len(items) and time.time() - t0 < 120:
        m = s.stats()
        peak = max(peak, m.running)
        assert m.pool_used_bytes <= m.pool_bytes
        time.sleep(0.001)
    s.drain(120)
    assert s.stats().completed == 5 and peak <= 2
    res = s.poll(10)
    assert all(r.status == lbm.LBM_OK for r in res)
    assert len({(r.steps) for r in res}) == 1          # identical problems, identical work
    # a request larger than the whole budget is refused at once
    with pytest.raises(lbm.LBMError) as ei:
        s.submit(lbm.make_request("D2Q37", 4096, 0.1, 0.1))
    assert ei.value.status == lbm.LBM_EBUDGET
    s.close()


def test_requests_admitted_while_others_run(lbm):
    # the long column takes a 4-CTA cluster, the short ones share the other 4
    s = lbm.Server(mem_budget_bytes=1 << 26, max_slots=8, chunk_steps=50)
    long_id = s.submit(lbm.make_request("D2Q37", 1024, 0.005, 0.2, tol=1e-6))
    time.sleep(0.05)
    short = [s.submit(lbm.make_request("D2Q17", 24, 0.5, 0.1, tol=1e-6)) for _ in range(6)]
    s.drain(300)
    res = {r.id: r for r in s.poll(16)}
    assert all(res[i].status == lbm.LBM_OK for i in [long_id] + short)
    # the short requests overtake the long one that arrived first
    assert max(res[i].t_done for i in short) < res[long_id].t_done
    st = s.stats()
    assert st.p99_latency_s >= st.p50_latency_s > 0 and st.solves_per_s > 0
    s.close()


def test_invalid_requests_are_refused(lbm):
    s = lbm.Server(mem_budget_bytes=1 << 24, max_slots=2, chunk_steps=20)
    bad = lbm.make_request("D2Q25", 32, float("nan"), 0.1)
    with pytest.raises(lbm.LBMError) as ei:
        s.submit(bad)
    assert ei.value.status == lbm.LBM_EINVAL
    ok = s.submit(lbm.make_request("D2Q25", 32, 0.2, 0.1, tol=1e-6))
    s.drain(60)
    assert s.poll(4)[0].id == ok
    s.close()


def test_batch_solve_entry_point(lbm):
    reqs = [lbm.make_request(lat, Ny, Kn, Uw, Tw, tol=1e-6, tag=i)
            for i, (lat, Ny, Kn, Uw, Tw) in enumerate(MIX[:4])]
    cfg = lbm.lbm_server_cfg_default()
    cfg.mem_budget_bytes, cfg.max_slots, cfg.chunk_steps = 1 << 26, 4, 50
    out = lbm.lbm_batch_solve(cfg, reqs)
    assert [r.tag for r in out] == [0, 1, 2, 3]
    assert all(r.status == lbm.LBM_OK and r.steps > 0 for r in out)


def test_graph_and_plain_launches_agree(lbm):
    # the chunk launches replayed as a CUDA graph and issued one by one give
    # the same results, bit for bit (clusters included)
    items = LONG[:2] + MIX[:4]
    a = fixed_steps(lbm, items, 1200)
    b = fixed_steps(lbm, items, 1200, use_graph=False)
    for it, x, y in zip(items, a, b):
        assert x[0].steps == y[0].steps and x[0].residual == y[0].residual, it
        assert all(np.array_equal(u, v) for u, v in zip(x[1:], y[1:])), it


@pytest.mark.parametrize("Ny", [257, 300, 511, 513, 1023, 1025, 1100, 2047, 2049, 2431, 2432,
                                2500, 4095, 4096, 4097, 8192])
def test_split_at_class_boundaries(lbm, Ny):
    # heights around every cluster-size boundary, up to the largest: the rows
    # split over 2, 4, 8 or 16 CTAs (shared memory or global memory) step
    # exactly like one CTA holding them all
    item = [("D2Q17", Ny, 0.002, 0.1, 1.0)]
    split = fixed_steps(lbm, item, 300, max_slots=16)[0]
    whole = fixed_steps(lbm, item, 300, max_slots=16, cluster_rows=8192)[0]
    assert split[0].steps == whole[0].steps and split[0].residual == whole[0].residual
    for x, y in zip(split[1:], whole[1:]):
        assert np.array_equal(x, y)
    assert abs(np.sum(split[1]) - Ny) < 1e-3 * Ny          # rho: the walls conserve mass


def test_running_request_promoted_to_a_cluster(lbm):
    # 16 CTAs of budget filled at once by 15 short requests (3000 steps each)
    # and a long one, which therefore starts on one CTA; once the short ones
    # are done the server moves it to a cluster (its state stays in place),
    # and its result equals that of a run on one CTA throughout, bit for bit
    item = ("D2Q37", 1024, 0.01, 0.1, 1.0)
    s = lbm.Server(mem_budget_bytes=1 << 28, max_slots=16, chunk_steps=50)
    for _ in range(15):
        s.submit(lbm.make_request("D2Q17", 24, 0.5, 0.1, tol=1e-30, max_steps=3000))
    rid = s.submit(lbm.make_request(*item, tol=1e-30, max_steps=20000))
    s.drain(300)
    promoted = s.stats().promoted
    r = {x.id: x for x in s.poll(64)}[rid]
    fields = s.fetch(rid, item[1])
    s.close()
    assert promoted >= 1
    whole = fixed_steps(lbm, [item], 20000, max_slots=16, cluster_rows=8192)[0]
    assert r.steps == whole[0].steps and r.residual == whole[0].residual
    for x, y in zip(fields, whole[1:]):
        assert np.array_equal(x, y)


def test_cluster_shrinks_for_queued_requests(lbm):
    # a long request alone on 16 CTAs of budget gets a 4-CTA cluster; 15
    # requests arriving later need 3 of its CTAs, so it shrinks to one CTA
    # and grows again once they are done; its result is that of a run on one
    # CTA throughout, bit for bit
    item = ("D2Q37", 1024, 0.01, 0.1, 1.0)
    s = lbm.Server(mem_budget_bytes=1 << 28, max_slots=16, chunk_steps=50)
    rid = s.submit(lbm.make_request(*item, tol=1e-30, max_steps=100000))
    time.sleep(0.05)
    for _ in range(15):
        s.submit(lbm.make_request("D2Q17", 24, 0.5, 0.1, tol=1e-30, max_steps=3000))
    s.drain(300)
    st = s.stats()
    r = {x.id: x for x in s.poll(64)}[rid]
    fields = s.fetch(rid, item[1])
    s.close()
    assert st.demoted >= 1 and st.promoted >= 1 and st.completed == 16
    whole = fixed_steps(lbm, [item], 100000, max_slots=16, cluster_rows=8192)[0]
    assert r.steps == whole[0].steps and r.residual == whole[0].residual
    for x, y in zip(fields, whole[1:]):
        assert np.array_equal(x, y)


def test_cancel_running_and_queued_requests(lbm):
    # one CTA of budget: a long request runs, a second waits in the queue;
    # cancelling the queued one drops it, cancelling the running one stops it
    # at the end of its chunk with the fields where it stopped
    # the running request cannot finish first: tol 1e-30 is below the FP32
    # floor, and its slowest mode alone takes ~1.6e5 steps per e-folding
    s = lbm.Server(mem_budget_bytes=1 << 26, max_slots=1, chunk_steps=50)
    run = s.submit(lbm.make_request("D2Q37", 1024, 0.001, 0.1, tol=1e-30, max_steps=10**9))
    wait = s.submit(lbm.make_request("D2Q17", 24, 0.5, 0.1, tol=1e-6))
    time.sleep(0.2)
    s.cancel(wait)
    s.cancel(run)
    with pytest.raises(lbm.LBMError):
        s.cancel(12345)                               # no such request
    s.drain(60)
    res = {r.id: r for r in s.poll(8)}
    assert res[wait].status == lbm.LBM_ECANCELLED and res[wait].steps == 0
    assert res[run].status == lbm.LBM_ECANCELLED and res[run].steps > 0
    rho, ux, _, _ = s.fetch(run, 1024)
    assert abs(np.sum(rho) - 1024) < 1e-2 and np.max(np.abs(ux)) > 0
    rho_w, _, _, _ = s.fetch(wait, 24)
    assert not np.any(rho_w)
    # the server keeps serving
    ok = s.submit(lbm.make_request("D2Q17", 24, 0.5, 0.1, tol=1e-6))
    s.drain(60)
    assert s.poll(4)[0].status == lbm.LBM_OK
    s.close()


def test_autotune_fills_the_configuration_and_leaves_results_unchanged(lbm):
    # the batched-path autotuner times lone columns on every usable cluster
    # size and full-GPU batches at several chunk lengths, and writes its
    # choices into the configuration; a server with the tuned cluster rows and
    # chunks per launch gives the same results, bit for bit, as one with the
    # built-in rules and the same chunk length
    import torch
    cfg = lbm.lbm_server_cfg_default()
    cfg.mem_budget_bytes = 1 << 28
    cfg.max_slots = 2 * torch.cuda.get_device_properties(0).multi_processor_count
    rep = lbm.lbm_server_autotune(cfg)
    assert cfg.chunk_steps in (25, 50, 100, 200, 400)
    assert 32 <= cfg.cluster_rows <= 1024 and cfg.cluster_rows % 32 == 0
    assert cfg.class_sub[0] == 1 and all(0 <= v <= 16 for v in cfg.class_sub)
    assert cfg.class_sub[1] >= 1 and cfg.class_sub[3] >= 1          # 2- and 8-CTA clusters
    for li in range(3):
        for hi in range(3):
            assert rep["lone_us"][li][hi][0] > 0                    # one CTA always usable
    assert all(g > 0 for g in rep["chunk_glups"]) and rep["seconds"] > 0
    # results do not depend on the tuned cluster rows or chunks per launch
    tuned = lbm.Server(cfg=cfg)
    base = lbm.lbm_server_cfg_default()
    base.mem_budget_bytes, base.max_slots, base.chunk_steps = 1 << 28, cfg.max_slots, cfg.chunk_steps
    plain = lbm.Server(cfg=base)
    items = LONG[1:4] + MIX[:3]
    out = []
    for s in (tuned, plain):
        ids = [s.submit(lbm.make_request(lat, Ny, Kn, Uw, Tw, tol=1e-30, max_steps=3000))
               for lat, Ny, Kn, Uw, Tw in items]
        s.drain(300)
        res = {r.id: r for r in s.poll(64)}
        out.append([(res[i].steps, res[i].residual, *s.fetch(i, it[1])) for i, it in zip(ids, items)])
        s.close()
    for it, a, b in zip(items, *out):
        assert a[0] == b[0] and a[1] == b[1], it
        assert all(np.array_equal(x, y) for x, y in zip(a[2:], b[2:])), it


def test_ns_start_reaches_the_same_steady_state_in_fewer_steps(lbm, oracle):
    # a request may start from the Navier-Stokes slip solution of the paper's
    # Couette problem instead of rest: the same steady state (within 1e-5 of
    # the oracle's, which starts from rest) in fewer steps for dense columns
    items = [("D2Q25", 400, 0.01, 0.20, 1.0), ("D2Q37", 300, 0.02, 0.25, 1.05),
             ("D2Q17", 200, 0.1, 0.15, 1.0)]
    steps = {}
    for init in (lbm.LBM_INIT_REST, lbm.LBM_INIT_NS):
        s = lbm.Server(mem_budget_bytes=1 << 28, max_slots=16, chunk_steps=50)
        ids = [s.submit(lbm.make_request(lat, Ny, Kn, Uw, Tw, tol=5e-6, init=init))
               for lat, Ny, Kn, Uw, Tw in items]
        s.drain(300)
        res = {r.id: r for r in s.poll(8)}
        for rid, (lat, Ny, Kn, Uw, Tw) in zip(ids, items):
            r = res[rid]
            assert r.status == lbm.LBM_OK, (init, lat, Ny)
            _, ux, _, T = s.fetch(rid, Ny)
            oux, oT = oracle_steady(oracle, lat, Ny, Kn, Uw, Tw)
            assert np.max(np.abs(ux - oux)) / Uw < 1e-5, (init, lat, Ny)
            if lat == "D2Q37":
                assert np.max(np.abs(T - oT)) < 1e-5, (init, lat, Ny)
            assert abs(r.mass - Ny) < 1e-5 * Ny
            steps[(init, lat)] = r.steps
        s.close()
    for lat in ("D2Q25", "D2Q37"):                  # the dense ones
        assert steps[(lbm.LBM_INIT_NS, lat)] < 0.8 * steps[(lbm.LBM_INIT_REST, lat)], steps
