"""Failure detection of the staged kernel without a GPU fault.

Every mbarrier wait of the TMA-staged step kernel is bounded; when a wait runs
out the kernel records a device flag, its CTAs stop taking tiles and each
producer waits for its copies in flight before exiting, and the host reports
LBM_ETIMEOUT.  A zero limit (lbm_solver_set_wait_limit) makes every wait give
up at once, so the path runs on demand: the step returns the error, the flag is
cleared, and the solver, given back a state and the default limit, steps
exactly like the FP64 oracle again.  Nothing here faults or hangs: the expiry
path only returns.
"""
import numpy as np
import pytest

from gpu_util import make_pair, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    return need_gpu()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16dev"])
def test_staged_wait_limit_expiry_reports_timeout_and_the_solver_recovers(lbm, oracle, precision):
    s, p, perm = make_pair(lbm, oracle, "D2Q17", 70, 12, precision=precision, Kn=0.08,
                           u_wall=(-0.1, 0.15))
    s.set_kernel(lbm.LBM_KERNEL_STAGED, 0)
    rng = np.random.default_rng(2)
    shp = (p.Ny, p.Nx)
    f = oracle.init_fields(p, 1 + 0.01 * rng.random(shp), 0.04 * rng.random(shp) - 0.02)
    start = oracle.collide(p, f)[perm]
    s.set_f(start)
    s.set_wait_limit(0)
    s.step(3)
    with pytest.raises(lbm.LBMError) as ei:
        s.sync()
    assert ei.value.status == lbm.LBM_ETIMEOUT
    s.sync()                                  # the flag was cleared
    # back to the default limit: a reloaded state steps like the oracle
    s.set_wait_limit(2_000_000_000)
    s.set_f(start)
    s.step(5)
    s.sync()
    oracle.run(p, f, 5)
    tol = {"fp64": 1e-12, "fp32": 1e-5, "bf16dev": 5e-2}[precision]
    assert rel_err(s.get_f(), oracle.collide(p, f)[perm]) < tol
    s.close()
