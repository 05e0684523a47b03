"""The product path has no CPU fallback: without the built library the
binding refuses to load, and without a GPU creating a solver or a server
raises instead of computing anywhere else."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_missing_library_fails_loudly():
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1209_5201_gb300 import lbm\n"
        "lbm.LIB_PATH = '/nonexistent/liblbm_gb300.so'\n"
        "lbm._lib = None\n"
        "try:\n"
        "    lbm.load()\n"
        "except ImportError as e:\n"
        "    print('ImportError', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(1)\n" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and "not built" in out.stdout, out.stdout + out.stderr


def test_no_gpu_no_solver():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import __graft_entry__ as ge
    ge.build_library()
    from paper_1209_5201_gb300 import lbm
    lbm.load()
    with pytest.raises(Exception):
        lbm.Solver(lbm.Config(lattice="D2Q25", Nx=1, Ny=64, Kn=0.1, precision="fp64"))
    with pytest.raises(Exception):
        lbm.Server(mem_budget_bytes=1 << 20, max_slots=4)


def test_no_gpu_c_abi_reports_cuda_errors():
    # the C ABI itself, with no stream from PyTorch: an error status and no
    # handle, never a host computation
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes as C
    import __graft_entry__ as ge
    ge.build_library()
    from paper_1209_5201_gb300 import lbm
    lib = lbm.load()
    cfg = lbm.lbm_server_cfg_default()
    h = C.c_void_p()
    assert lib.lbm_server_create(C.byref(cfg), None, C.byref(h)) == lbm.LBM_ECUDA and not h.value
    lat = lbm.lbm_lattice_create(25)
    try:
        s = C.c_void_p()
        p = lbm.lbm_params_default()
        assert lib.lbm_solver_create(lat, C.byref(p), None, None, 0, C.byref(s)) == lbm.LBM_ECUDA
        assert not s.value
    finally:
        lbm.lbm_lattice_destroy(lat)
