"""Helpers shared by the GPU tests: build both sides of a comparison."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build_library()
    from paper_1209_5201_gb300 import lbm
    lbm.load()
    return lbm


def order_for(lattice):
    return (4, True) if lattice == "D2Q37" else (2, False)


def make_pair(lbm, orc, lattice, Nx, Ny, precision="fp64", Kn=0.05, u_wall=(-0.1, 0.1),
              T_wall=(1.0, 1.0), eq_order=None, thermal=None, kernel=0, tau=0.0):
    o, t = order_for(lattice)
    eq_order = o if eq_order is None else eq_order
    thermal = t if thermal is None else thermal
    cfg = lbm.Config(lattice=lattice, Nx=Nx, Ny=Ny, eq_order=eq_order, thermal=thermal, Kn=Kn,
                     tau=tau, u_wall=u_wall, T_wall=T_wall, precision=precision, kernel=kernel)
    s = lbm.Solver(cfg)
    p = orc.Problem(lattice=lattice, Nx=Nx, Ny=Ny, eq_order=eq_order, thermal=thermal, Kn=Kn,
                    tau=tau, u_wall=u_wall, T_wall=T_wall)
    pos = {tuple(v): i for i, v in enumerate(p.lat.e.tolist())}
    perm = np.array([pos[tuple(v)] for v in s.lat.e.tolist()])
    return s, p, perm


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def report(name, data):
    """Write measured numbers to $LBM_REPORT_DIR/<name>.json when set."""
    import json
    import os
    d = os.environ.get("LBM_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, name + ".json"), "w") as fh:
            json.dump(data, fh, indent=1, default=float)
