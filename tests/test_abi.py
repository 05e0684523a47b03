"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/lbm.h declares, and its host-side parts (lattice solver, parameter
checks, memory sizing) agree with the oracle and the paper."""
import os
import re

import numpy as np
import pytest

from oracle import lattice as olat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    import __graft_entry__ as ge
    ge.build_library()
    from paper_1209_5201_gb300 import lbm as m
    m.load()
    return m


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_\w+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lbm):
    lib = lbm.load()
    names = declared_symbols()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_symbol(lbm):
    for n in declared_symbols():
        assert hasattr(lbm, n), n


@pytest.mark.parametrize("name,kind", [("D2Q17", 17), ("D2Q25", 25), ("D2Q25b", 26),
                                       ("D2Q37", 37)])
def test_library_lattice_matches_oracle(lbm, name, kind):
    # two independent derivations: the oracle's Newton / closed form in numpy and
    # the library's determinant root search in long double
    h = lbm.lbm_lattice_create(kind)
    try:
        Q, r, N, deg = lbm.lbm_lattice_info(h)
        e, w = lbm.lbm_lattice_tables(h)
        ol = olat.get(name)
        assert Q == ol.Q and N == 3
        # the oracle solves in float64, the library in long double: 1e-14 relative
        assert abs(r - ol.r) < 1e-14 * r
        ow = {tuple(v): x for v, x in zip(ol.e.tolist(), ol.w)}
        assert set(map(tuple, e.tolist())) == set(ow)
        for v, x in zip(e.tolist(), w):
            assert abs(x - ow[tuple(v)]) < 1e-14 * x
        assert lbm.lbm_lattice_verify(h, deg) < 1e-12
        assert lbm.lbm_lattice_verify(h, deg + 1) > 1e-3
    finally:
        lbm.lbm_lattice_destroy(h)


@pytest.mark.parametrize("kind", [17, 25, 37])
def test_library_velocity_order_is_paired(lbm, kind):
    # rest first, then opposite pairs (kernels share even/odd equilibrium parts)
    h = lbm.lbm_lattice_create(kind)
    e, w = lbm.lbm_lattice_tables(h)
    lbm.lbm_lattice_destroy(h)
    assert tuple(e[0]) == (0, 0)
    for a in range(1, len(e), 2):
        assert tuple(e[a + 1]) == tuple(-e[a])
        assert w[a] == w[a + 1]
    assert np.abs(e[:, 1]).max() == 3


def test_params_default_and_checks(lbm):
    p = lbm.lbm_params_default()
    assert (p.Nx, p.Ny, p.eq_order, p.precision) == (1, 64, 2, 0)
    assert (p.u_wall[0], p.u_wall[1], p.seed) == (-0.1, 0.1, 7)
    h = lbm.lbm_lattice_create(37)
    try:
        bad = lbm.lbm_params_default()
        bad.Ny = 5                        # fewer rows than two ghost depths
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_solver_required_bytes(h, bad)
        assert ei.value.status == lbm.LBM_EINVAL
        bad = lbm.lbm_params_default()
        bad.eq_order = 5
        with pytest.raises(lbm.LBMError):
            lbm.lbm_solver_required_bytes(h, bad)
        bad = lbm.lbm_params_default()
        bad.Kn = float("nan")
        with pytest.raises(lbm.LBMError):
            lbm.lbm_solver_required_bytes(h, bad)
        # the large-grid workload: two FP32 state buffers of 37 x 2048 rows of 4
        # x-tiles of 1056 elements, FP64 staging planes, reduction scratch
        p = lbm.lbm_params_default()
        p.Nx, p.Ny, p.precision = 4096, 2048, lbm.LBM_FP32
        n = lbm.lbm_solver_required_bytes(h, p)
        assert 2 * 37 * 2048 * 4224 * 4 < n < 2 * 37 * 2048 * 4224 * 4 + 7 * 4096 * 2048 * 8 + (1 << 20)
        # the largest buffer the kernels' 32-bit offsets address (8 tiles of
        # 1056: 37 * 6870 * 8448 < 2^31 elements), and one past it
        p.Nx, p.Ny = 8192, 6870
        lbm.lbm_solver_required_bytes(h, p)
        p.Ny = 6871
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_solver_required_bytes(h, p)
        assert ei.value.status == lbm.LBM_EINVAL
    finally:
        lbm.lbm_lattice_destroy(h)


def test_bf16_formats_memory_and_checks(lbm):
    # BF16SHIFT stores the FP32 format's deviations d = f - w in BF16 and has
    # no density plane: its requirement is BF16DEV's less the two FP32 planes
    # (one row of 4224 padded elements per row and buffer at 4096 x 2048); the
    # staged kernel is not built for it, and no precision follows it
    h = lbm.lbm_lattice_create(37)
    try:
        p = lbm.lbm_params_default()
        p.Nx, p.Ny, p.eq_order, p.thermal = 4096, 2048, 4, 1
        p.precision = lbm.LBM_BF16DEV
        dev = lbm.lbm_solver_required_bytes(h, p)
        p.precision = lbm.LBM_BF16SHIFT
        shift = lbm.lbm_solver_required_bytes(h, p)
        assert dev - shift == 2 * 2048 * 4224 * 4
        p.precision = lbm.LBM_FP32
        assert lbm.lbm_solver_required_bytes(h, p) - shift == 2 * 37 * 2048 * 4224 * 2
        p.precision, p.kernel = lbm.LBM_BF16SHIFT, lbm.LBM_KERNEL_STAGED
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_solver_required_bytes(h, p)
        assert ei.value.status == lbm.LBM_EINVAL
        p.precision, p.kernel = lbm.LBM_BF16SHIFT + 1, lbm.LBM_KERNEL_AUTO
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_solver_required_bytes(h, p)
        assert ei.value.status == lbm.LBM_EINVAL
    finally:
        lbm.lbm_lattice_destroy(h)


def test_status_strings(lbm):
    assert lbm.lbm_status_string(0) == "ok"
    assert lbm.lbm_status_string(4) == "not converged"
    assert lbm.lbm_version()[0] == 0


def test_server_request_validation(lbm):
    r = lbm.make_request("D2Q37", 2048, 0.05, 0.3)
    assert lbm.lbm_request_bytes(r) == (2 * 37 * 2048 + 2 * 2048) * 4
    r = lbm.make_request("D2Q17", 33, 0.05, 0.1)
    n = lbm.lbm_request_bytes(r)
    assert n % 256 == 0 and n >= (2 * 17 * 33 + 2 * 33) * 4
    for bad in (dict(Ny=5), dict(Ny=9000), dict(Kn=0.0), dict(tol=0.0)):
        q = lbm.make_request("D2Q25", 64, 0.1, 0.1)
        for k, v in bad.items():
            setattr(q, k, v)
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_request_bytes(q)
        assert ei.value.status == lbm.LBM_EINVAL
    c = lbm.lbm_server_cfg_default()
    assert (c.max_slots, c.chunk_steps, c.mem_budget_bytes) == (256, 100, 40 << 30)


def test_accommodation_parameter_checks(lbm):
    h = lbm.lbm_lattice_create(25)
    try:
        p = lbm.lbm_params_default()
        assert (p.accom[0], p.accom[1]) == (1.0, 1.0)
        for bad in (-0.1, 1.5, float("nan")):
            p.accom[0] = bad
            with pytest.raises(lbm.LBMError):
                lbm.lbm_solver_required_bytes(h, p)
    finally:
        lbm.lbm_lattice_destroy(h)
    r = lbm.make_request("D2Q25", 32, 0.1, 0.1, accom=(0.5, 2.0))
    with pytest.raises(lbm.LBMError):
        lbm.lbm_request_bytes(r)


def test_custom_lattice_from_tables(lbm):
    ref = lbm.Lattice("D2Q25b")
    perm = np.random.default_rng(3).permutation(ref.Q)
    cus = lbm.Lattice("custom", custom=(ref.e[perm], ref.w[perm], ref.r))
    assert cus.Q == 25 and cus.r == ref.r and cus.ghost_depth == 3 and cus.degree == 7
    assert np.array_equal(cus.e, ref.e) and np.array_equal(cus.w, ref.w)  # library order
    assert cus.verify(7) < 1e-12
    bad = ref.w.copy()
    bad[1] *= 1.001                                  # breaks a shell's symmetry
    with pytest.raises(lbm.LBMError):
        lbm.Lattice("custom", custom=(ref.e, bad, ref.r))
    with pytest.raises(lbm.LBMError):
        lbm.Lattice("custom", custom=(ref.e[:, ::-1] * 2, ref.w, ref.r))   # not the built-in set
    with pytest.raises(lbm.LBMError):
        lbm.Lattice("custom", custom=(ref.e, -ref.w, ref.r))
    # a weight set that is not a quadrature is accepted but its degree says so
    w = np.full(25, 1.0 / 25)
    assert lbm.Lattice("custom", custom=(ref.e, w, ref.r)).degree < 3


def test_binding_covers_every_declaration_with_its_arity(lbm):
    # every function include/lbm.h declares has a ctypes signature in the
    # binding with the same number of parameters (marshalling only)
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = {}
    for m in re.finditer(r"\b(?:const char\s*\*|int|void|double|int32_t|int64_t|size_t)\s*\**\s*"
                         r"(lbm_\w+)\s*\(([^)]*)\)\s*;", src, flags=re.S):
        params = m.group(2).strip()
        decls[m.group(1)] = 0 if params in ("", "void") else len(params.split(","))
    assert len(decls) >= 40 and set(decls) == set(declared_symbols())
    for name, n in decls.items():
        assert name in lbm._SIGS, name
        assert len(lbm._SIGS[name][0]) == n, (name, n, len(lbm._SIGS[name][0]))


def test_struct_layouts_match_the_header(lbm, tmp_path):
    # every struct the binding mirrors has the header's size and field offsets
    # (a C program compiled against include/lbm.h prints them)
    import ctypes
    import subprocess
    structs = ["lbm_params", "lbm_stats", "lbm_request", "lbm_result", "lbm_server_cfg",
               "lbm_server_metrics", "lbm_server_tuning"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', "int main(void) {"]
    for st in structs:
        py = getattr(lbm, st)
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for name, _ in py._fields_:
            lines.append(f'printf("{st}.{name} %zu\\n", offsetof({st}, {name}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    for st in structs:
        py = getattr(lbm, st)
        assert int(got[st]) == ctypes.sizeof(py), st
        for name, _ in py._fields_:
            assert int(got[f"{st}.{name}"]) == getattr(py, name).offset, (st, name)


def test_binding_constants_match_the_header(lbm):
    # every integer constant include/lbm.h defines (status codes, lattices,
    # storage formats, kernels, rounding and start modes) has the same value in
    # the binding
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    consts = {m.group(1): int(m.group(2))
              for m in re.finditer(r"^#define\s+(LBM_\w+)\s+(-?\d+)\b", src, flags=re.M)}
    assert len(consts) >= 27 and "LBM_BF16SHIFT" in consts
    for name, v in consts.items():
        assert getattr(lbm, name) == v, name
    assert lbm.PRECISION == {"fp64": lbm.LBM_FP64, "fp32": lbm.LBM_FP32,
                             "bf16dev": lbm.LBM_BF16DEV, "bf16shift": lbm.LBM_BF16SHIFT}
