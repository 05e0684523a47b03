"""Host logic of the batched path's column split (batch_internal.h), compiled
as a small C++ program and checked for every height the server accepts:
the cluster size it picks is a power of two within the device's and the CTA
budget's limits, every CTA of a split gets whole 32-row residual chunks and at
least 32 rows (the last one included), the CTAs cover the column, the split
grows only while a CTA holds more than the requested rows, and the chunks per
launch stay within what the kernel accepts."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1209_5201_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "batch_internal.h"
using namespace lbm;

static int fail(int Ny, int rows, int ctas, int mcl, int cl, const char *what) {
    std::printf("FAIL Ny=%d rows=%d ctas=%d max_cl=%d cl=%d: %s\n", Ny, rows, ctas, mcl, cl, what);
    return 1;
}

int main() {
    const int rows_list[] = {32, 64, 128, 256, 1024, 8192};
    const int ctas_list[] = {1, 2, 3, 4, 8, 16, 304};
    const int mcl_list[] = {8, 16};
    long checked = 0;
    for (int Ny = 6; Ny <= kMaxNy; ++Ny)
        for (int rows : rows_list)
            for (int ctas : ctas_list)
                for (int mcl : mcl_list) {
                    const int cl = batch_cluster_size(Ny, rows, ctas, mcl);
                    if (cl != 1 && cl != 2 && cl != 4 && cl != 8 && cl != 16)
                        return fail(Ny, rows, ctas, mcl, cl, "not a class size");
                    if (cl > mcl || cl > ctas) return fail(Ny, rows, ctas, mcl, cl, "over a limit");
                    if (!batch_split_ok(Ny, cl)) return fail(Ny, rows, ctas, mcl, cl, "unusable split");
                    const int sub = batch_sub_chunks(cl);
                    if (sub < 1 || sub > kMaxSub) return fail(Ny, rows, ctas, mcl, cl, "sub-chunks");
                    if (cl > 1) {
                        const int R = batch_rows_per_cta(Ny, cl);
                        if (R % kResidualChunk) return fail(Ny, rows, ctas, mcl, cl, "partial chunk");
                        if (cl * R < Ny) return fail(Ny, rows, ctas, mcl, cl, "rows not covered");
                        if (Ny - (cl - 1) * R < 32) return fail(Ny, rows, ctas, mcl, cl, "short last CTA");
                    }
                    // a larger usable split within the limits exists only if
                    // this one already meets the requested rows per CTA
                    const int up = cl * 2;
                    if (up <= mcl && up <= ctas && batch_split_ok(Ny, up) &&
                        batch_rows_per_cta(Ny, cl) > rows) {
                        // growing further was allowed; the search must have
                        // stopped only because every larger size up to
                        // max_cl was unusable or over the budget
                        bool any = false;
                        for (int c = up; c <= mcl; c *= 2)
                            any = any || (c <= ctas && batch_split_ok(Ny, c) &&
                                          batch_rows_per_cta(Ny, c) <= rows);
                        if (any) return fail(Ny, rows, ctas, mcl, cl, "stopped early");
                    }
                    ++checked;
                }
    std::printf("OK %ld\n", checked);
    return 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        d = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
        if os.path.exists(os.path.join(d, "cuda_runtime.h")):
            return d
    return None


def test_split_rules_for_every_height(tmp_path):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "split.cpp"
    exe = tmp_path / "split"
    src.write_text(PROGRAM)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout + out.stderr
