"""Lint: device code reads the compile-time lattice tables (Lat<Q>::ex / ey /
sh / e2) with a variable index only inside loops marked `#pragma unroll`
(whose index is a constant after unrolling), with a template parameter, or
with a `constexpr int` index (the StaticFor / PairLoop compile-time loops).

A table lookup in a loop the compiler did not unroll returned wrong indices on
sm_103a (out-of-bounds reads in the batched kernel); host code builds any table
that device code needs at run time and ships it as data."""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1209_5201_gb300", "csrc")
CALL = re.compile(r"\bL::(ex|ey|sh|e2)\(\s*([A-Za-z_]\w*)\s*\)")


def test_lattice_table_lookups_are_compile_time():
    bad = []
    for fn in sorted(os.listdir(CSRC)):
        if not fn.endswith((".cuh", ".cu")):
            continue
        lines = open(os.path.join(CSRC, fn)).read().splitlines()
        for i, line in enumerate(lines):
            for m in CALL.finditer(line):
                var = m.group(2)
                if var.isupper() or var in ("A",):       # template parameter
                    continue
                # nearest enclosing declaration of the index: a compile-time
                # constant, or a loop header that must be marked for unrolling
                j = i
                decl = re.compile(r"for\s*\(\s*int\s+%s\b|constexpr\s+int\s+%s\s*=" % (var, var))
                while j >= 0 and not decl.search(lines[j]):
                    j -= 1
                ok = j >= 0 and ("constexpr" in lines[j] or (j > 0 and "#pragma unroll" in lines[j - 1]))
                if not ok:
                    bad.append(f"{fn}:{i + 1}: {line.strip()}")
    assert not bad, "lattice-table lookups outside unrolled loops:\n" + "\n".join(bad)
