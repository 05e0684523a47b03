"""Oracle lattice tables: velocity sets xi = {c_a, w_a} (Sec. II, after Eq. (3)).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Shares nothing with the
CUDA library, which derives its own tables in C++.

A lattice is a set of integer vectors e_a with weights w_a and a scale r, so
that c_a = r e_a.  The weights and r make the discrete sums reproduce the
moments of the unit Gaussian weight function:

    sum_a w_a (r e_ax)^(2p) (r e_ay)^(2q) = (2p-1)!! (2q-1)!!

for every monomial up to the lattice's degree (odd moments vanish by the
symmetry of each shell).  This is the quadrature requirement behind Eq. (4):
the truncated Maxwellian's moments are only reproduced when the sums above are
exact to the order the expansion needs.

  * D2Q17 (Shan, Yuan & Chen 2006, used in Sec. IV): shells (0,0), (1,0),
    (1,1), (2,2), (3,0); degree 7.  Six unknowns (five shell weights and r^2)
    against the six even-moment conditions of degree <= 6; solved by Newton.
  * D2Q25: tensor product of the D1Q5 set {0, +-1, +-3}; 1-D moments m0, m2,
    m4, m6 give w3 = (3 - s)/(144 s^2), w1 = 1/(2s) - 9 w3 and
    3 s^2 - 10 s + 5 = 0 for s = r^2.  Root 0 is s = (5 + sqrt 10)/3 (larger
    rest weight), root 1 is s = (5 - sqrt 10)/3.
  * D2Q37 (the degree-9 set of the paper's cited lattice solution, Shan 2010):
    shells (0,0), (1,0), (1,1), (2,0), (2,1), (2,2), (3,0), (3,1); nine
    unknowns (eight shell weights and r^2) against the nine even-moment
    conditions of degree <= 8; solved by Newton.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class OracleLattice:
    name: str
    e: np.ndarray          # (Q, 2) int32
    w: np.ndarray          # (Q,) float64
    r: float

    @property
    def Q(self) -> int:
        return int(self.e.shape[0])


def _shell(a: int, b: int) -> list[tuple[int, int]]:
    """All sign/axis permutations of (a, b)."""
    pts = set()
    for sx in (1, -1):
        for sy in (1, -1):
            pts.add((sx * a, sy * b))
            pts.add((sx * b, sy * a))
    return sorted(pts)


def _dfact(n: int) -> int:
    return 1 if n <= 0 else n * _dfact(n - 2)


def _newton_shell_system(shells, conds, guess):
    """Solve sum_k w_k S_pq(k) s^(p+q) = (2p-1)!!(2q-1)!! for (w, s).

    S_pq(k) = sum over shell k of e_x^(2p) e_y^(2q); analytic Jacobian.  The
    residual is evaluated in numpy's extended precision and the float64 Newton
    correction is applied to the extended-precision iterate (iterative
    refinement), so the result is correctly rounded to float64.
    """
    ld = np.longdouble
    pts = [_shell(*s) for s in shells]
    S = np.array([[sum(ex ** (2 * p) * ey ** (2 * q) for ex, ey in pk) for pk in pts]
                  for (p, q) in conds], dtype=ld)
    deg = np.array([p + q for (p, q) in conds], dtype=ld)
    rhs = np.array([_dfact(2 * p - 1) * _dfact(2 * q - 1) for (p, q) in conds], dtype=ld)
    x = np.array(guess, dtype=ld)
    for _ in range(200):
        w, s = x[:-1], x[-1]
        sp = s ** deg
        F = (S @ w) * sp - rhs
        J = np.empty((len(conds), len(x)))
        J[:, :-1] = (S * sp[:, None]).astype(np.float64)
        J[:, -1] = ((S @ w) * deg * s ** (deg - 1)).astype(np.float64)
        dx = np.linalg.solve(J, -F.astype(np.float64))
        x = x + dx.astype(ld)
        if np.max(np.abs(dx)) < 1e-19 * max(1.0, float(np.max(np.abs(x)))):
            break
    return x[:-1].astype(np.float64), x[-1], pts


def _from_shells(name, shells, w_shell, s):
    e, w = [], []
    for k, sh in enumerate(shells):
        for p in _shell(*sh):
            e.append(p)
            w.append(w_shell[k])
    return OracleLattice(name, np.array(e, dtype=np.int32),
                         np.array(w, dtype=np.float64), float(np.sqrt(np.longdouble(s))))


def d2q17() -> OracleLattice:
    shells = [(0, 0), (1, 0), (1, 1), (2, 2), (3, 0)]
    conds = [(0, 0), (1, 0), (2, 0), (1, 1), (3, 0), (2, 1)]
    w, s, _ = _newton_shell_system(shells, conds, [0.4, 0.1, 0.03, 1e-4, 3e-4, 2.7])
    if np.any(w <= 0):
        raise ValueError("D2Q17 Newton converged to a non-positive root")
    return _from_shells("D2Q17", shells, w, s)


def d2q37() -> OracleLattice:
    shells = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1)]
    conds = [(0, 0), (1, 0), (2, 0), (1, 1), (3, 0), (2, 1), (4, 0), (3, 1), (2, 2)]
    w, s, _ = _newton_shell_system(
        shells, conds, [0.23, 0.1, 0.06, 0.01, 0.005, 0.001, 2e-4, 3e-4, 1.4])
    if np.any(w <= 0):
        raise ValueError("D2Q37 Newton converged to a non-positive root")
    return _from_shells("D2Q37", shells, w, s)


def d2q25(root: int = 0) -> OracleLattice:
    # closed form evaluated in extended precision, then rounded
    ld = np.longdouble
    r10 = np.sqrt(ld(10))
    s = (ld(5) + r10) / ld(3) if root == 0 else (ld(5) - r10) / ld(3)
    w3 = (ld(3) - s) / (ld(144) * s * s)
    w1 = ld(1) / (ld(2) * s) - ld(9) * w3
    w0 = ld(1) - ld(2) * w1 - ld(2) * w3
    w1d = {0: w0, 1: w1, 3: w3}
    e, w = [], []
    for ex in (0, 1, -1, 3, -3):
        for ey in (0, 1, -1, 3, -3):
            e.append((ex, ey))
            w.append(float(w1d[abs(ex)] * w1d[abs(ey)]))
    return OracleLattice("D2Q25" if root == 0 else "D2Q25b",
                         np.array(e, dtype=np.int32), np.array(w, dtype=np.float64),
                         float(np.sqrt(s)))


def get(name: str) -> OracleLattice:
    if name == "D2Q17":
        return d2q17()
    if name == "D2Q25":
        return d2q25(0)
    if name == "D2Q25b":
        return d2q25(1)
    if name == "D2Q37":
        return d2q37()
    raise KeyError(name)
