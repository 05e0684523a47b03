"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA side.

This module holds no arithmetic of the lattice Boltzmann method: only random
draws and the recipes of the Couette workloads.  Both the oracle and the CUDA
library receive what it produces as plain inputs.

Counter-based generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  The draw for counter k under
seed s is the first output of a SplitMix64 stream seeded with (s XOR k):

    z  = (s ^ k) + 0x9E3779B97F4A7C15
    z  = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z  = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z  =  z ^ (z >> 31)
    U  = (z >> 11) * 2^-53            in [0, 1)

The CUDA library implements the same published generator on the device for
its own initialisation; tests compare the two.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

LATTICES = ("D2Q17", "D2Q25", "D2Q37")


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) ^ np.asarray(k, dtype=np.uint64)) + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, k: np.ndarray) -> np.ndarray:
    return (splitmix64(seed, k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def rho_field(Nx: int, Ny: int, amp: float = 0.0, seed: int = 7, rho0: float = 1.0):
    """rho(x, j) = rho0 (1 + amp (2U - 1)), U drawn at counter j*Nx + x."""
    if amp == 0.0:
        return np.full((Ny, Nx), rho0, dtype=np.float64)
    k = np.arange(Ny * Nx, dtype=np.uint64).reshape(Ny, Nx)
    return rho0 * (1.0 + amp * (2.0 * uniform01(seed, k) - 1.0))


class _Stream:
    """Sequential uniform draws from the counter generator (for workload recipes)."""

    def __init__(self, seed: int):
        self.seed = seed
        self.k = 0

    def u(self) -> float:
        v = float(uniform01(self.seed, np.uint64(self.k)))
        self.k += 1
        return v


@dataclass
class Instance:
    """One Couette solve: Nx = 1 column, walls at -U_w (bottom) and +U_w (top)."""
    lattice: str
    Ny: int
    Kn: float
    U_w: float
    T_w: float
    eq_order: int
    thermal: bool
    arrival: float = 0.0


def _order_for(lat: str) -> tuple[int, bool]:
    # D2Q17 / D2Q25: isothermal second order; D2Q37: thermal fourth order.
    return (4, True) if lat == "D2Q37" else (2, False)


def batched_instances(n: int = 256, seed: int = 7, ny_lo: int = 32, ny_hi: int = 2048,
                      kn_lo: float = 0.01, kn_hi: float = 1.0):
    """Batched workload: lattice uniform over the three sets, Ny uniform integer
    in [ny_lo, ny_hi], Kn log-uniform in [kn_lo, kn_hi], U_w uniform in
    [0.05, 0.3], T_w uniform in [0.9, 1.1] (used by the thermal lattice only)."""
    s = _Stream(seed)
    out = []
    for _ in range(n):
        lat = LATTICES[min(int(s.u() * 3), 2)]
        Ny = ny_lo + min(int(s.u() * (ny_hi - ny_lo + 1)), ny_hi - ny_lo)
        Kn = math.exp(math.log(kn_lo) + s.u() * (math.log(kn_hi) - math.log(kn_lo)))
        U_w = 0.05 + 0.25 * s.u()
        T_w = 0.9 + 0.2 * s.u()
        order, thermal = _order_for(lat)
        out.append(Instance(lat, Ny, Kn, U_w, T_w if thermal else 1.0, order, thermal))
    return out


def serving_requests(n: int = 10000, seed: int = 11, rate: float = 200.0,
                     ny_lo: int = 32, ny_hi: int = 4096, kn_lo: float = 0.005,
                     kn_hi: float = 1.0):
    """Serving workload: Poisson arrivals at `rate` per second; lattice uniform,
    Ny log-uniform in [ny_lo, ny_hi] (rounded), Kn log-uniform in
    [kn_lo, kn_hi], U_w uniform in [0.05, 0.3], T_w = 1."""
    s = _Stream(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += -math.log(1.0 - s.u()) / rate
        lat = LATTICES[min(int(s.u() * 3), 2)]
        Ny = int(round(math.exp(math.log(ny_lo) + s.u() * (math.log(ny_hi) - math.log(ny_lo)))))
        Kn = math.exp(math.log(kn_lo) + s.u() * (math.log(kn_hi) - math.log(kn_lo)))
        U_w = 0.05 + 0.25 * s.u()
        order, thermal = _order_for(lat)
        out.append(Instance(lat, Ny, Kn, U_w, 1.0, order, thermal, arrival=t))
    return out
