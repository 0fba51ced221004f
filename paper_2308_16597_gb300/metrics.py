"""Throughput and roofline arithmetic used by the benchmark.

MLUPS follows the paper's definition (Sec. 3): mesh size x iteration steps /
(running time x 1e6), where the mesh size counts every node, solid ones
included.
"""
from __future__ import annotations

import math

# Algorithmic HBM bytes of one lattice update of the fused stream-collide:
# 9 flow + 5 temperature populations, each read once and written once.
POPULATIONS = 14


def bytes_per_update(bytes_per_value: int) -> int:
    return POPULATIONS * 2 * bytes_per_value


def mlups(nx: int, ny: int, steps: int, seconds: float) -> float:
    return nx * ny * steps / (seconds * 1e6)


def volume_fraction(n: int, d: float, W: float, H: float) -> float:
    """Solid area fraction of n disks of diameter d in a W x H box (same units)."""
    return n * math.pi * (d / 2) ** 2 / (W * H)


def lattice_viscosity(nu_phys: float, t_star: float, l_star: float) -> float:
    """nu_lu = nu t* / l*^2 (unit conversion of the parameter tables)."""
    return nu_phys * t_star / l_star ** 2


def reynolds_from_archimedes(Ar: float) -> float:
    """Re_p = sqrt(pi/2) Ar for the reference velocity of Sec. 2.6.1."""
    return math.sqrt(math.pi / 2) * Ar


def parallel_efficiency(mlups_n: float, mlups_1: float, n: int) -> float:
    return mlups_n / (n * mlups_1)
