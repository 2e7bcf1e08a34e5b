"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This package holds none of the method's arithmetic: only a counter-based noise
generator and the workload descriptions (grid sizes, extents, boundary
conditions, physical parameters, seeds, step counts).  Each side builds its own
initial state from these with its own equilibrium.
"""
from .noise import splitmix64, uniform_pm1  # noqa: F401
from .workloads import (  # noqa: F401
    Workload, SOD, DISC_NOISE, VORTEX, ADJOINT, THROUGHPUT, EXPLOSION, RWI, ALL, by_name, scaled,
    GEOM_BOX, GEOM_CYL, BC_PERIODIC, BC_OUTFLOW, BC_EQUILIBRIUM,
    F_MU, F_MV, F_MW, F_EN, F_RHO, F_DMU, F_DMV, F_DMW, F_DRHO,
    RECON_CONSERVATIVE, RECON_PRIMITIVE, RECON_PRESSURE,
)
