"""Seeded synthetic inputs for the lat-lon pressure-correction system.

This package draws the random fields and lays out the finite-volume
geometry of a latitude-longitude shell grid.  It computes the coefficient
arrays and right-hand sides that BOTH the CPU oracle and the CUDA library
take as inputs; it holds none of the multigrid method's arithmetic
(no operator application, no smoother, no transfers, no solver).
"""
from .latlon import (  # noqa: F401
    ShellGrid,
    make_ns_problem,
    make_problem,
    box_filter_3pt,
    WORKLOADS,
    workload_seed,
)
