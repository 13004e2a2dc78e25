"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds random draws and workload parameters only: no step of the
method's arithmetic lives here, so the oracle and the CUDA path can both
consume the same inputs without sharing any numerics.
"""
from .seeded import (  # noqa: F401
    Workload,
    WORKLOADS,
    psi_coefficients,
    temperature_coefficients,
    ensemble_members,
    random_state,
)
