"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This package holds no arithmetic of the discretisation itself: it only turns
node coordinates into initial states (a balanced warm-core vortex with seeded
potential-temperature noise, or random smooth perturbations) and describes the
benchmark workloads.  Both the CUDA library and the CPU oracle receive the
arrays it produces; neither is imported here.
"""
from .vortex import VortexSpec, vortex_state, splitmix64_uniform  # noqa: F401
from .workloads import WORKLOADS, Workload  # noqa: F401
