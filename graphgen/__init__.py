"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

Only input construction lives here (graphs as symmetric CSR, query pairs);
nothing in this package computes any part of the resistance-distance method.
"""
from .graph import CSRGraph, to_csr, largest_component, unique_undirected, component_labels  # noqa: F401
from . import families, rng, workloads  # noqa: F401
