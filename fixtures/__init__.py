"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This package holds random draws and the workload generators only (random-walk
and embedding-like series, noise-perturbed query sets, weight initialisations,
SGD shuffles).  It contains none of the search method's arithmetic.
"""
from .generators import *  # noqa: F401,F403
