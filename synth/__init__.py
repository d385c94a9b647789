"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This package holds input generators only (geometry, random numbers, job
lists, parameter presets).  It contains none of the method's arithmetic and
imports neither the oracle nor the CUDA package; both of those consume what
it produces.
"""
from .workloads import *  # noqa: F401,F403
