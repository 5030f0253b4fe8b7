"""Seeded synthetic multispectral manuscript cubes.

This module only draws inputs: band cubes, ground-truth class maps and
training label maps.  It holds none of the Canonical Variates Analysis
arithmetic, so both the FP64 oracle and the CUDA path can take their inputs
from it without sharing any of the method's code.
"""
from .cubes import (  # noqa: F401
    Workload,
    make_workload,
    named_workload,
    batch_workloads,
    WORKLOADS,
)
