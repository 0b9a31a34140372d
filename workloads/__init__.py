"""Seeded synthetic inputs for the sparse Fast Chebyshev Transform.

This package is shared by the CUDA path and by the CPU oracle.  It only draws
random numbers and lays out workload descriptions: supports, L-grid sizes,
single-point nodes and function parameters.  It holds none of the transform's
arithmetic: no DCT, no fold, no solve, no function evaluation.
"""
from .generators import *  # noqa: F401,F403
