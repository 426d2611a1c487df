"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the FP64 oracle.

This package holds no arithmetic of the method itself: it only draws the
matrices and vectors a WSSR step consumes (planted-spectrum O, drift, the
gradient g, the random start subspace, MLP weights and electron samples).
"""
from .workloads import *  # noqa: F401,F403
