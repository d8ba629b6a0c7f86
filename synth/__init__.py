"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package produces *inputs only*: tetrahedral gel meshes, rigid indenter
surface meshes, indenter pose schedules and sensor pixel grids, all drawn from
a counter-based generator (splitmix64) so that every test and benchmark input
is reproducible from a seed.  It contains none of the method's arithmetic
(no deformation gradient, stress, barrier, contact or binning code): the oracle
and the CUDA library each implement those on their own.

The shapes stand in for the paper's workloads (Sec. IV-A: a GelSight-Mini pad
of 1,920 tets; Sec. IV-E: GelSight Mini / DIGIT / 9DTact sensors pressed by
spheres and cylinders); no dataset is used.
"""
from .rng import SplitMix64  # noqa: F401
from . import meshes, indenters, workloads  # noqa: F401
