"""Seeded synthetic inputs for the muffin-tin H/S generator.

This package is shared by the CUDA path, its tests, the benchmark and the
oracle's tests. It only draws the problem statement (cell, plane-wave list,
atoms, radial boundary data, radial integrals); it contains none of the
arithmetic that builds A, B, T, H or S.
"""
from .synth import (  # noqa: F401
    AtomType,
    System,
    Workload,
    make_config,
    make_system,
    kpoint_list,
    reciprocal,
    shift_energies,
    CONFIG_NAMES,
)
