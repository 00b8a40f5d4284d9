"""Seeded synthetic inputs for the coupled Maxwell-Schroedinger step.

This package is the only code shared by the CUDA path's tests/bench and the
FP64 oracle.  It draws geometry, molecule positions, orientations and the
species/pulse parameters of each workload; it contains none of the method's
arithmetic (no field update, no propagator, no observable).
"""
from .configs import (  # noqa: F401
    Workload, Species, config0, config1, config2, config3, config4,
    custom, prescribed_drive, species_config0, CONFIG_BUILDERS,
)
