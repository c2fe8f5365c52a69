"""Seeded synthetic inputs for the DMPT/TDA Bethe-Salpeter hot path.

This package draws the *inputs* of the method (cell, plane-wave sphere, model
local potential, occupied orbitals and energies, PDEP basis and eigenvalues,
pair-selection rule). It contains none of the Liouville-operator, screened
integral or Davidson arithmetic: the CPU oracle (``oracle/``) and the CUDA
library both consume what it writes, and neither imports the other.
"""
from .instance import (Instance, sphere_half, make_tiny, make_localized,  # noqa: F401
                       make_config, CONFIGS)
