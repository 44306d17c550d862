"""Seeded synthetic inputs for the Galerkin-FFT solver.

This package holds no arithmetic of the method itself: it only draws the
microstructures (periodic Voronoi grains, crystal orientations, spherical
particles), the random operator inputs and the macroscopic loading histories
that both the CUDA path and the CPU oracle consume.  Every random number is
produced by SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
counter-based generator, so the same seed yields the same arrays on x86 and
Arm hosts.
"""

from .rng import splitmix64, uniform01, standard_normal
from .microstructure import (
    batch_rves,
    periodic_voronoi,
    random_quaternions,
    place_spheres,
    Microstructure,
    polycrystal,
    polycrystal_with_particles,
)
from .loading import (
    cyclic_history,
    ramp_history,
    LoadHistory,
)

__all__ = [
    "splitmix64",
    "uniform01",
    "standard_normal",
    "periodic_voronoi",
    "random_quaternions",
    "place_spheres",
    "Microstructure",
    "polycrystal",
    "polycrystal_with_particles",
    "batch_rves",
    "cyclic_history",
    "ramp_history",
    "LoadHistory",
]
