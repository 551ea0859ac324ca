"""Seeded synthetic inputs for the layer-potential workloads.

This package only *describes* problems: curves discretised into Gauss-Legendre
panels, densities at the panel nodes and target points.  It holds none of the
evaluation method's arithmetic (no centres, trees, expansions or quadrature of
the layer potentials); both the CUDA path and the CPU oracle consume what it
produces.
"""
from .starfish import (  # noqa: F401
    Curve,
    discretize,
    starfish_c1,
    starfish_grid,
    unit_circle,
    small_grid,
    random_fourier_curves,
    order_training_curves,
    order_training_problem,
)
