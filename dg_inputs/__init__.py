"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds meshes (vertex coordinates, element-to-vertex lists and
face connectivity) and initial states evaluated at caller-supplied node
coordinates.  It contains none of the discontinuous Galerkin arithmetic: no
reference-element operators, no fluxes, no time stepping.  Both sides of every
parity test take their inputs from here and nothing else.
"""
from .meshes import periodic_square, ogrid_cylinder, Mesh
from .states import (isentropic_vortex, free_stream, splitmix64_uniform,
                     perturb, shu_vortex_params)
from .sweeps import viv_sweep, sweep_mesh

__all__ = ["periodic_square", "ogrid_cylinder", "Mesh", "isentropic_vortex",
           "free_stream", "splitmix64_uniform", "perturb", "shu_vortex_params",
           "viv_sweep", "sweep_mesh"]
