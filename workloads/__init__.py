"""Seeded synthetic inputs for the VIP fractional-step solver.

This package generates node sets (coordinates, node kinds, boundary normals,
local spacing) and initial/boundary states shaped like the flows of Park, Jo
and Choe, "Virtual Interpolation Point Method for Viscous Flows in Complex
Geometries" (Sec. 5: decaying vortices, lid-driven cavity, flow past a
circular and a bumpy cylinder, triangular cavity).

It is the one module that both the FP64 oracle and the CUDA path consume.  It
holds none of the method's arithmetic: no weight function, no moving
least-squares fit, no operator and no time stepping -- only geometry and the
initial data of each workload.
"""
from .geometry import (  # noqa: F401
    KIND_INTERIOR, KIND_WALL, KIND_SLIP, KIND_OUTLET,
    NodeSet, periodic_box, cavity, channel_body, triangle_cavity, wedge_cavity,
    triangle_batch, taylor_green, workload,
)
from .geometry3d import NodeSet3, box3d, sphere_in_box3d  # noqa: F401
