"""Seeded synthetic inputs for the multi-block Euler residual and RK stage.

This module builds grids, initial states, manufactured-solution source terms
and block-connection tables.  It is the only code shared by the CPU oracle
(``oracle/``) and the CUDA library (``paper_2012_02925_gb300``): it holds the
problem definitions (geometry, initial/boundary data, the manufactured PDE
source) and none of the discrete method's arithmetic (no metrics, no
reconstruction, no limiter, no Riemann flux, no residual, no time stepping).

Layout conventions used everywhere:

* A block has interior cells ``i in [0,ni), j in [0,nj), k in [0,nk)`` and
  ``G = 2`` ghost layers on every side.  A ghosted state array has shape
  ``(5, nk+4, nj+4, ni+4)`` (variable, k, j, i; i fastest), cell ``(i,j,k)`` at
  ``[:, k+2, j+2, i+2]``.  Variables are the conserved
  ``(rho, rho*u, rho*v, rho*w, rho*E)`` (paper Section 2, vector Q).
* Nodes of a curvilinear block have shape ``(nk+1, nj+1, ni+1, 3)``.
* The packed multi-block state is the concatenation of the ghosted arrays of
  all blocks, flattened in block order.
"""
from .core import (GAMMA, GHOST, BlockDesc, Connection, Problem, prim_to_cons,
                   ghosted_shape, pack_state, unpack_state, packed_size,
                   interior_view, nominal_dt, FACE_IMIN, FACE_IMAX, FACE_JMIN,
                   FACE_JMAX, FACE_KMIN, FACE_KMAX, periodic_connections,
                   conn_array, BCPatch, bc_arrays, BC_FIXED, BC_SUPERSONIC_INFLOW,
                   BC_EXTRAPOLATE, BC_SLIP_WALL, BC_FARFIELD, BC_NOSLIP_WALL, BC_NAMES)
from .workloads import (vortex_2d, mms_3d, multiblock_batched, large_periodic,
                        perturbed_nodes, uniform_3d, split_problem_i,
                        mms_primitives, mms_source, rotated_split_problem,
                        inlet_2d, ellipse_ogrid, channel_uniform, table_state,
                        INLET_INFLOW, AIRFOIL_FARFIELD, WING_FARFIELD, mms_periodic_3d,
                        mms_viscous_divergence, viscosity)

__all__ = [
    "GAMMA", "GHOST", "BlockDesc", "Connection", "Problem", "prim_to_cons",
    "ghosted_shape", "pack_state", "unpack_state", "packed_size",
    "interior_view", "nominal_dt", "FACE_IMIN", "FACE_IMAX", "FACE_JMIN",
    "FACE_JMAX", "FACE_KMIN", "FACE_KMAX", "periodic_connections", "conn_array",
    "BCPatch", "bc_arrays", "BC_FIXED", "BC_SUPERSONIC_INFLOW", "BC_EXTRAPOLATE",
    "BC_SLIP_WALL", "BC_FARFIELD", "BC_NOSLIP_WALL", "BC_NAMES",
    "vortex_2d", "mms_3d", "multiblock_batched", "large_periodic",
    "perturbed_nodes", "uniform_3d", "split_problem_i", "mms_primitives",
    "mms_source", "rotated_split_problem", "inlet_2d", "ellipse_ogrid",
    "channel_uniform", "table_state", "INLET_INFLOW", "AIRFOIL_FARFIELD", "WING_FARFIELD", "mms_periodic_3d", "mms_viscous_divergence", "viscosity",
]
