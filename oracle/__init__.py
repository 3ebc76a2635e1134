"""Plain, slow FP64 CPU oracle for direct ghost-cell reconstruction.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA
library and does not import it; both sides receive the same seeded inputs
from the input generator, which holds none of the method's arithmetic.

What it computes (paper: "Stable, Compact, and Direct Ghost-Cell
Reconstruction: A Non-Iterative Approach for Embedded-Boundary Methods"):

* ``geometry``     -- Cartesian grid, analytic bodies, signed normal distance
                      psi, boundary point S and unit normal n (Sec. 3.1,
                      Eq. signed_distance).
* ``classify``     -- fluid/solid tags, CGC / HGC / CGC_ES ghost placement
                      (Sec. 3.1, Eqs. delta_n, HGC_criterion; Sec. 7,
                      Eq. stencil_anisotropic), stencil members.
* ``levels``       -- dependency DAG and topological levels L_1..L_n
                      (Sec. 3.2), by memoised depth-first longest path.
* ``reconstruct``  -- closed-form Dirichlet / Neumann reconstruction in 2D and
                      3D (Secs. 4-5, Eqs. phi_G_Dir_2d, phi_G_Neu_2d,
                      phi_G_Dir_3d, phi_G_Neu_3d), the Vandermonde solve of
                      Appendix A used to pin them, and the level-by-level fill.
* ``surface``      -- boundary value, normal derivative and Cartesian gradients
                      at S (Sec. 6, Eqs. derivative_bilinear,
                      normal_derivative_trilinear, derivative_trilinear_x/y/z)
                      and the pressure / viscous force sums.
* ``tiles``        -- the fill run by rectangular tiles (subdomains) that
                      exchange, after each level, only the ghosts of that level
                      read by another tile's stencil (Sec. 3.2, distributed
                      memory), and the halo volume of a conventional exchange.
* ``adjoint``      -- gradient of (drag, lift) with respect to the fluid field
                      values and the boundary data, and the vector-Jacobian
                      product of the fill, from the explicit sparse matrix of
                      the (linear) map.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` except
the force quadrature weights, which the paper does not specify ("parity
unpinned" against the paper; see ``surface.face_weights``).
"""

from .geometry import Grid, Body, closest_point, inside
from .classify import classify, Classification, stencil_offsets, EBRError, ghost_x2
from .levels import build_levels, Levels
from .reconstruct import (fill, ghost_weights, ghost_value, vandermonde_ghost_value,
                          DIRICHLET, NEUMANN)
from .surface import boundary_quantities, forces, face_weights
from .adjoint import adjoint_gradient, fill_vjp, linear_map
from . import tiles

__all__ = [
    "Grid", "Body", "closest_point", "inside",
    "classify", "Classification", "stencil_offsets", "EBRError", "ghost_x2",
    "build_levels", "Levels",
    "fill", "ghost_weights", "ghost_value", "vandermonde_ghost_value",
    "DIRICHLET", "NEUMANN",
    "boundary_quantities", "forces", "face_weights",
    "adjoint_gradient", "fill_vjp", "linear_map",
]
