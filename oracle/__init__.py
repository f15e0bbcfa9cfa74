"""Plain FP64 CPU oracle of the KFBI layer-potential apply and the Dirichlet BVP solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its Python
binding) may import, call or link anything in this package.  Only the tests, the
``smoke()`` check in ``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code with the CUDA path; the only common
module is ``kfbi_workloads`` (seeded input generators, no method arithmetic).

Every function follows the method as the paper states it (Sec. 2.1-2.2, Alg. 1-5),
with the readings of unstated details written out in each docstring.

Each function is pinned to facts outside itself (tests/test_oracle_pins.py,
tests/test_oracle3d_pins.py): box solves to dense LU and exact eigen-pairs; the applies to
the double layer of a constant (the indicator of Omega), to closed-form box double-layer
potentials on a circle (also on circles grazing a grid row, which exercises the grazing
rule of Geometry2D) and on a sphere (through the 3-D apply and its fitted-density split),
to exactly reproduced piecewise quadratics, and to the spectrum of the continuous operator
(the 3-D split); GMRES and Richardson to a dense solve of the assembled operator; the BVP
to second-order convergence on manufactured solutions; error_norms to hand-computed values.
"""
from .kfbi2d import (GeometryError, Geometry2D, jumps_cartesian, box_solve_dst,
                     box_solve_dense, correct_rhs, interpolate_plus, apply_interface,
                     apply_double_layer, apply_volume, combined_grid_solution, gmres,
                     richardson, solve_bvp, error_norms, lagrange_basis,
                     interpolate_plus_grad, apply_interface_dn, apply_single_layer,
                     apply_single_layer_dn, apply_volume_dn, solve_neumann_bvp)

__all__ = ["GeometryError", "Geometry2D", "jumps_cartesian", "box_solve_dst",
           "box_solve_dense", "correct_rhs", "interpolate_plus", "apply_interface",
           "apply_double_layer", "apply_volume", "combined_grid_solution", "gmres",
           "richardson", "solve_bvp", "error_norms", "lagrange_basis",
           "interpolate_plus_grad", "apply_interface_dn", "apply_single_layer",
           "apply_single_layer_dn", "apply_volume_dn", "solve_neumann_bvp"]
from . import kfbi3d  # noqa: E402  (3-D oracle: oracle.kfbi3d)
