"""Seeded synthetic H-matrix EFIE problems (mesh, RWG, Eq. 7 entries, octree, Eq. 8
partition, ACA).  Input generation only: shared by the solver library's tests and
benchmark and by the CPU oracle; holds none of the preconditioner or Krylov arithmetic."""
from .builder import (SPECS, Problem, build, build_lib, EntryEvaluator, plane_wave_rhs, far_field,
                      bistatic_rcs, quadrature_rule, potential_integrals, recompress, make_mesh)
from .mesh import RWG, icosphere, plate
