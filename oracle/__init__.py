"""Plain CPU oracle for the microwave-imaging hot path (test infrastructure only).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it; the product
path (the CUDA library and its Python binding) never calls it and shares no
code with it.

What it computes, in complex128, by the plain definitions:

* the edge-element discretisation of the variational problem of Section 2
  (Eq. pbdirectvarf) with lowest-order Nedelec (Whitney) elements and a
  second-order hierarchical Nedelec element, element integrals by numerical
  quadrature built from the basis definitions (``fem``, ``assemble``);
* one linear system per transmitting antenna, A u_j = b_j (Eq. linsys),
  solved by a sparse direct LU (``solve``);
* S-parameters (Eq. sij), the misfit J (Eq. defJ), the adjoint problem
  (Eq. pbadj) and the per-tetrahedron gradient of J (Section 5) (``solve``);
* the one-level ORAS preconditioner (Eq. ORAS) with the partition of unity of
  Section 3.2 (Eq. algebPartUnity, Eq. chi) and a right-preconditioned
  flexible GMRES, used where a direct solve is too large and to check the
  preconditioner's pieces one by one, and a two-level variant with a
  geometric coarse space (Section 7) (``dd``);
* the nodal (P1) permittivity parameter with the gradient penalty and the
  normalised misfit weights of Eq. defJ2 (``p1``);
* block flexible GMRES, one Krylov space shared by the right-hand sides of a
  block (the block methods of Section 7) (``block_gmres``).

Parity status: every function is pinned by the tests under ``tests/`` that run
with ``-m "not gpu"`` (closed forms, the discrete curl-grad identity, symmetry,
a plane-wave manufactured solution with its convergence rate, reciprocity,
finite-difference gradients, the partition-of-unity identity).
"""

from .constants import C0, MU0, k0_of
from .topology import Topology, build_topology
from .fem import element_matrices, face_matrix, basis_at
from .assemble import assemble_system, antenna_edges, build_rhs
from .solve import (
    direct_solve,
    s_matrix,
    misfit,
    adjoint_rhs,
    gradient,
    forward,
    misfit_and_gradient,
)
from . import dd
from . import p1
from . import block_gmres

__all__ = [
    "C0", "MU0", "k0_of", "Topology", "build_topology", "element_matrices", "face_matrix",
    "basis_at", "assemble_system", "antenna_edges", "build_rhs", "direct_solve", "s_matrix",
    "misfit", "adjoint_rhs", "gradient", "forward", "misfit_and_gradient", "dd", "p1",
    "block_gmres",
]
