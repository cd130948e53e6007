"""Pins for the oracle's two-level ORAS (coarse space of Section 7).

* with the fine mesh as its own coarse mesh the prolongation is the identity
  (a Whitney function's tangential integral along its own edge is 1, along the
  other edges 0, and it is constant along an edge, so the midpoint rule is exact);
* a constant field is reproduced: the coarse DOFs of a constant field F
  prolong to its fine DOFs F . (x_hi - x_lo) (Whitney elements contain the
  constants), on two different meshes of the cube;
* with the fine mesh as coarse mesh, Q = A^{-1} and the deflated two-level
  preconditioner is exact: FGMRES stops after one step;
* on the chamber, FGMRES with the two-level preconditioner reaches the direct
  solution.
"""

import numpy as np

import oracle as O
from oracle import dd
from synthetic import antenna_array, chamber_eps, chamber_mesh, cube_eps, cube_mesh, ring_antennas

FREQ = 1e9


def _prob(mesh, eps, nsub):
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    A = O.assemble_system(mesh.xyz, topo, eps, FREQ).tocsr()
    part = dd.rcb_partition(mesh.xyz, mesh.tet, nsub)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    oras = dd.ORAS(dec, dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ))
    return topo, A, oras


def test_self_prolongation_is_identity_and_two_level_exact():
    mesh = chamber_mesh(8, 7)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    topo, A, oras = _prob(mesh, eps, 4)
    cs = dd.CoarseSpace(mesh.xyz, topo, mesh.xyz, topo, A, oras)
    I = cs.P.toarray()
    assert np.abs(I - np.eye(topo.ndof)).max() <= 1e-12
    b = np.zeros(topo.ndof, dtype=np.complex128)
    b[7] = 1.0
    x, it, _ = dd.fgmres(A, b, cs.apply, rtol=1e-10)
    assert it == 1


def test_constant_field_is_reproduced():
    fine, coarse = cube_mesh(5), cube_mesh(3)
    ft = O.build_topology(fine.tet, fine.bface_tag, fine.nv, 1)
    ct = O.build_topology(coarse.tet, coarse.bface_tag, coarse.nv, 1)
    A = O.assemble_system(fine.xyz, ft, cube_eps(fine.xyz, fine.tet), FREQ).tocsr()
    cs = dd.CoarseSpace(fine.xyz, ft, coarse.xyz, ct, A, None)
    F = np.array([0.3, -1.1, 0.7])

    def dofs(xyz, topo):
        out = np.zeros(topo.ndof)
        e = topo.edges
        d = np.full(e.shape[0], -1, dtype=np.int64)
        d[topo.tet_edges.ravel()] = topo.tet_dofs[:, :6].ravel()
        ok = d >= 0
        out[d[ok]] = (xyz[e[ok, 1]] - xyz[e[ok, 0]]) @ F
        return out

    assert ft.ndof == int((~ft.pec_edge).sum())  # impedance cube: nothing removed
    f = dofs(fine.xyz, ft)
    assert np.abs(cs.P @ dofs(coarse.xyz, ct) - f).max() <= 1e-12 * np.abs(f).max()


def test_two_level_reaches_direct_solution():
    mesh = chamber_mesh(10, 9)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    topo, A, oras = _prob(mesh, eps, 8)
    cm = chamber_mesh(6, 5, jitter=0.0, permute=False)
    ct = O.build_topology(cm.tet, cm.bface_tag, cm.nv, 1)
    cs = dd.CoarseSpace(mesh.xyz, topo, cm.xyz, ct, A, oras)
    tx = antenna_array(ring_antennas(2, radius=0.08))
    d, s = O.antenna_edges(mesh.xyz, topo, tx)
    B = O.build_rhs(topo.ndof, d, s, tx[:, 6] + 1j * tx[:, 7], FREQ)
    U = O.direct_solve(A, B)[0]
    for c in range(B.shape[1]):
        x, it, _ = dd.fgmres(A, B[:, c], cs.apply, rtol=1e-10)
        assert np.linalg.norm(x - U[:, c]) <= 1e-8 * np.linalg.norm(U[:, c])
